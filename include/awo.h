/*
 * awo.h -- C ABI of the GB300 avalanche-overlay library (libawo.so).
 *
 * The library computes the data-parallel hot path of the avalanche overlay of
 * "Data-Driven Compute Overlays for Interactive Geographic Simulation and
 * Visualization" (Komon et al., VIS 2025): per-cell normals and steepness from
 * a DEM, release-cell selection by a steepness range, Monte-Carlo particle
 * trajectories that run downslope under persistence, random variation and a
 * runout-angle stop (Sec. 5.2), and the overlay raster with its mipmap
 * (Sec. 3).  The paper gives the method in prose; the exact arithmetic each
 * call performs is stated beside it below.
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; the
 *    caller allocates and owns every buffer.  The library never allocates;
 *    the only device memory of its own is the fixed 128 KiB scratch array of
 *    awo_release_noalloc (a static device array in the library image).  The
 *    one other state it keeps is a table of texture objects (descriptors of
 *    a caller's DEM buffer: address, width, height; no copy) that
 *    awo_simulate reads its gathers through; see there.
 *  - Rasters are row-major, width x height, index y * width + x; cell (x, y)
 *    has its centre at cell coordinates (u, v) = (x, y).
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream) and returns after enqueueing.
 *  - Errors are returned as awo_status, never trapped.  Argument checks run
 *    on the host before anything is enqueued (AWO_EINVAL); a failed launch
 *    returns AWO_ECUDA.
 *  - Grids: 1 <= width, height <= 65536, width * height < 2^31,
 *    cell_size > 0 and finite.
 *  - Arithmetic is IEEE-754 FP32 with no fused multiply-add in the steps
 *    marked "exact": results are reproducible bit for bit from the formulas.
 */
#ifndef AWO_H
#define AWO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AWO_OK = 0,
    AWO_EINVAL = 1,     /* bad argument: null pointer, size, range, alignment */
    AWO_ENOMEM = 2,     /* workspace smaller than required                    */
    AWO_ECUDA = 3,      /* a CUDA launch or copy failed                        */
    AWO_ETIMEOUT = 4,   /* a bounded device wait gave up                       */
    AWO_EOVERFLOW = 5,  /* a 32-bit count could have wrapped                   */
    AWO_ECANCELLED = 6  /* work was cancelled before completion                */
} awo_status;

typedef struct {
    int32_t width;      /* cells along x (columns)                  */
    int32_t height;     /* cells along y (rows)                     */
    float cell_size;    /* metres per cell                          */
} awo_grid;

/* Trajectory parameters (Sec. 5.2: persistence, random variation, runout
 * angle, particles per release texel). */
typedef struct {
    float mu;             /* tan(runout angle); >= 0                                  */
    float drag_k;         /* velocity-squared drag per metre; >= 0, drag_k*D < 1      */
    float persistence;    /* P in [0, 1]: weight of the previous direction            */
    float randomness;     /* R >= 0: scale of the uniform random variation            */
    float step_scale;     /* s in (0, 1]: horizontal move in cells; D = s*cell_size m  */
    float gravity;        /* m/s^2, > 0; used by awo_finalize                          */
    uint32_t traj_per_cell; /* particles per release cell                             */
    uint32_t max_steps;   /* moves per particle at most                               */
    uint64_t seed;        /* Philox key (low word, high word)                         */
    uint32_t flags;       /* AWO_SIM_* bits below; 0 = accumulate                     */
    int32_t release_log2; /* r in [-3, 3]: the release list holds texels of the release */
                          /* texture at 2^r x the DEM resolution (awo_release_texture); */
                          /* 0: the list holds DEM cells                               */
} awo_sim_params;

/* awo_sim_params.flags: clear d_count and d_maxe (cudaMemsetAsync on the
 * stream) before the particles run, instead of accumulating into them. */
#define AWO_SIM_CLEAR_OUTPUTS 1u

/* Statistics of one awo_simulate call (device layout, 6 x uint64). */
typedef struct {
    uint64_t total_steps; /* recorded moves, summed over particles          */
    uint64_t n_traj;      /* particles run                                   */
    uint64_t n_exited;    /* left the sampling domain                        */
    uint64_t n_capped;    /* reached max_steps                               */
    uint64_t n_stopped;   /* energy reached zero (or zero direction)         */
    uint64_t n_rejected;  /* particles skipped: release index >= W*H (Wr*Hr) */
} awo_sim_stats;

const char* awo_status_string(awo_status s);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int32_t awo_version(void);

/*
 * a0. Decode quantised heights (Sec. 5.2 input DEM; the workloads store
 * decimetres as uint16):  d_h[i] = (float)d_q[i] * scale  (one rounding, exact).
 * d_q: uint16 [height*width]; d_h: float [height*width].  scale > 0, finite.
 */
awo_status awo_decode_u16(const uint16_t* d_q, awo_grid g, float scale, float* d_h, void* stream);

/*
 * a1. Normals and steepness (Sec. 5.1/5.2: "compute the surface normals";
 * release selection evaluates local steepness).  Exact.  For cell (x, y),
 * with xl = max(x-1, 0), xr = min(x+1, W-1) (same for y):
 *   gx = (h[y][xr] - h[y][xl]) / (cs * (xr - xl))   (0 when xr == xl)
 *   gy = (h[yr][x] - h[yl][x]) / (cs * (yr - yl))   (0 when yr == yl)
 *   tan2 = gx*gx + gy*gy                               (tan^2 of the slope)
 *   inv = 1 / sqrt(tan2 + 1);  normal = (-gx*inv, -gy*inv, inv)
 *   slope_deg = atan(sqrt(tan2)) in degrees (NOT exact: within a few ulp).
 * d_h: float [H*W].  d_normal: float [3*H*W], planes nx, ny, nz (nullable).
 * d_tan2: float [H*W] (nullable).  d_slope_deg: float [H*W] (nullable).
 */
awo_status awo_normals(const float* d_h, awo_grid g, float* d_normal, float* d_tan2,
                       float* d_slope_deg, void* stream);

/*
 * a0 + a1 in one pass: exactly awo_decode_u16(d_q, g, scale, d_h) followed
 * by awo_normals(d_h, g, d_normal, d_tan2, d_slope_deg), with the heights
 * decoded where the normals read them, so d_h is written once and never read
 * back.  With all three outputs null it is awo_decode_u16.  Arguments,
 * ranges and errors as in the two calls.
 */
awo_status awo_normals_u16(const uint16_t* d_q, awo_grid g, float scale, float* d_h, float* d_normal,
                           float* d_tan2, float* d_slope_deg, void* stream);

/*
 * b. Release cells (Sec. 5.2: a texel is a potential release point when its
 * local steepness lies in the user's range; the node outputs a binary map).
 * Exact.  T = tan(deg * pi / 180)^2 is computed on the host in double and
 * rounded to float once for each bound; cell i is selected iff
 * T_lo <= d_tan2[i] <= T_hi.
 * Outputs: d_mask uint8 [H*W] (0/1, nullable); d_cells uint32 [capacity H*W]:
 * indices of the selected cells in increasing order; d_n: one uint32, the
 * number selected.  Requires 0 <= lo_deg <= hi_deg < 90.
 * Workspace: d_ws of at least awo_release_workspace_bytes(g) bytes, 16-byte
 * aligned, contents undefined on entry and exit.
 */
size_t awo_release_workspace_bytes(awo_grid g);
awo_status awo_release(const float* d_tan2, awo_grid g, double slope_lo_deg, double slope_hi_deg,
                       uint8_t* d_mask, uint32_t* d_cells, uint32_t* d_n,
                       void* d_ws, size_t ws_bytes, void* stream);

/*
 * b'. Release cells from a caller's mask (Sec. 5.2: known release points,
 * e.g. of historic avalanches, provided as a pre-computed texture).  Exact:
 * d_cells receives, in increasing order, the indices i with d_mask[i] != 0;
 * d_n their number.  Same workspace as awo_release.
 */
awo_status awo_release_from_mask(const uint8_t* d_mask, awo_grid g, uint32_t* d_cells, uint32_t* d_n,
                                 void* d_ws, size_t ws_bytes, void* stream);

/*
 * b''. Release points on a texture of chosen resolution (Sec. 5.2: the user
 * chooses the texture resolution at which potential release points are
 * evaluated).  The release texture covers the DEM's extent at 2^r times its
 * resolution, r = release_log2 in [-AWO_RELEASE_LOG2_MAX, AWO_RELEASE_LOG2_MAX]:
 * Wr x Hr = (W 2^r) x (H 2^r) for r >= 0, ceil(W 2^r) x ceil(H 2^r) for r < 0
 * (awo_release_texture_dims; Wr * Hr < 2^31).  Exact.  Texel (a, b) has its
 * centre at
 *   u = (a + 1/2) 2^-r - 1/2,  v = (b + 1/2) 2^-r - 1/2   (cell units: cell
 *   (x, y) is centred at (x, y)), each clamped to [0, W-1] resp. [0, H-1]
 * (exact in FP32).  Its steepness T is the bilinear interpolation of d_tan2
 * with the footprint and weights of the particle's height sampling (see
 * awo_simulate); the texel is a release point iff T_lo <= T <= T_hi, the
 * bounds as in awo_release.  At r = 0 this is awo_release.
 * Outputs: d_mask uint8 [Hr*Wr] (0/1, required); d_texels uint32 [capacity
 * Hr*Wr]: texel indices b*Wr + a in increasing order; d_n: their number.
 * A caller's mask at the texture's resolution (known release points) goes
 * through awo_release_from_mask with the grid {Wr, Hr, cell_size 2^-r}.
 * Run the particles with awo_sim_params.release_log2 = r.
 * Workspace: awo_release_texture_workspace_bytes(g, r) bytes, 16-byte
 * aligned, contents undefined on entry and exit.
 */
#define AWO_RELEASE_LOG2_MAX 3
awo_status awo_release_texture_dims(awo_grid g, int32_t release_log2, int32_t* width, int32_t* height);
size_t awo_release_texture_workspace_bytes(awo_grid g, int32_t release_log2);
awo_status awo_release_texture(const float* d_tan2, awo_grid g, int32_t release_log2, double slope_lo_deg,
                               double slope_hi_deg, uint8_t* d_mask, uint32_t* d_texels, uint32_t* d_n,
                               void* d_ws, size_t ws_bytes, void* stream);

/*
 * Release selection without a caller-provided workspace.  (The paper has no
 * counterpart: this is a library convenience.)  Some callers cannot hand the
 * library any extra device memory: a plug-in inside a host application, such
 * as a map renderer, whose allocator owns all device memory; or a real-time
 * loop that allocates nothing once it has started.  This entry point computes
 * exactly what awo_release computes, with the same arguments except the
 * workspace.  Its scratch (two 32-bit words per tile of 4096 cells) lives in
 * a fixed array of 128 KiB in device memory that the library holds on every
 * GPU that loads it, until the process exits; the call allocates nothing.
 *  - Grids of more than AWO_RELEASE_NOALLOC_MAX_CELLS cells (8192 x 8192) are
 *    rejected with AWO_ENOMEM before anything is enqueued.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  A failed lookup returns AWO_ECUDA.
 *  - Every call uses the same array, which keeps the last call's contents.
 *    Nothing in it needs to start at zero: each call writes every entry it
 *    later reads.  Calls that can overlap on the GPU (on different streams,
 *    or from several host threads) race on the array: serialise them.
 */
#define AWO_RELEASE_NOALLOC_MAX_CELLS (8192ll * 8192ll)
awo_status awo_release_noalloc(const float* d_tan2, awo_grid g, double slope_lo_deg, double slope_hi_deg,
                               uint8_t* d_mask, uint32_t* d_cells, uint32_t* d_n, void* stream);

/*
 * c. Particle trajectories (Sec. 5.2, avalanche trajectory node).  Exact.
 * Runs traj_per_cell particles j = 0..N-1 from every listed release cell and
 * ACCUMULATES their visits into d_count / d_maxe (so several calls compose;
 * zero-fill both before the first call, or set AWO_SIM_CLEAR_OUTPUTS).
 * Particle (cell c, j):
 *   start: p = centre of c, e = 0, d = g(p) (zero vector on flat ground);
 *          the start is a visit of c with e = 0.  With release_log2 = r != 0
 *          the list entry c is a texel of the release texture (see
 *          awo_release_texture), p is that texel's centre, and the start is a
 *          visit of the cell of p (rule below); the random counter keeps c.
 *   move n = 0, 1, ... while n < max_steps:
 *     footprint of p: i0 = floor(u), j0 = floor(v), fx = u - i0, fy = v - j0,
 *       i1 = min(i0+1, W-1), j1 = min(j0+1, H-1); heights h00 = h[j0][i0],
 *       h10 = h[j0][i1], h01 = h[j1][i0], h11 = h[j1][i1]
 *     z  = (h00*(1-fx) + h10*fx)*(1-fy) + (h01*(1-fx) + h11*fx)*fy
 *     a  = (h10-h00)*(1-fy) + (h11-h01)*fy;  b = (h01-h00)*(1-fx) + (h11-h10)*fx
 *     g  = (-a*inv, -b*inv), inv = 1/sqrt(a*a + b*b); g = d when a*a+b*b == 0
 *     (w0..w3) = Philox4x32-10(counter (c, j, n>>1, 0), key (seed lo, seed hi));
 *       words (w0, w1) for even n, (w2, w3) for odd n;
 *       xi = (float)(w >> 8) * 2^-23 - 1   in [-1, 1)
 *     r  = (P*d + (1-P)*g) + R*xi per component; r == 0 -> stopped
 *     d  = r * (1/sqrt(r.x*r.x + r.y*r.y));  p' = p + s*d
 *     p' outside [0, W-1] x [0, H-1] -> exited (not recorded)
 *     e' = (e - (k*D)*e) + (z - z') - mu*D,  D = s*cs   (k*D, mu*D rounded once)
 *     e' <= 0 -> stopped (not recorded); else p = p', e = e', and cell
 *     (i0 + [fx >= 1/2], j0 + [fy >= 1/2]) of p' is visited with e'.
 *   visit(cell, e): count += 1; maxe = max(maxe, e)
 * With drag_k = 0, e is the energy-line height: e_n = z_0 - z_n - mu * (path
 * length), and stopping at e <= 0 is the runout-angle criterion.
 * d_h: float [H*W].  d_cells: uint32 cell indices (< H*W; texel indices
 * < Wr*Hr when release_log2 != 0; a larger index is skipped on the device
 * and counted in n_rejected).  The number of
 * release cells is min(*d_n_cells, n_cells_max) when d_n_cells is non-null
 * (read on the device, so no host sync is needed after awo_release), else
 * n_cells_max.  d_count: uint32 [H*W], wraps modulo 2^32 (the call is
 * overflow-free whenever existing counts + n_traj + total_steps < 2^32).
 * d_maxe: float [H*W], non-negative (metres of energy-line height).
 * d_stats: awo_sim_stats on the device, overwritten (nullable).
 * Workspace: at least awo_simulate_workspace_bytes(n_cells_max) bytes,
 * 16-byte aligned (a work counter, the statistics, and a start record of up
 * to 32 bytes per release-list entry); contents undefined on entry and exit.
 * Gathers: on grids of at least 2^20 cells whose row pitch (4 * width bytes)
 * and d_h are aligned to the device's texture pitch alignment (32 bytes on
 * GB300), the particle kernel fetches each 2x2 footprint with one texture
 * gather through a texture object that views d_h's 32-bit words (returned
 * bit for bit, subnormal heights included; clamp addressing, which is the
 * i1, j1 clamp above; indices and weights computed as stated).  The
 * object is created at the first call with that (d_h, width, height, device)
 * and kept for the life of the process, so that a captured CUDA graph keeps
 * a valid one; after 256 such buffers, further ones use plain loads, and a
 * call made while `stream` is being captured creates none (it uses an
 * existing view, else the loads).  Both fetch the same heights: results do
 * not depend on the path.  The same holds for awo_simulate_batched (per
 * request) and the soft-deposit calls.
 */
size_t awo_simulate_workspace_bytes(uint32_t n_cells_max);
awo_status awo_simulate(const float* d_h, awo_grid g, const uint32_t* d_cells,
                        const uint32_t* d_n_cells, uint32_t n_cells_max,
                        const awo_sim_params* p, uint32_t* d_count, float* d_maxe,
                        awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream);

/*
 * Footprint path of a DEM buffer (a diagnostic of this library; the paper has
 * no counterpart).  Sets *texture to 1 when the particle kernels
 * (awo_simulate, awo_simulate_batched, the soft-deposit calls) fetch the 2x2
 * footprints of the W x H DEM at d_h by one texture gather through a texture
 * view of the buffer, 0 when they fetch them with four loads (grids under
 * 2^20 cells, a base address or row pitch off the texture alignment, 256
 * views already made, or `stream` being captured).  Like the first launch
 * with that buffer, the call creates the view when one can be made.  Results
 * never depend on the path.  AWO_EINVAL: d_h or texture NULL, or a bad grid.
 */
awo_status awo_dem_gather_path(const float* d_h, awo_grid g, void* stream, int32_t* texture);

/*
 * Kernel timing (a diagnostic of this library; the paper has no counterpart).
 * Hands two CUDA events (cudaEvent_t, passed as void*, created by the
 * caller) to the next awo_simulate call made from the calling host thread,
 * which records them on its stream immediately before and after its particle
 * kernel -- not around the output clear or the start-record prologue -- so
 * that kernel can be timed alone (when the call launches no particle kernel,
 * both are recorded after its work).  The events are consumed by that call
 * (also when it returns an error before enqueueing, unrecorded then); NULL,
 * NULL withdraws them.  AWO_EINVAL: exactly one of them NULL.
 */
awo_status awo_simulate_time_kernel(void* ev_start, void* ev_stop);

/*
 * c (batched). Particle trajectories for many regions in one persistent
 * launch (the paper's workflow re-run for many regions and parameter sets;
 * Sec. 5.2 lets the user change the parameters interactively).  Every request
 * gets exactly the rasters and statistics that awo_simulate would give it
 * alone (same formulas, same Philox streams; reductions are
 * order-independent), whatever the tuning.
 *  - reqs: HOST array of n_req (1..AWO_BATCH_MAX) requests; each one as in
 *    awo_simulate (its own DEM, grid, release list with optional device-side
 *    count, parameters incl. seed and AWO_SIM_CLEAR_OUTPUTS, and rasters).
 *    Rasters of different requests must not overlap.  The sum of n_cells_max
 *    over the requests must be < 2^31.
 *  - tuning: NULL for the default, or a configuration from awo_tune_batched.
 *  - d_stats: device array of n_req awo_sim_stats, overwritten (nullable).
 *  - Workspace: awo_simulate_batched_workspace_bytes(reqs, n_req) bytes,
 *    16-byte aligned, contents undefined on entry and exit.
 * The request table travels in the kernel's parameter block: the call makes
 * no host-to-device copy and no allocation.
 */
#define AWO_BATCH_MAX 128

typedef struct {
    const float* d_h;
    awo_grid grid;
    const uint32_t* d_cells;
    const uint32_t* d_n_cells;   /* nullable */
    uint32_t n_cells_max;
    uint32_t reserved;
    awo_sim_params params;
    uint32_t* d_count;
    float* d_maxe;
} awo_sim_request;

/* Launch shape of the batched particle kernel (the autotuner's search space).
 *   threads_per_block: 64, 128 or 256 (0 = 128)
 *   group_particles:   particles a warp takes per fetch, 32 .. 65536 (0 = chosen
 *                      per launch: about all particles / (4 x the grid's warps),
 *                      rounded down to a multiple of 32, within 32 .. 1024)
 *   refill: AWO_REFILL_LANE -- ended lanes take the next particles while the
 *           warp's other lanes keep moving, once the idle lanes add up to 12
 *           idle lane-iterations (trajectory per thread, continuously
 *           refilled);
 *           AWO_REFILL_WARP -- a warp starts 32 particles together and takes
 *           the next 32 only when all have ended (trajectories per warp, in
 *           lock-step batches). */
#define AWO_REFILL_LANE 0
#define AWO_REFILL_WARP 1
typedef struct {
    int32_t threads_per_block;
    int32_t group_particles;
    int32_t refill;
    int32_t reserved;
} awo_tuning;

size_t awo_simulate_batched_workspace_bytes(const awo_sim_request* reqs, int32_t n_req);
awo_status awo_simulate_batched(const awo_sim_request* reqs, int32_t n_req, const awo_tuning* tuning,
                                awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream);

/*
 * Autotuner: times every launch shape of the search space (threads per block
 * x group size x refill policy) on this batch with CUDA events and returns
 * the fastest in *best (and its time in *best_ms, nullable).  Each timed run
 * clears the requests' rasters first, so on return they hold the batch's
 * result.  Synchronises `stream`; not for use during stream capture.
 */
awo_status awo_tune_batched(const awo_sim_request* reqs, int32_t n_req, void* d_ws, size_t ws_bytes,
                            void* stream, awo_tuning* best, float* best_ms);

/*
 * c (soft). Soft-deposit particles and their gradient -- a differentiable
 * variant of the trajectory node for fitting friction parameters and release
 * weights (the paper has no gradients; this mode is this library's).
 * Each particle follows exactly the path of awo_simulate (same direction and
 * move arithmetic, same Philox streams) but its energy does not stop it: it
 * carries a survival S_0 = 1, S_n = S_{n-1} * sigma(e_n / tau) with
 * sigma(x) = 1 / (1 + exp(-x)) (FP32, expf), deposits w (S_{n-1} - S_n) at
 * the cell of p_n, and ends when it leaves the grid, has no direction,
 * reaches max_steps, or S_n < 1e-7; the rest, w S_last, goes to the last cell
 * reached.  w is the particle's release-cell weight (d_weight, FP32 per
 * release-list entry).  e is FP32 as in awo_simulate, so results match an
 * FP64 evaluation to FP32 rounding, not bit for bit.
 *
 * awo_soft_forward ACCUMULATES deposits into d_deposit (int64 per cell, fixed
 * point: deposit = value * 2^-32; AWO_SIM_CLEAR_OUTPUTS zeroes it first).
 * Each particle adds exactly round(w 2^32) (cumulative quantisation), so the
 * raster is deterministic.  d_stats (nullable): total_steps, n_traj and
 * n_rejected are set, the other fields are 0.
 *
 * awo_soft_backward, given G = dL/dD (FP32 per cell), overwrites
 * d_grad_theta[0] = dL/dlog(mu), d_grad_theta[1] = dL/dlog(drag_k) (FP64) and
 * d_grad_weight[i] = dL/dw_i (FP32, for the first min(*d_n_cells,
 * n_cells_max) entries).  It recomputes every particle from its start with
 * the same draws and carries forward tangents of the energy and survival
 * (the path itself does not depend on mu, k or w), so it stores nothing per
 * step.  Sums over particles are FP64.
 * Both take a workspace of awo_soft_workspace_bytes(n_cells_max) bytes.
 * tau > 0 in metres of energy-line height (1 m in the differentiable
 * workload).  The release list holds DEM cells: release_log2 must be 0.
 */
size_t awo_soft_workspace_bytes(uint32_t n_cells_max);
awo_status awo_soft_forward(const float* d_h, awo_grid g, const uint32_t* d_cells, const uint32_t* d_n_cells,
                            uint32_t n_cells_max, const float* d_weight, const awo_sim_params* p, float tau,
                            int64_t* d_deposit, awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream);
awo_status awo_soft_backward(const float* d_h, awo_grid g, const uint32_t* d_cells, const uint32_t* d_n_cells,
                             uint32_t n_cells_max, const float* d_weight, const awo_sim_params* p, float tau,
                             const float* d_grad_deposit, double* d_grad_theta, float* d_grad_weight,
                             void* d_ws, size_t ws_bytes, void* stream);
/* Fixed-point deposits to FP64: d_out[i] = (double)d_q[i] * 2^-32. */
awo_status awo_fixed_to_real(const int64_t* d_q, int64_t n, double* d_out, void* stream);

/*
 * c'. Velocity indicator (Fig. 4: the colour encodes Z^delta_max, read as a
 * velocity): d_vel[i] = sqrt((2*gravity) * d_maxe[i]).  Exact.
 * d_vel may alias d_maxe.
 */
awo_status awo_finalize(const float* d_maxe, awo_grid g, float gravity, float* d_vel, void* stream);

/*
 * d. Overlay mipmap (Sec. 3: "from the high-resolution overlay texture, we
 * then compute a mipmap").  Exact.  Level l+1 has size ceil(W_l/2) x
 * ceil(H_l/2); its texel (x, y) reduces the texels (2x+dx, 2y+dy),
 * dx, dy in {0, 1}, that exist in level l: counts are summed and saturated
 * at 2^32-1, velocities take the maximum.  Level 0 is (d_count, d_vel).
 * d_count_lv and d_vel_lv are HOST arrays of levels-1 device pointers that
 * receive levels 1 .. levels-1.  1 <= levels <= 16.
 */
awo_status awo_overlay_lod(const uint32_t* d_count, const float* d_vel, awo_grid g, int32_t levels,
                           uint32_t* const* d_count_lv, float* const* d_vel_lv, void* stream);

/*
 * c' + d in one pass: exactly awo_finalize(d_maxe, g, gravity, d_vel)
 * followed by awo_overlay_lod(d_count, d_vel, g, levels, ...), but level 0's
 * velocity is made from d_maxe as the mipmap reads it, so the velocity
 * raster is written once and never read back.  d_vel may alias d_maxe.
 * Arguments, ranges and errors as in the two calls.
 */
awo_status awo_finalize_lod(const float* d_maxe, const uint32_t* d_count, awo_grid g, float gravity,
                            int32_t levels, float* d_vel, uint32_t* const* d_count_lv, float* const* d_vel_lv,
                            void* stream);

/*
 * Compose (Sec. 3: the compose pass alpha-blends the data-driven overlay over
 * the base map; Fig. 4: colour encodes Z^delta_max, read as velocity).
 * Exact.  Per texel: x = d_value[i] clamped to [value[0], value[n_stops-1]];
 * k the segment with value[k] <= x (last segment for the top stop);
 * t = (x - value[k]) / (value[k+1] - value[k]); per channel
 * c = rgb[k] + t * (rgb[k+1] - rgb[k]); a = alpha if d_count[i] >= count_min
 * else 0.  With d_base_rgba: out.rgb = rint(a*c + (1-a)*base.rgb),
 * out.a = base.a; without: out.rgb = rint(c), out.a = rint(255*a).  FP32,
 * no fused multiply-add, round half to even, clamped to [0, 255].
 * d_value: float [H*W]; d_count: uint32 [H*W]; RGBA8 buffers [4*H*W],
 * 4-byte aligned.  Requires 2 <= n_stops <= 16, strictly increasing values,
 * alpha in [0, 1].
 */
typedef struct {
    int32_t n_stops;
    float value[16];
    uint8_t rgb[16][3];
    uint8_t pad[4];
    float alpha;
    uint32_t count_min;
} awo_colormap;
awo_status awo_compose(const float* d_value, const uint32_t* d_count, awo_grid g, const awo_colormap* cm,
                       const uint8_t* d_base_rgba, uint8_t* d_out_rgba, void* stream);

/*
 * Snow cover (Sec. 5.1: snow line altitude, maximum steepness and blending
 * factors; snow-covered texels white, alpha the blending factor).  Exact.
 * With nz the normal's z component (awo_normals' third plane, the cosine of
 * the slope angle):
 *   alpha = smoothstep(L - b/2, L + b/2, h) * smoothstep(cos(m + c/2), cos(m - c/2), nz)
 * L = snow_line_m, b = blend_alt_m, m = max_slope_deg, c = blend_slope_deg
 * (slope bounds clamped to [0, 90] degrees); the four edges computed in
 * double on the host and rounded to float once; smoothstep(e0, e1, x) =
 * t*t*(3 - 2*t), t = clamp((x - e0) / (e1 - e0), 0, 1), a step x >= e0 when
 * e0 == e1.  Outputs: d_alpha float [H*W] and/or d_rgba (255, 255, 255,
 * rint(255*alpha)) [4*H*W].
 */
typedef struct {
    float snow_line_m;
    float blend_alt_m;
    float max_slope_deg;
    float blend_slope_deg;
} awo_snow_params;
awo_status awo_snow_cover(const float* d_h, const float* d_nz, awo_grid g, const awo_snow_params* p,
                          float* d_alpha, uint8_t* d_rgba, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AWO_H */
