// awo_simulate.cu -- Monte-Carlo avalanche trajectories (Sec. 5.2).
//
// Design (GB300):
//  * Persistent kernel, one lane per particle.  The particles are numbered
//    cell-major (start record, then particle j); a warp takes a chunk of
//    consecutive particles at a time from a global counter (one atomic per
//    chunk) and walks it with a warp-uniform cursor; a lane is refilled the
//    moment its particle ends, so lanes never idle behind a long particle of
//    the same warp.  The chunk size (32 .. 1024 particles) follows from the
//    particle count and the grid, so that a release list of a few cells is
//    still spread over many warps.  The start records are in a processing
//    order that spreads consecutive blocks of release cells over the grid
//    (order_slot): the lanes of a warp work on neighbouring cells, while the
//    warps of the GPU work all over the grid and its memory partitions.
//  * One integer division per chunk and none per particle: the cursor
//    carries (release-list entry, j), and the start record holds the cell's
//    coordinates.
//  * A particle starts at refill time from the 16-byte start record of its
//    release cell (position, height, first direction), written by a prologue
//    kernel that also records the release visits of all N particles of the
//    cell with one reduction.  Each loop iteration is then two moves and
//    their visits from one Philox block (moves n and n + 1 take words 0-1 and
//    2-3 of block n >> 1; live lanes are always at an even n there) --
//    direction from the footprint kept in registers, step, footprint and
//    energy at the new position, record -- written without data-dependent
//    branches (selects and predicated reductions), so a warp runs one
//    instruction stream.
//  * Visits go to the rasters as fire-and-forget reductions (RED.ADD on the
//    count, RED.MAX on the bits of the non-negative energy), one pair per
//    lane: measured on GB300, merging the lanes of a warp that hit the same
//    cell (__match_any_sync + __reduce_max_sync) costs more issue slots than
//    the L2 spends on the duplicate reductions.
//  * Philox4x32-10 round keys are computed once on the host and read from the
//    kernel's parameter bank.
//  * On grids of at least 2^20 cells the 2x2 footprint of a move is one
//    texture gather through a texture object that views the DEM's words
//    (clamp addressing is the footprint clamp; indices and weights are still
//    computed here), in place of four loads, their addresses and clamps.
//  * Arithmetic is FP32 with explicit round-to-nearest intrinsics: no fused
//    multiply-add, IEEE sqrt and reciprocal, so every particle follows the
//    formulas of awo.h bit for bit.
#include <math.h>
#include <string.h>

#include <mutex>

#include "awo_particle.cuh"

namespace awo {

struct SimWorkspace {
    unsigned long long next_item;  // global work counter, in particles
    unsigned long long stats[6];   // total_steps, n_traj, n_exited, n_capped, n_stopped, n_rejected
    unsigned long long pad;
};
static_assert(sizeof(SimWorkspace) == 64, "workspace layout");

struct SimArgs {
    // request constants (names read by AWO_MOVE_WORDS)
    const float* h;
    uint32_t* count;
    float* maxe;
    int W, H;
    float Wm1, Hm1;        // W-1, H-1 as floats (exact for W, H <= 2^24)
    float P, oneP, R, s;   // persistence, 1-P, randomness, step in cells
    float kD, muD;         // drag_k*D, mu*D  (D = s*cell_size)
    uint32_t max_steps;
    KeysTable keys;        // Philox round keys
    // work
    const uint32_t* cells;
    const uint32_t* n_cells_dev;
    uint32_t n_cells_max;
    uint32_t n_grid;       // W*H
    uint32_t N;
    TexelGeom tg;          // release texture (texel mode only)
    SimWorkspace* ws;
    void* starts;          // one start record per release-list entry (CellStart or TexelStart)
    cudaTextureObject_t tex;  // texture view of h (the gathers of k_simulate<_, true>), or 0
};

constexpr int SIM_THREADS = 128;
constexpr uint32_t SIM_CHUNK_MAX = 1024;  // particles per global fetch, at most
// fetches a warp makes on an even split, at least: chunks of neighbouring
// cells carry similar work, so few large chunks leave some warps with much
// more of it (2048^2 workload: 4 -> 16 chunks a warp, 1.80 -> 1.72 ms)
constexpr uint32_t SIM_CHUNKS_PER_WARP = 16;
// A warp refills its idle lanes once they add up to SIM_REFILL_IDLE idle
// lane-iterations since its last refill (or when every lane is idle): a
// refill round costs issue slots whether it starts one particle or thirty,
// so refilling for a single idle lane wastes slots, and waiting too long
// leaves lanes idle.  Measured on GB300 (8192^2 particle kernel, ms, with the
// counters folded per particle): 1 -> 20.61, 2 -> 20.50, 3 -> 20.46,
// 4 -> 20.46, 6 -> 20.46, 8 -> 20.54, 12 -> 20.67, 16 -> 20.88.
constexpr uint32_t SIM_REFILL_IDLE = 4;

__device__ __forceinline__ uint32_t release_count(const SimArgs& a)
{
    uint32_t n = a.n_cells_max;
    if (a.n_cells_dev) n = min(n, *a.n_cells_dev);
    return n;
}

// Prologue: per release-list entry, the start record (at its slot in the
// processing order of awo_particle.cuh) and the release visit of all N particles (count +=
// N; their energy is 0, so the maximum is unchanged).  Grid-stride over the
// entries, whose number may be on the device.
// TEXELS: the entries are texels of the release texture.  It also counts the
// particles of entries outside the grid (rejected) and, when max_steps = 0
// (every particle capped at its release visit; the particle kernel is not
// launched), the particles and caps.
template <bool TEXELS>
__global__ void __launch_bounds__(256) k_sim_starts(const __grid_constant__ SimArgs a)
{
    const uint32_t n_cells = release_count(a);
    const uint32_t B = order_block(a.N);
    const uint32_t nb = n_cells / B;
    __shared__ uint32_t s_sinv;
    if (threadIdx.x == 0) s_sinv = order_stride_inverse(nb);
    __syncthreads();
    const uint32_t Sinv = s_sinv;
    // the slot of the thread's entries, advanced per grid stride G (a
    // multiple of B: B <= 32 divides the block size) instead of one 64-bit
    // modulo per entry: entry ci + G is in block ci / B + G / B, same offset
    const uint32_t G = gridDim.x * blockDim.x;
    const uint32_t ci0 = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long step = nb ? ((unsigned long long)(G / B) * Sinv) % nb : 0ull;
    unsigned long long sb = nb ? ((unsigned long long)(ci0 / B) * Sinv) % nb : 0ull;
    unsigned long long good = 0ull, bad = 0ull;
    for (uint32_t ci = ci0; ci < n_cells; ci += G) {
        const uint32_t slot = ci < nb * B ? (uint32_t)sb * B + (ci & (B - 1u)) : ci;  // = order_slot(ci)
        sb += step;
        if (sb >= nb) sb -= nb;
        const uint32_t entry = __ldg(a.cells + ci);
        bool ok;
        if (TEXELS) {
            const TexelStart st = texel_start(a.h, a.W, a.H, a.tg, entry);
            ok = st.t != ~0u;
            if (ok) atomicAdd(a.count + st.vcell, a.N);
            static_cast<TexelStart*>(a.starts)[slot] = st;
        } else {
            const CellStart st = cell_start(a.h, a.W, a.H, a.n_grid, entry);
            ok = st.xy != ~0u;
            if (ok) atomicAdd(a.count + entry, a.N);
            static_cast<CellStart*>(a.starts)[slot] = st;
        }
        good += ok ? 1ull : 0ull;
        bad += ok ? 0ull : 1ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        good += __shfl_xor_sync(0xffffffffu, good, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(&a.ws->stats[5], bad * a.N);
        if (good && a.max_steps == 0u) {
            atomicAdd(&a.ws->stats[1], good * a.N);
            atomicAdd(&a.ws->stats[3], good * a.N);
        }
    }
}

template <bool TEXELS, bool TEX>
__global__ void __launch_bounds__(SIM_THREADS) k_simulate(const __grid_constant__ SimArgs a)
{
    constexpr int kGather = TEX ? 1 : 0;  // footprints by texture gather or loads (read by AWO_MOVE_WORDS)
    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;
    const uint32_t n_cells = release_count(a);

    // particles in all, and the chunk a warp takes per fetch: a multiple of
    // 32 in [32, SIM_CHUNK_MAX], about total / (warps * SIM_CHUNKS_PER_WARP)
    const unsigned long long total = (unsigned long long)n_cells * a.N;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long chunk = total / (warps * SIM_CHUNKS_PER_WARP);
    chunk = chunk < 32ull ? 32ull : (chunk > SIM_CHUNK_MAX ? (unsigned long long)SIM_CHUNK_MAX : chunk);
    chunk &= ~31ull;

    // warp-uniform cursor: next particle (t, and as (entry, j)) and the end of the chunk
    unsigned long long cur_t = 0ull, end_t = 0ull;
    uint32_t cur_ci = 0, cur_j = 0;
    bool exhausted = (total == 0ull);
    uint32_t idle_acc = 0u;  // idle lane-iterations since the last refill (warp-uniform)

    AWO_LANE_STATE

    while (true) {
        // ---- refill idle lanes (once they add up to SIM_REFILL_IDLE) --------
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        idle_acc += (uint32_t)__popc(idle);
        if (idle != 0u && idle_acc >= SIM_REFILL_IDLE && !exhausted) {
            idle_acc = 0u;
            if (cur_t >= end_t) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&a.ws->next_item, chunk);
                base = __shfl_sync(0xffffffffu, base, 0);
                exhausted = base >= total;
                if (!exhausted) {
                    cur_t = base;
                    end_t = min(total, base + chunk);
                    cur_ci = (uint32_t)(base / a.N);  // one division per chunk
                    cur_j = (uint32_t)(base - (unsigned long long)cur_ci * a.N);
                }
            }
            if (!exhausted) {
                // particles left in the chunk (capped at 32)
                const unsigned long long left = end_t - cur_t;
                const unsigned avail = left < 32ull ? (unsigned)left : 32u;
                const unsigned want = (unsigned)__popc(idle);
                const unsigned take = want < avail ? want : avail;
                const unsigned rank = (unsigned)__popc(idle & lane_lt);
                const bool mine = ((idle >> lane) & 1u) && rank < take;
                uint32_t ci = cur_ci, jj = cur_j;
                advance(ci, jj, rank < take ? rank : 0u, a.N);
                uint4 st = make_uint4(~0u, 0u, 0u, 0u), st1 = make_uint4(0u, 0u, 0u, 0u);
                if (TEXELS) {
                    if (mine) {
                        st = __ldg(reinterpret_cast<const uint4*>(a.starts) + 2u * ci);
                        st1 = __ldg(reinterpret_cast<const uint4*>(a.starts) + 2u * ci + 1u);
                    }
                } else {
                    if (mine) st = __ldg(reinterpret_cast<const uint4*>(a.starts) + ci);
                }
                // entries outside the grid are skipped here and counted by the prologue
                const bool ok = mine && st.x != ~0u;
                AWO_FOLD_LANE(mine, a.max_steps);
                if (TEXELS)
                    AWO_LANE_START_TEXEL(ok, st, st1, jj);
                else
                    AWO_LANE_START(ok, st, jj, a.W);
                my_traj += ok ? 1u : 0u;  // particles are counted when they start
                live = live || ok;
                advance(cur_ci, cur_j, take, a.N);
                cur_t += take;
            }
        }
        if (__ballot_sync(0xffffffffu, live) == 0u) {
            if (exhausted) break;
            continue;
        }
        AWO_MOVE_PAIR(a, a.keys);
    }
    AWO_FOLD_LANE(true, a.max_steps);
    AWO_FLUSH_COUNTERS(a.ws->stats);
}

template <bool TEXELS, bool TEX>
static int sim_blocks_per_sm()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_simulate<TEXELS, TEX>, SIM_THREADS, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        cached[dev] = b;
    }
    return cached[dev];
}

// Texture views of DEM buffers for the gathers of k_simulate: a texture
// object is a descriptor of (address, width, height, row pitch) -- no copy;
// the words are viewed as 32-bit unsigned texels, returned bit for bit --
// created on the first call with a buffer and kept for the life of the
// process (at most DEM_VIEWS_MAX of them; further buffers take the load
// path), so that a graph that captured a launch keeps a valid view.  A view
// needs the row pitch and the base address aligned to the device's texture
// pitch alignment and a grid within the 2D pitch-linear texture limits;
// otherwise (or if creation fails) the kernel gathers with loads.  While the
// launch stream is being captured into a graph no view is created (an
// existing one is used, else the loads), so a capture never sees a call it
// might refuse.  Grids
// under DEM_VIEW_MIN_CELLS take the loads too: measured on GB300 (particle
// kernel, texture gathers against loads), 8192^2 -5.5%, 2048^2 -1%, 256^2
// +4% (a DEM that small stays in L1, where the loads' latency is shorter).
constexpr int DEM_VIEWS_MAX = 256;
constexpr int64_t DEM_VIEW_MIN_CELLS = int64_t(1) << 20;

struct DemView {
    const float* h;
    int W, H, dev;
    cudaTextureObject_t tex;
};

cudaTextureObject_t dem_texture(const float* d_h, awo_grid g, cudaStream_t s)
{
    if (cells_of(g) < DEM_VIEW_MIN_CELLS) return 0;
    static std::mutex mu;
    static DemView views[DEM_VIEWS_MAX];
    static int n_views = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < n_views; ++i)
        if (views[i].h == d_h && views[i].W == g.width && views[i].H == g.height && views[i].dev == dev)
            return views[i].tex;
    if (n_views == DEM_VIEWS_MAX) return 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 0;
    }
    int pitch_align = 0, max_w = 0, max_h = 0;
    if (cudaDeviceGetAttribute(&pitch_align, cudaDevAttrTexturePitchAlignment, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture2DLinearWidth, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxTexture2DLinearHeight, dev) != cudaSuccess || pitch_align <= 0)
        return 0;
    const size_t pitch = (size_t)g.width * sizeof(float);
    if ((pitch % (size_t)pitch_align) != 0 || ((uintptr_t)d_h % (uintptr_t)pitch_align) != 0 || g.width > max_w ||
        g.height > max_h)
        return 0;
    cudaResourceDesc rd;
    memset(&rd, 0, sizeof(rd));
    rd.resType = cudaResourceTypePitch2D;
    rd.res.pitch2D.devPtr = const_cast<float*>(d_h);
    rd.res.pitch2D.desc = cudaCreateChannelDesc<unsigned int>();  // raw words: no subnormal flush
    rd.res.pitch2D.width = (size_t)g.width;
    rd.res.pitch2D.height = (size_t)g.height;
    rd.res.pitch2D.pitchInBytes = pitch;
    cudaTextureDesc td;
    memset(&td, 0, sizeof(td));
    td.addressMode[0] = cudaAddressModeClamp;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaTextureObject_t t = 0;
    if (cudaCreateTextureObject(&t, &rd, &td, nullptr) != cudaSuccess) {
        cudaGetLastError();  // a failed creation is not a launch error
        return 0;
    }
    views[n_views++] = DemView{d_h, g.width, g.height, dev, t};
    return t;
}

}  // namespace awo

using namespace awo;

static size_t starts_offset() { return 256; }

// Events of awo_simulate_time_kernel for the next awo_simulate of this thread.
static thread_local cudaEvent_t t_kernel_events[2] = {nullptr, nullptr};

extern "C" awo_status awo_simulate_time_kernel(void* ev_start, void* ev_stop)
{
    if ((ev_start == nullptr) != (ev_stop == nullptr)) return AWO_EINVAL;
    t_kernel_events[0] = static_cast<cudaEvent_t>(ev_start);
    t_kernel_events[1] = static_cast<cudaEvent_t>(ev_stop);
    return AWO_OK;
}

extern "C" awo_status awo_dem_gather_path(const float* d_h, awo_grid g, void* stream, int32_t* texture)
{
    if (!d_h || !texture || !grid_ok(g)) return AWO_EINVAL;
    *texture = dem_texture(d_h, g, as_stream(stream)) != 0 ? 1 : 0;
    return AWO_OK;
}

extern "C" size_t awo_simulate_workspace_bytes(uint32_t n_cells_max)
{
    return starts_offset() + (size_t)n_cells_max * sizeof(TexelStart);
}

extern "C" awo_status awo_simulate(const float* d_h, awo_grid g, const uint32_t* d_cells, const uint32_t* d_n_cells,
                                   uint32_t n_cells_max, const awo_sim_params* p, uint32_t* d_count, float* d_maxe,
                                   awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream)
{
    const cudaEvent_t ev_start = t_kernel_events[0], ev_stop = t_kernel_events[1];  // consumed by this call
    t_kernel_events[0] = t_kernel_events[1] = nullptr;
    if (!d_h || !d_count || !d_maxe || !d_ws || !grid_ok(g)) return AWO_EINVAL;
    if (n_cells_max > 0 && !d_cells) return AWO_EINVAL;
    if (!sim_params_ok(p, g)) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0 || (((uintptr_t)d_count) & 3u) != 0 || (((uintptr_t)d_maxe) & 3u) != 0)
        return AWO_EINVAL;
    if (ws_bytes < awo_simulate_workspace_bytes(n_cells_max)) return AWO_ENOMEM;
    cudaStream_t s = as_stream(stream);
    SimWorkspace* ws = static_cast<SimWorkspace*>(d_ws);
    if (cudaMemsetAsync(ws, 0, sizeof(SimWorkspace), s) != cudaSuccess) return AWO_ECUDA;
    if (p->flags & AWO_SIM_CLEAR_OUTPUTS) {
        const size_t bytes = (size_t)cells_of(g) * sizeof(uint32_t);
        if (cudaMemsetAsync(d_count, 0, bytes, s) != cudaSuccess) return AWO_ECUDA;
        if (cudaMemsetAsync(d_maxe, 0, bytes, s) != cudaSuccess) return AWO_ECUDA;
    }

    // host-side constants, each one FP32 rounding in the documented order
    const float D = p->step_scale * g.cell_size;
    SimArgs a;
    a.h = d_h;
    a.cells = d_cells;
    a.n_cells_dev = d_n_cells;
    a.n_cells_max = n_cells_max;
    a.W = g.width;
    a.H = g.height;
    a.n_grid = (uint32_t)cells_of(g);
    a.Wm1 = (float)(g.width - 1);
    a.Hm1 = (float)(g.height - 1);
    a.P = p->persistence;
    a.oneP = 1.0f - p->persistence;
    a.R = p->randomness;
    a.s = p->step_scale;
    a.kD = p->drag_k * D;
    a.muD = p->mu * D;
    a.N = p->traj_per_cell;
    a.max_steps = p->max_steps;
    uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.keys.k0[r] = k0;
        a.keys.k1[r] = k1;
        k0 += 0x9E3779B9u;  // Weyl key schedule of Philox4x32
        k1 += 0xBB67AE85u;
    }
    a.count = d_count;
    a.maxe = d_maxe;
    a.ws = ws;
    a.starts = static_cast<char*>(d_ws) + starts_offset();
    int64_t wr = 0, hr = 0;
    release_texture_dims(g, p->release_log2, &wr, &hr);  // checked by sim_params_ok
    a.tg.Wr = (uint32_t)wr;
    a.tg.n_tex = (uint32_t)(wr * hr);
    a.tg.scale = ldexpf(1.0f, -p->release_log2);
    const bool texels = p->release_log2 != 0;

    a.tex = dem_texture(d_h, g, s);

    if (a.N > 0 && n_cells_max > 0 && a.max_steps == 0u) {  // every particle capped at its release visit
        const unsigned pro_blocks = stream_blocks((int64_t)n_cells_max, 256);
        if (texels)
            k_sim_starts<true><<<pro_blocks, 256, 0, s>>>(a);
        else
            k_sim_starts<false><<<pro_blocks, 256, 0, s>>>(a);
        awo_status st = launch_status();
        if (st != AWO_OK) return st;
    } else if (a.N > 0 && n_cells_max > 0) {
        const unsigned pro_blocks = stream_blocks((int64_t)n_cells_max, 256);
        const unsigned sms = (unsigned)sm_count();
        if (texels)
            k_sim_starts<true><<<pro_blocks, 256, 0, s>>>(a);
        else
            k_sim_starts<false><<<pro_blocks, 256, 0, s>>>(a);
        if (ev_start && cudaEventRecord(ev_start, s) != cudaSuccess) return AWO_ECUDA;
        if (texels) {
            if (a.tex)
                k_simulate<true, true><<<sms * sim_blocks_per_sm<true, true>(), SIM_THREADS, 0, s>>>(a);
            else
                k_simulate<true, false><<<sms * sim_blocks_per_sm<true, false>(), SIM_THREADS, 0, s>>>(a);
        } else {
            if (a.tex)
                k_simulate<false, true><<<sms * sim_blocks_per_sm<false, true>(), SIM_THREADS, 0, s>>>(a);
            else
                k_simulate<false, false><<<sms * sim_blocks_per_sm<false, false>(), SIM_THREADS, 0, s>>>(a);
        }
        if (ev_stop && cudaEventRecord(ev_stop, s) != cudaSuccess) return AWO_ECUDA;
        awo_status st = launch_status();
        if (st != AWO_OK) return st;
    } else if (ev_start) {  // no particle kernel: an empty interval after the call's work
        if (cudaEventRecord(ev_start, s) != cudaSuccess || cudaEventRecord(ev_stop, s) != cudaSuccess)
            return AWO_ECUDA;
    }
    if (a.N > 0 && n_cells_max > 0 && a.max_steps == 0u && ev_start) {  // prologue only: an empty interval
        if (cudaEventRecord(ev_start, s) != cudaSuccess || cudaEventRecord(ev_stop, s) != cudaSuccess)
            return AWO_ECUDA;
    }
    if (d_stats) {
        if (cudaMemcpyAsync(d_stats, ws->stats, sizeof(awo_sim_stats), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return AWO_ECUDA;
    }
    return AWO_OK;
}
