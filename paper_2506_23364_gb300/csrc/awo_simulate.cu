// awo_simulate.cu -- Monte-Carlo avalanche trajectories (Sec. 5.2).
//
// Design (GB300):
//  * Persistent kernel, one lane per particle.  A warp takes a few release
//    cells at a time from a global counter (one atomic per cell group) and
//    walks their particles (cell-major, particle j minor) with a warp-uniform
//    cursor; a lane is refilled the moment its particle ends, so lanes never
//    idle behind a long particle of the same warp.  The particles in flight
//    come from a compact window of the release list, so the lanes of a warp,
//    and the warps of the GPU, touch a compact region of the DEM and of the
//    rasters, which stays L2-resident even when the DEM does not.
//  * No integer division on the refill path: the cursor carries (cell, j),
//    and a cell index becomes (x, y) through a float reciprocal of W and one
//    exact correction step.
//  * A particle starts at refill time: the 2x2 footprint of its release cell
//    is gathered and its release visit recorded (merged over the particles of
//    the cell that start together).  Each loop iteration is then exactly one
//    move and its visit -- direction from the footprint kept in registers,
//    draw, step, footprint and energy at the new position, record -- written
//    without data-dependent branches (selects and predicated reductions), so
//    a warp runs one instruction stream.
//  * Visits go to the rasters as fire-and-forget reductions (RED.ADD on the
//    count, RED.MAX on the bits of the non-negative energy), one pair per
//    lane: measured on GB300, merging the lanes of a warp that hit the same
//    cell (__match_any_sync + __reduce_max_sync) costs more issue slots than
//    the L2 spends on the duplicate reductions.
//  * Philox4x32-10 round keys are computed once on the host and read from the
//    kernel's parameter bank.
//  * Arithmetic is FP32 with explicit round-to-nearest intrinsics: no fused
//    multiply-add, IEEE sqrt and reciprocal, so every particle follows the
//    formulas of awo.h bit for bit.
#include "awo_internal.cuh"

namespace awo {

struct SimWorkspace {
    unsigned long long next_cell;  // global work counter, in release-list entries
    unsigned long long total_steps, n_traj, n_exited, n_capped, n_stopped, n_rejected;
    unsigned long long pad;
};
static_assert(sizeof(SimWorkspace) == 64, "workspace layout");

// Start of the particles of one release cell, shared by all N of them:
// position, height and initial direction (the steepest descent at the cell
// centre, zero on flat ground).  xy = x | y << 16; xy = ~0u marks an index
// outside the grid.
struct __align__(16) CellStart {
    uint32_t xy;
    float z0, d0x, d0y;
};
static_assert(sizeof(CellStart) == 16, "start record layout");

struct SimArgs {
    const float* h;
    const uint32_t* cells;
    const uint32_t* n_cells_dev;
    uint32_t n_cells_max;
    int W, H;
    uint32_t n_grid;       // W*H
    float invW;            // 1/W rounded, for the cell -> (x, y) split
    float Wm1, Hm1;        // W-1, H-1 as floats (exact for W, H <= 2^24)
    float P, oneP, R, s;   // persistence, 1-P, randomness, step in cells
    float kD, muD;         // drag_k*D, mu*D  (D = s*cell_size)
    uint32_t N, max_steps;
    uint32_t cells_per_fetch;
    uint32_t rk0[10], rk1[10];  // Philox round keys
    uint32_t* count;
    float* maxe;
    SimWorkspace* ws;
    CellStart* starts;     // one per release-list entry
};

constexpr int SIM_THREADS = 128;
constexpr uint32_t SIM_FETCH_ITEMS = 1024;  // particles per global fetch, at least

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// of the even words and a word permutation that mixes in the round key.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t* __restrict__ rk0,
                                               const uint32_t* __restrict__ rk1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk0[r], lo1, hi0 ^ c.w ^ rk1[r], lo0);
    }
    return c;
}

// (w >> 8) * 2^-23 - 1: exact uniform in [-1, 1).
__device__ __forceinline__ float uniform_pm1(uint32_t w)
{
    return __fsub_rn(__fmul_rn(__uint2float_rn(w >> 8), 1.1920928955078125e-7f), 1.0f);
}

struct Foot {
    int i0, j0;
    float fx, fy, h00, h10, h01, h11;
};

__device__ __forceinline__ Foot gather(const float* __restrict__ h, int W, int H, float u, float v)
{
    Foot f;
    f.i0 = __float2int_rd(u);
    f.j0 = __float2int_rd(v);
    f.fx = __fsub_rn(u, __int2float_rn(f.i0));
    f.fy = __fsub_rn(v, __int2float_rn(f.j0));
    // 32-bit offsets: W * H < 2^31
    const int di = f.i0 + 1 < W ? 1 : 0;
    const int dj = f.j0 + 1 < H ? W : 0;
    const int o = f.j0 * W + f.i0;
    f.h00 = __ldg(h + o);
    f.h10 = __ldg(h + (o + di));
    f.h01 = __ldg(h + (o + dj));
    f.h11 = __ldg(h + (o + dj + di));
    return f;
}

__device__ __forceinline__ float bilinear(const Foot& f, float ox, float oy)
{
    float top = __fadd_rn(__fmul_rn(f.h00, ox), __fmul_rn(f.h10, f.fx));
    float bot = __fadd_rn(__fmul_rn(f.h01, ox), __fmul_rn(f.h11, f.fx));
    return __fadd_rn(__fmul_rn(top, oy), __fmul_rn(bot, f.fy));
}

// Merged visit of the lanes in `active` that record (idx, e).  Lanes with the
// same cell are grouped; the group leader issues one RED.ADD with the group
// size and, unless every e of the group is 0 (release visits), one RED.MAX
// with the group maximum of the energy bits (non-negative floats order like
// their bit patterns).
__device__ __forceinline__ void record(uint32_t* __restrict__ count, float* __restrict__ maxe, unsigned active,
                                       uint32_t idx, float e)
{
    unsigned grp = __match_any_sync(active, idx);
    unsigned emax = __reduce_max_sync(grp, __float_as_uint(e));
    if ((threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1)) {
        atomicAdd(count + idx, (unsigned)__popc(grp));
        if (emax != 0u) atomicMax(reinterpret_cast<unsigned*>(maxe) + idx, emax);
    }
}

// Advances a (cell, j) cursor by k <= 32 particles of N per cell.
__device__ __forceinline__ void advance(uint32_t& ci, uint32_t& j, uint32_t k, uint32_t N)
{
    j += k;
    if (j >= N) {
        if (N >= 32u) {
            j -= N;
            ci += 1u;
        } else {
            uint32_t q = j / N;
            ci += q;
            j -= q * N;
        }
    }
}

// Prologue: per release-list entry, the start record and the release visit
// of all N particles (count += N; their energy is 0, so the maximum is
// unchanged).  Grid-stride over the entries, whose number may be on the device.
__global__ void __launch_bounds__(256) k_sim_starts(const __grid_constant__ SimArgs a)
{
    uint32_t n_cells = a.n_cells_max;
    if (a.n_cells_dev) n_cells = min(n_cells, *a.n_cells_dev);
    for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < n_cells; ci += gridDim.x * blockDim.x) {
        const uint32_t cell = __ldg(a.cells + ci);
        CellStart st;
        if (cell < a.n_grid) {
            const int y = (int)(cell / (uint32_t)a.W);
            const int x = (int)(cell - (uint32_t)y * (uint32_t)a.W);
            const Foot f = gather(a.h, a.W, a.H, __int2float_rn(x), __int2float_rn(y));
            const float ox = __fsub_rn(1.0f, f.fx), oy = __fsub_rn(1.0f, f.fy);
            const float ga = __fadd_rn(__fmul_rn(__fsub_rn(f.h10, f.h00), oy), __fmul_rn(__fsub_rn(f.h11, f.h01), f.fy));
            const float gb = __fadd_rn(__fmul_rn(__fsub_rn(f.h01, f.h00), ox), __fmul_rn(__fsub_rn(f.h11, f.h10), f.fx));
            const float gn2 = __fadd_rn(__fmul_rn(ga, ga), __fmul_rn(gb, gb));
            st.xy = (uint32_t)x | ((uint32_t)y << 16);
            st.z0 = bilinear(f, ox, oy);
            st.d0x = 0.0f;
            st.d0y = 0.0f;
            if (gn2 != 0.0f) {
                const float inv = __frcp_rn(__fsqrt_rn(gn2));
                st.d0x = __fmul_rn(-ga, inv);
                st.d0y = __fmul_rn(-gb, inv);
            }
            atomicAdd(a.count + cell, a.N);
        } else {
            st.xy = ~0u;
            st.z0 = st.d0x = st.d0y = 0.0f;
        }
        a.starts[ci] = st;
    }
}

__global__ void __launch_bounds__(SIM_THREADS) k_simulate(const __grid_constant__ SimArgs a)
{
    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;

    uint32_t n_cells = a.n_cells_max;
    if (a.n_cells_dev) n_cells = min(n_cells, *a.n_cells_dev);

    // warp-uniform cursor over (release-list entry, particle) and the end of
    // the current cell group
    uint32_t cur_ci = 0, cur_j = 0, end_ci = 0;
    bool exhausted = (n_cells == 0u);

    // lane state: position, its footprint and height, direction, energy,
    // recorded moves n (n == 0 only before the first move, when the footprint
    // registers are not used).  A dead lane keeps a position inside the grid,
    // so the loads it issues in the branch-free body stay in bounds.
    bool live = false;
    uint32_t cell = 0, j = 0, n = 0;
    float u = 0.f, v = 0.f, z = 0.f, dx = 0.f, dy = 0.f, e = 0.f;
    float fx = 0.f, fy = 0.f, h00 = 0.f, h10 = 0.f, h01 = 0.f, h11 = 0.f;

    unsigned long long my_steps = 0;
    unsigned my_traj = 0, my_exit = 0, my_cap = 0, my_bad = 0;

    while (true) {
        // ---- refill idle lanes (one round per move) ------------------------
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        if (idle != 0u && !exhausted) {
            if (cur_ci >= end_ci) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&a.ws->next_cell, (unsigned long long)a.cells_per_fetch);
                base = __shfl_sync(0xffffffffu, base, 0);
                exhausted = base >= n_cells;
                cur_ci = (uint32_t)min(base, (unsigned long long)n_cells);
                cur_j = 0;
                end_ci = (uint32_t)min((unsigned long long)n_cells, base + a.cells_per_fetch);
            }
            if (!exhausted) {
                // particles left in the group (capped at 32)
                const unsigned long long left = (unsigned long long)(end_ci - cur_ci) * a.N - cur_j;
                const unsigned avail = left < 32ull ? (unsigned)left : 32u;
                const unsigned want = (unsigned)__popc(idle);
                const unsigned take = want < avail ? want : avail;
                const unsigned rank = (unsigned)__popc(idle & lane_lt);
                const bool mine = ((idle >> lane) & 1u) && rank < take;
                uint32_t ci = cur_ci, jj = cur_j;
                advance(ci, jj, rank < take ? rank : 0u, a.N);
                uint4 st = make_uint4(~0u, 0u, 0u, 0u);
                if (mine) st = __ldg(reinterpret_cast<const uint4*>(a.starts) + ci);
                const bool ok = mine && st.x != ~0u;
                my_bad += (mine && !ok) ? 1u : 0u;  // release index outside the grid: skipped, reported
                const uint32_t sx = st.x & 0xffffu, sy = st.x >> 16;
                cell = ok ? sy * (uint32_t)a.W + sx : cell;
                j = ok ? jj : j;
                u = ok ? __int2float_rn((int)sx) : u;
                v = ok ? __int2float_rn((int)sy) : v;
                z = ok ? __uint_as_float(st.y) : z;
                dx = ok ? __uint_as_float(st.z) : dx;
                dy = ok ? __uint_as_float(st.w) : dy;
                n = ok ? 0u : n;
                e = ok ? 0.0f : e;
                const bool cap0 = ok && a.max_steps == 0u;  // capped at the release visit
                my_cap += cap0 ? 1u : 0u;
                my_traj += cap0 ? 1u : 0u;
                live = live || (ok && !cap0);
                advance(cur_ci, cur_j, take, a.N);
            }
        }
        const unsigned active = __ballot_sync(0xffffffffu, live);
        if (active == 0u) {
            if (exhausted) break;
            continue;
        }

        // ---- one move: direction at p, draw, step, energy at p' ------------
        // (every lane computes; only live lanes record and update)
        const float ox = __fsub_rn(1.0f, fx), oy = __fsub_rn(1.0f, fy);
        // steepest descent of the bilinear patch at p; the previous direction
        // when flat.  Before the first move d holds d_0 = g(p_0) from the
        // start record, which is also the steepest descent at p_0.
        const float ga = __fadd_rn(__fmul_rn(__fsub_rn(h10, h00), oy), __fmul_rn(__fsub_rn(h11, h01), fy));
        const float gb = __fadd_rn(__fmul_rn(__fsub_rn(h01, h00), ox), __fmul_rn(__fsub_rn(h11, h10), fx));
        const float gn2 = __fadd_rn(__fmul_rn(ga, ga), __fmul_rn(gb, gb));
        const float ginv = __frcp_rn(__fsqrt_rn(gn2));
        const bool keep = (gn2 == 0.0f) || (n == 0u);
        const float gx = keep ? dx : __fmul_rn(-ga, ginv);
        const float gy = keep ? dy : __fmul_rn(-gb, ginv);

        const uint4 w = philox4x32_10(make_uint4(cell, j, n >> 1, 0u), a.rk0, a.rk1);
        const bool odd = (n & 1u) != 0u;
        const float xix = uniform_pm1(odd ? w.z : w.x);
        const float xiy = uniform_pm1(odd ? w.w : w.y);
        const float rx = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dx), __fmul_rn(a.oneP, gx)), __fmul_rn(a.R, xix));
        const float ry = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dy), __fmul_rn(a.oneP, gy)), __fmul_rn(a.R, xiy));
        const float r2 = __fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry));
        const float rinv = __frcp_rn(__fsqrt_rn(r2));
        const bool zero_dir = (r2 == 0.0f);
        const float ndx = __fmul_rn(rx, rinv), ndy = __fmul_rn(ry, rinv);
        const float u1 = __fadd_rn(u, __fmul_rn(a.s, ndx));
        const float v1 = __fadd_rn(v, __fmul_rn(a.s, ndy));
        const bool inside = !zero_dir && u1 >= 0.0f && u1 <= a.Wm1 && v1 >= 0.0f && v1 <= a.Hm1;

        // footprint at p' (at p when p' is outside, so every load stays in the grid)
        const Foot f = gather(a.h, a.W, a.H, inside ? u1 : u, inside ? v1 : v);
        const float z1 = bilinear(f, __fsub_rn(1.0f, f.fx), __fsub_rn(1.0f, f.fy));
        const float e1 = __fsub_rn(__fadd_rn(__fsub_rn(e, __fmul_rn(a.kD, e)), __fsub_rn(z, z1)), a.muD);
        const bool moved = live && inside && e1 > 0.0f;

        // the visit: two fire-and-forget reductions per lane that moved (the
        // L2 absorbs lanes of a warp that hit the same cell more cheaply than
        // merging them in the warp first)
        const uint32_t vidx = (uint32_t)(f.j0 + (f.fy >= 0.5f ? 1 : 0)) * (uint32_t)a.W +
                              (uint32_t)(f.i0 + (f.fx >= 0.5f ? 1 : 0));
        if (moved) {
            atomicAdd(a.count + vidx, 1u);
            atomicMax(reinterpret_cast<unsigned*>(a.maxe) + vidx, __float_as_uint(e1));
        }

        u = moved ? u1 : u;
        v = moved ? v1 : v;
        z = moved ? z1 : z;
        e = moved ? e1 : e;
        dx = moved ? ndx : dx;
        dy = moved ? ndy : dy;
        fx = moved ? f.fx : fx;
        fy = moved ? f.fy : fy;
        h00 = moved ? f.h00 : h00;
        h10 = moved ? f.h10 : h10;
        h01 = moved ? f.h01 : h01;
        h11 = moved ? f.h11 : h11;
        n += moved ? 1u : 0u;
        my_steps += moved ? 1u : 0u;
        const bool capped = moved && n == a.max_steps;
        const bool ended = live && (!moved || capped);
        my_cap += capped ? 1u : 0u;
        my_exit += (live && !inside && !zero_dir) ? 1u : 0u;  // the other ends are stops
        my_traj += ended ? 1u : 0u;
        live = live && !ended;
    }

    // ---- statistics -----------------------------------------------------
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_steps += __shfl_xor_sync(0xffffffffu, my_steps, o);
        my_traj += __shfl_xor_sync(0xffffffffu, my_traj, o);
        my_exit += __shfl_xor_sync(0xffffffffu, my_exit, o);
        my_cap += __shfl_xor_sync(0xffffffffu, my_cap, o);
        my_bad += __shfl_xor_sync(0xffffffffu, my_bad, o);
    }
    if (lane == 0) {
        atomicAdd(&a.ws->total_steps, my_steps);
        atomicAdd(&a.ws->n_traj, (unsigned long long)my_traj);
        atomicAdd(&a.ws->n_exited, (unsigned long long)my_exit);
        atomicAdd(&a.ws->n_capped, (unsigned long long)my_cap);
        atomicAdd(&a.ws->n_stopped, (unsigned long long)(my_traj - my_exit - my_cap));
        if (my_bad) atomicAdd(&a.ws->n_rejected, (unsigned long long)my_bad);
    }
}

static int sim_blocks_per_sm()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_simulate, SIM_THREADS, 0) != cudaSuccess || b < 1)
            b = 1;
        cached[dev] = b;
    }
    return cached[dev];
}

static bool params_ok(const awo_sim_params* p, float cs)
{
    if (!p) return false;
    if (!(p->persistence >= 0.0f && p->persistence <= 1.0f)) return false;
    if (!(p->randomness >= 0.0f) || !(p->randomness < 3.0e38f)) return false;
    if (!(p->mu >= 0.0f) || !(p->mu < 3.0e38f)) return false;
    if (!(p->drag_k >= 0.0f) || !(p->drag_k < 3.0e38f)) return false;
    if (!(p->step_scale > 0.0f) || !(p->step_scale <= 1.0f)) return false;
    if (!(p->gravity > 0.0f) || !(p->gravity < 3.0e38f)) return false;
    float D = p->step_scale * cs;
    float kD = p->drag_k * D;
    if (!(kD < 1.0f)) return false;
    if ((p->flags & ~AWO_SIM_CLEAR_OUTPUTS) != 0u) return false;
    return true;
}

}  // namespace awo

using namespace awo;

static size_t starts_offset() { return 256; }

extern "C" size_t awo_simulate_workspace_bytes(uint32_t n_cells_max)
{
    return starts_offset() + (size_t)n_cells_max * sizeof(CellStart);
}

extern "C" awo_status awo_simulate(const float* d_h, awo_grid g, const uint32_t* d_cells, const uint32_t* d_n_cells,
                                   uint32_t n_cells_max, const awo_sim_params* p, uint32_t* d_count, float* d_maxe,
                                   awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream)
{
    if (!d_h || !d_count || !d_maxe || !d_ws || !grid_ok(g)) return AWO_EINVAL;
    if (n_cells_max > 0 && !d_cells) return AWO_EINVAL;
    if (!params_ok(p, g.cell_size)) return AWO_EINVAL;
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
    a.invW = 1.0f / (float)g.width;
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
    a.cells_per_fetch = a.N >= SIM_FETCH_ITEMS ? 1u : (SIM_FETCH_ITEMS + a.N - 1u) / a.N;
    uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk0[r] = k0;
        a.rk1[r] = k1;
        k0 += 0x9E3779B9u;  // Weyl key schedule of Philox4x32
        k1 += 0xBB67AE85u;
    }
    a.count = d_count;
    a.maxe = d_maxe;
    a.ws = ws;
    a.starts = reinterpret_cast<CellStart*>(static_cast<char*>(d_ws) + starts_offset());

    if (a.N > 0 && (n_cells_max > 0)) {
        const unsigned pro_blocks = stream_blocks((int64_t)n_cells_max, 256);
        k_sim_starts<<<pro_blocks, 256, 0, s>>>(a);
        unsigned blocks = (unsigned)(sm_count() * sim_blocks_per_sm());
        k_simulate<<<blocks, SIM_THREADS, 0, s>>>(a);
        awo_status st = launch_status();
        if (st != AWO_OK) return st;
    }
    if (d_stats) {
        if (cudaMemcpyAsync(d_stats, &ws->total_steps, sizeof(awo_sim_stats), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return AWO_ECUDA;
    }
    return AWO_OK;
}
