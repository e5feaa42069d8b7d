// awo_simulate.cu -- Monte-Carlo avalanche trajectories (Sec. 5.2).
//
// Design (GB300):
//  * Persistent kernel, one lane per particle.  Each warp takes chunks of
//    consecutive work items (item t = release-list index * N + j) from a
//    global counter and refills a lane as soon as its particle ends, so lanes
//    never idle behind a long particle of the same warp.  Consecutive items
//    are particles of the same or neighbouring release cells, so the lanes of
//    a warp, and the warps in flight, touch a compact region of the DEM and
//    the rasters (it stays L2-resident even when the DEM does not).
//  * The loop body is the same for a fresh particle and a moving one: gather
//    the 4-texel footprint at the current position, account for the move that
//    arrived there (or for the release visit), then draw and move.  New and
//    old lanes of a warp therefore execute one instruction stream.
//  * Visits go to the rasters with fire-and-forget reductions (RED.ADD on the
//    count, RED.MAX on the float bits of the non-negative energy); lanes of a
//    warp that hit the same cell are merged first (__match_any_sync), which
//    removes most reductions in the first moves, when all particles of a cell
//    are still together.
//  * Arithmetic is FP32 with explicit round-to-nearest intrinsics: no fused
//    multiply-add, IEEE sqrt and reciprocal, so every particle follows the
//    formulas of awo.h bit for bit.
#include "awo_internal.cuh"

namespace awo {

struct SimWorkspace {
    unsigned long long next_item;  // global work counter
    unsigned long long total_steps, n_traj, n_exited, n_capped, n_stopped, n_rejected;
    unsigned long long pad;
};
static_assert(sizeof(SimWorkspace) == 64, "workspace layout");

struct SimArgs {
    const float* h;
    const uint32_t* cells;
    const uint32_t* n_cells_dev;
    uint32_t n_cells_max;
    int W, H;
    uint32_t n_grid;       // W*H
    float Wm1, Hm1;        // W-1, H-1 as floats (exact for W, H <= 2^24)
    float P, oneP, R, s;   // persistence, 1-P, randomness, step in cells
    float kD, muD;         // drag_k*D, mu*D  (D = s*cell_size)
    uint32_t N, max_steps;
    uint32_t key0, key1;
    uint32_t* count;
    float* maxe;
    SimWorkspace* ws;
};

constexpr int SIM_THREADS = 256;
constexpr uint32_t SIM_CHUNK = 256;  // items per global fetch

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// of the even words, word permutation with key injection, Weyl key bumps.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
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
    int i1 = min(f.i0 + 1, W - 1);
    int j1 = min(f.j0 + 1, H - 1);
    const float* r0 = h + (size_t)f.j0 * (size_t)W;
    const float* r1 = h + (size_t)j1 * (size_t)W;
    f.h00 = __ldg(r0 + f.i0);
    f.h10 = __ldg(r0 + i1);
    f.h01 = __ldg(r1 + f.i0);
    f.h11 = __ldg(r1 + i1);
    return f;
}

__device__ __forceinline__ float bilinear(const Foot& f)
{
    float ox = __fsub_rn(1.0f, f.fx), oy = __fsub_rn(1.0f, f.fy);
    float top = __fadd_rn(__fmul_rn(f.h00, ox), __fmul_rn(f.h10, f.fx));
    float bot = __fadd_rn(__fmul_rn(f.h01, ox), __fmul_rn(f.h11, f.fx));
    return __fadd_rn(__fmul_rn(top, oy), __fmul_rn(bot, f.fy));
}

// Steepest descent of the bilinear patch; fallback (fbx, fby) when flat.
__device__ __forceinline__ void downslope(const Foot& f, float fbx, float fby, float& gx, float& gy)
{
    float ox = __fsub_rn(1.0f, f.fx), oy = __fsub_rn(1.0f, f.fy);
    float a = __fadd_rn(__fmul_rn(__fsub_rn(f.h10, f.h00), oy), __fmul_rn(__fsub_rn(f.h11, f.h01), f.fy));
    float b = __fadd_rn(__fmul_rn(__fsub_rn(f.h01, f.h00), ox), __fmul_rn(__fsub_rn(f.h11, f.h10), f.fx));
    float n2 = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
    if (n2 == 0.0f) {
        gx = fbx;
        gy = fby;
    } else {
        float inv = __frcp_rn(__fsqrt_rn(n2));
        gx = __fmul_rn(-a, inv);
        gy = __fmul_rn(-b, inv);
    }
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
    int lane = threadIdx.x & 31;
    if (lane == __ffs(grp) - 1) {
        atomicAdd(count + idx, (unsigned)__popc(grp));
        if (emax != 0u) atomicMax(reinterpret_cast<unsigned*>(maxe) + idx, emax);
    }
}

__global__ void __launch_bounds__(SIM_THREADS) k_simulate(SimArgs a)
{
    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;

    uint64_t n_cells = a.n_cells_max;
    if (a.n_cells_dev) {
        uint32_t nd = *a.n_cells_dev;
        if (nd < n_cells) n_cells = nd;
    }
    const uint64_t total = n_cells * (uint64_t)a.N;

    // warp-uniform chunk of items
    uint64_t chunk_next = 0, chunk_end = 0;
    bool exhausted = (total == 0);

    // lane state
    bool live = false;
    bool fresh = false;
    uint32_t cell = 0, j = 0, n = 0;
    float u = 0.f, v = 0.f, dx = 0.f, dy = 0.f, e = 0.f, z = 0.f;

    unsigned long long my_steps = 0;
    unsigned my_traj = 0, my_exit = 0, my_cap = 0, my_stop = 0, my_bad = 0;

    while (true) {
        // ---- refill idle lanes from the warp's chunk --------------------
        unsigned idle = __ballot_sync(0xffffffffu, !live);
        while (idle != 0u && !exhausted) {
            if (chunk_next == chunk_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&a.ws->next_item, (unsigned long long)SIM_CHUNK);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= total) {
                    exhausted = true;
                    break;
                }
                chunk_next = base;
                chunk_end = base + SIM_CHUNK < total ? base + SIM_CHUNK : total;
            }
            unsigned avail = (unsigned)(chunk_end - chunk_next);
            unsigned want = (unsigned)__popc(idle);
            unsigned take = want < avail ? want : avail;
            unsigned rank = (unsigned)__popc(idle & lane_lt);
            if (((idle >> lane) & 1u) && rank < take) {
                uint64_t t = chunk_next + rank;
                uint64_t ci = t / a.N;
                j = (uint32_t)(t - ci * a.N);
                cell = __ldg(a.cells + ci);
                if (cell < a.n_grid) {
                    u = __int2float_rn((int)(cell % (uint32_t)a.W));
                    v = __int2float_rn((int)(cell / (uint32_t)a.W));
                    n = 0;
                    e = 0.f;
                    dx = 0.f;
                    dy = 0.f;
                    live = true;
                    fresh = true;
                } else {
                    ++my_bad;  // release index outside the grid: skipped, reported
                }
            }
            chunk_next += take;
            idle = __ballot_sync(0xffffffffu, !live);
        }
        unsigned active = __ballot_sync(0xffffffffu, live);
        if (active == 0u) break;
        if (!live) continue;

        // ---- footprint at the current position ------------------------
        Foot f = gather(a.h, a.W, a.H, u, v);
        float z1 = bilinear(f);
        bool alive = true;
        uint32_t vidx = (uint32_t)(f.j0 + (f.fy >= 0.5f ? 1 : 0)) * (uint32_t)a.W + (uint32_t)(f.i0 + (f.fx >= 0.5f ? 1 : 0));
        bool moved = !fresh;
        if (moved) {
            // energy of the move that arrived here
            float e1 = __fsub_rn(__fadd_rn(__fsub_rn(e, __fmul_rn(a.kD, e)), __fsub_rn(z, z1)), a.muD);
            if (!(e1 > 0.0f)) {
                alive = false;  // stopped before this position: not recorded
                ++my_stop;
                ++my_traj;
            } else {
                e = e1;
                ++n;
                ++my_steps;
            }
        }
        // visits: the release cell (e = 0, count only) or the new position
        unsigned rec = __ballot_sync(active, alive);
        if (alive) record(a.count, a.maxe, rec, vidx, e);  // e == 0 on the release visit

        if (alive && n == a.max_steps) {
            alive = false;
            ++my_cap;
            ++my_traj;
        }
        if (alive) {
            float gx, gy;
            downslope(f, fresh ? 0.0f : dx, fresh ? 0.0f : dy, gx, gy);
            if (fresh) {
                dx = gx;
                dy = gy;
            }
            uint4 w = philox4x32_10(make_uint4(cell, j, n >> 1, 0u), a.key0, a.key1);
            uint32_t wx = (n & 1u) ? w.z : w.x;
            uint32_t wy = (n & 1u) ? w.w : w.y;
            float xix = uniform_pm1(wx), xiy = uniform_pm1(wy);
            float rx = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dx), __fmul_rn(a.oneP, gx)), __fmul_rn(a.R, xix));
            float ry = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dy), __fmul_rn(a.oneP, gy)), __fmul_rn(a.R, xiy));
            float r2 = __fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry));
            if (r2 == 0.0f) {
                alive = false;
                ++my_stop;
                ++my_traj;
            } else {
                float inv = __frcp_rn(__fsqrt_rn(r2));
                dx = __fmul_rn(rx, inv);
                dy = __fmul_rn(ry, inv);
                float u1 = __fadd_rn(u, __fmul_rn(a.s, dx));
                float v1 = __fadd_rn(v, __fmul_rn(a.s, dy));
                if (!(u1 >= 0.0f && u1 <= a.Wm1 && v1 >= 0.0f && v1 <= a.Hm1)) {
                    alive = false;
                    ++my_exit;
                    ++my_traj;
                } else {
                    u = u1;
                    v = v1;
                    z = z1;
                }
            }
        }
        fresh = false;
        live = alive;
    }

    // ---- statistics -----------------------------------------------------
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_steps += __shfl_xor_sync(0xffffffffu, my_steps, o);
        my_traj += __shfl_xor_sync(0xffffffffu, my_traj, o);
        my_exit += __shfl_xor_sync(0xffffffffu, my_exit, o);
        my_cap += __shfl_xor_sync(0xffffffffu, my_cap, o);
        my_stop += __shfl_xor_sync(0xffffffffu, my_stop, o);
        my_bad += __shfl_xor_sync(0xffffffffu, my_bad, o);
    }
    if (lane == 0) {
        atomicAdd(&a.ws->total_steps, my_steps);
        atomicAdd(&a.ws->n_traj, (unsigned long long)my_traj);
        atomicAdd(&a.ws->n_exited, (unsigned long long)my_exit);
        atomicAdd(&a.ws->n_capped, (unsigned long long)my_cap);
        atomicAdd(&a.ws->n_stopped, (unsigned long long)my_stop);
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

extern "C" size_t awo_simulate_workspace_bytes(void) { return sizeof(SimWorkspace); }

extern "C" awo_status awo_simulate(const float* d_h, awo_grid g, const uint32_t* d_cells, const uint32_t* d_n_cells,
                                   uint32_t n_cells_max, const awo_sim_params* p, uint32_t* d_count, float* d_maxe,
                                   awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream)
{
    if (!d_h || !d_count || !d_maxe || !d_ws || !grid_ok(g)) return AWO_EINVAL;
    if (n_cells_max > 0 && !d_cells) return AWO_EINVAL;
    if (!params_ok(p, g.cell_size)) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0 || (((uintptr_t)d_count) & 3u) != 0 || (((uintptr_t)d_maxe) & 3u) != 0)
        return AWO_EINVAL;
    if (ws_bytes < sizeof(SimWorkspace)) return AWO_ENOMEM;
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
    a.key0 = (uint32_t)(p->seed & 0xffffffffu);
    a.key1 = (uint32_t)(p->seed >> 32);
    a.count = d_count;
    a.maxe = d_maxe;
    a.ws = ws;

    if (a.N > 0 && (n_cells_max > 0)) {
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
