// awo_soft.cu -- soft-deposit particles and their gradient (differentiable
// extension of the Sec. 5.2 trajectory node; the paper has no gradients).
//
// Forward: each particle follows exactly the path of the hard mode (same
// FP32 direction and move arithmetic, same Philox draws) but is not stopped
// by its energy: it carries a survival S (S_0 = 1) multiplied at every move
// by sigma(e / tau), deposits the lost mass w (S_{n-1} - S_n) at the cell it
// reached, and ends when it leaves the grid, has no direction, reaches
// max_steps, or S < 1e-7; the remainder w S goes to the last cell.  Deposits
// are 64-bit fixed point (2^-32 per unit weight) accumulated with integer
// atomics, so the deposit raster is deterministic; cumulative quantisation
// makes every particle deposit exactly round(w 2^32).
//
// Backward: the path does not depend on mu, k or the weights -- only the
// energy recurrence e' = (e - k D e) + (z - z') - mu D does.  The kernel
// recomputes each particle from its start record (frozen draws: the Philox
// counter is (cell, particle, move)) and carries two forward tangents,
// de/dmu and de/dk, and the matching tangents of S, accumulating the
// vector-Jacobian product sum_cells G_c dD_c/dtheta along the way.  That is
// the exact gradient in one pass with O(1) state per particle: no step or
// segment has to be stored, because the state that is not carried (the path)
// does not depend on the parameters.  Per-particle sums are FP32; the sums
// over particles (parameter gradient reductions) are FP64.
#include <cstring>

#include "awo_particle.cuh"

namespace awo {

struct SoftArgs {
    const float* h;
    int W, H;
    float Wm1, Hm1, P, oneP, R, s;
    float kD, muD, D;      // drag_k*D, mu*D, D = s*cell_size (metres)
    float mu, k;           // for the log-parameter chain rule
    float inv_tau;
    uint32_t max_steps, N, n_grid;
    KeysTable keys;
    const uint32_t* cells;
    const uint32_t* n_cells_dev;
    uint32_t n_cells_max;
    const float* weight;   // per release entry
    CellStart* starts;
    unsigned long long* deposit;  // fixed point, W*H
    const float* grad;     // dL/dD, W*H (backward)
    double* grad_theta;    // 2 (backward)
    double* grad_w;        // per release entry, FP64 scratch (backward)
    unsigned long long* stats;  // 6
    unsigned long long* next_item;  // work counter (zeroed with the stats)
    cudaTextureObject_t tex;    // texture view of h for the footprint gathers (k_soft<_, true>), or 0
};

constexpr float SOFT_S_MIN = 1e-7f;
constexpr float FIX_SCALE = 4294967296.0f;  // 2^32

__device__ __forceinline__ uint32_t soft_count(const SoftArgs& a)
{
    uint32_t n = a.n_cells_max;
    if (a.n_cells_dev) n = min(n, *a.n_cells_dev);
    return n;
}

// Start records, and the particles of entries outside the grid counted as
// rejected (the particle kernel skips them).
__global__ void __launch_bounds__(256) k_soft_starts(const __grid_constant__ SoftArgs a)
{
    const uint32_t n_cells = soft_count(a);
    unsigned long long bad = 0ull;
    for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < n_cells; ci += gridDim.x * blockDim.x) {
        const CellStart st = cell_start(a.h, a.W, a.H, a.n_grid, __ldg(a.cells + ci));
        a.starts[ci] = st;
        bad += st.xy == ~0u ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad && a.stats) atomicAdd(a.stats + 5, bad * a.N);
}

constexpr int SOFT_THREADS = 128;
constexpr uint32_t SOFT_CHUNK_MAX = 1024;
constexpr uint32_t SOFT_CHUNKS_PER_WARP = 16;
constexpr uint32_t SOFT_REFILL_IDLE = 4;

// Soft particles, GRAD = false: deposits; GRAD = true: gradient sums.  TEX:
// footprints by texture gather through a.tex (else by loads).  Persistent,
// one lane per particle, with the lane refill of the particle kernels
// (awo_simulate.cu): a warp takes chunks of consecutive particles (entry,
// then particle j) and restarts a lane whose particle has ended, so a long
// particle does not keep the other lanes of its warp idle.  Each loop
// iteration is two moves from one Philox block (moves n and n + 1 take words
// 0-1 and 2-3 of block n >> 1; lanes start at n = 0 and move in pairs).  Per
// particle the arithmetic is that of the hard mode's moves plus the
// survival, its tangents and the deposits, in a fixed order.
template <bool GRAD, bool TEX>
__global__ void __launch_bounds__(SOFT_THREADS) k_soft(const __grid_constant__ SoftArgs a)
{
    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;
    const uint32_t n_cells = soft_count(a);
    const unsigned long long total = (unsigned long long)n_cells * a.N;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long chunk = total / (warps * SOFT_CHUNKS_PER_WARP);
    chunk = chunk < 32ull ? 32ull : (chunk > SOFT_CHUNK_MAX ? (unsigned long long)SOFT_CHUNK_MAX : chunk);
    chunk &= ~31ull;
    unsigned long long cur_t = 0ull, end_t = 0ull;
    uint32_t cur_ci = 0u, cur_j = 0u, idle_acc = 0u;
    bool exhausted = (total == 0ull);

    // the lane's particle
    bool live = false;
    uint32_t ci = 0u, cell = 0u, j = 0u, n = 0u, last = 0u;
    float u = 0.f, v = 0.f, z = 0.f, dx = 0.f, dy = 0.f, e = 0.f, S = 1.f, w = 0.f;
    float fx = 0.f, fy = 0.f, h00 = 0.f, h10 = 0.f, h01 = 0.f, h11 = 0.f;
    long long Q = 0;  // forward: cumulative fixed-point deposit
    float tmu = 0.f, tk = 0.f, smu = 0.f, sk = 0.f, acc_mu = 0.f, acc_k = 0.f, acc_w = 0.f;  // backward
    // the lane's counters
    double sum_mu = 0.0, sum_k = 0.0;
    unsigned long long steps = 0ull, traj = 0ull;
    bool pend = false;  // backward: an ended particle whose FP64 sums are still to be added

    // End of the lane's particle: the remainder w S to its last cell
    // (forward), or the last cell's term (backward; its FP64 sums are added
    // by flush(), at the next refill round or at the end, where the warp's
    // ended lanes take them together: FP64 issue slots are scarce on GB300,
    // and issued here they would be taken once for every move at which some
    // lane of the warp ends).
    auto finish = [&]() {
        steps += n;
        if (GRAD) {
            const float G = __ldg(a.grad + last);
            acc_mu += G * smu;
            acc_k += G * sk;
            acc_w += G * S;
            pend = true;
        } else {
            const long long Wq = __float2ll_rn(w * FIX_SCALE);
            if (Wq != Q) atomicAdd(a.deposit + last, (unsigned long long)(Wq - Q));
        }
        live = false;
    };
    auto flush = [&]() {
        if (GRAD && pend) {
            sum_mu += (double)w * (double)acc_mu * (double)a.mu;  // d/dlog(mu) = mu d/dmu
            sum_k += (double)w * (double)acc_k * (double)a.k;
            atomicAdd(a.grad_w + ci, (double)acc_w);
            pend = false;
        }
    };

    // One move of a live lane's particle with random words WX, WY (the move
    // loop of the hard mode: a particle ends at max_steps moves, with no
    // direction, outside the grid, or when S < 1e-7 after a move).
    auto move = [&](uint32_t WX, uint32_t WY) {
        if (!live) return;
        if (n >= a.max_steps) {
            finish();
            return;
        }
        const float ox = __fsub_rn(1.0f, fx), oy = __fsub_rn(1.0f, fy);
        const float ga = __fadd_rn(__fmul_rn(__fsub_rn(h10, h00), oy), __fmul_rn(__fsub_rn(h11, h01), fy));
        const float gb = __fadd_rn(__fmul_rn(__fsub_rn(h01, h00), ox), __fmul_rn(__fsub_rn(h11, h10), fx));
        const float gn2 = __fadd_rn(__fmul_rn(ga, ga), __fmul_rn(gb, gb));
        float gx = dx, gy = dy;
        if (n != 0u && gn2 != 0.0f) {
            const float ginv = rcp_sqrt_rn(gn2);
            gx = __fmul_rn(-ga, ginv);
            gy = __fmul_rn(-gb, ginv);
        }
        const float xix = uniform_pm1(WX);
        const float xiy = uniform_pm1(WY);
        const float rx = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dx), __fmul_rn(a.oneP, gx)), __fmul_rn(a.R, xix));
        const float ry = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dy), __fmul_rn(a.oneP, gy)), __fmul_rn(a.R, xiy));
        const float r2 = __fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry));
        if (r2 == 0.0f) {
            finish();
            return;
        }
        const float rinv = rcp_sqrt_rn(r2);
        dx = __fmul_rn(rx, rinv);
        dy = __fmul_rn(ry, rinv);
        const float u1 = __fadd_rn(u, __fmul_rn(a.s, dx));
        const float v1 = __fadd_rn(v, __fmul_rn(a.s, dy));
        if (!(u1 >= 0.0f && u1 <= a.Wm1 && v1 >= 0.0f && v1 <= a.Hm1)) {
            finish();
            return;
        }
        const Foot f = foot_at<TEX ? 1 : 0>(a, u1, v1);
        const float z1 = bilinear(f, __fsub_rn(1.0f, f.fx), __fsub_rn(1.0f, f.fy));
        const float e1 = __fsub_rn(__fadd_rn(__fsub_rn(e, __fmul_rn(a.kD, e)), __fsub_rn(z, z1)), a.muD);
        const float sig = 1.0f / (1.0f + expf(-e1 * a.inv_tau));
        const float S1 = S * sig;
        const uint32_t c1 = (uint32_t)(f.j0 + (f.fy >= 0.5f ? 1 : 0)) * (uint32_t)a.W +
                            (uint32_t)(f.i0 + (f.fx >= 0.5f ? 1 : 0));
        if (GRAD) {
            const float tmu1 = (1.0f - a.kD) * tmu - a.D;
            const float tk1 = (1.0f - a.kD) * tk - a.D * e;
            const float ds = sig * (1.0f - sig) * a.inv_tau;
            const float smu1 = smu * sig + S * ds * tmu1;
            const float sk1 = sk * sig + S * ds * tk1;
            const float G = __ldg(a.grad + c1);
            acc_mu += G * (smu - smu1);
            acc_k += G * (sk - sk1);
            acc_w += G * (S - S1);
            tmu = tmu1;
            tk = tk1;
            smu = smu1;
            sk = sk1;
        } else {
            const long long Q1 = __float2ll_rn((1.0f - S1) * w * FIX_SCALE);
            if (Q1 != Q) atomicAdd(a.deposit + c1, (unsigned long long)(Q1 - Q));
            Q = Q1;
        }
        u = u1;
        v = v1;
        z = z1;
        e = e1;
        S = S1;
        fx = f.fx;
        fy = f.fy;
        h00 = f.h00;
        h10 = f.h10;
        h01 = f.h01;
        h11 = f.h11;
        last = c1;
        ++n;
        if (S1 < SOFT_S_MIN) finish();
    };

    while (true) {
        // ---- refill idle lanes (as in k_simulate) ----
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        idle_acc += (uint32_t)__popc(idle);
        if (idle != 0u && idle_acc >= SOFT_REFILL_IDLE && !exhausted) {
            idle_acc = 0u;
            flush();
            if (cur_t >= end_t) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.next_item, chunk);
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
                const unsigned long long left = end_t - cur_t;
                const unsigned avail = left < 32ull ? (unsigned)left : 32u;
                const unsigned want = (unsigned)__popc(idle);
                const unsigned take = want < avail ? want : avail;
                const unsigned rank = (unsigned)__popc(idle & lane_lt);
                const bool mine = ((idle >> lane) & 1u) && rank < take;
                uint32_t c = cur_ci, jj = cur_j;
                advance(c, jj, rank < take ? rank : 0u, a.N);
                uint4 st = make_uint4(~0u, 0u, 0u, 0u);
                if (mine) st = __ldg(reinterpret_cast<const uint4*>(a.starts) + c);
                // entries outside the grid are counted by k_soft_starts
                if (mine && st.x != ~0u) {
                    const uint32_t sx = st.x & 0xffffu, sy = st.x >> 16;
                    live = true;
                    ci = c;
                    j = jj;
                    cell = sy * (uint32_t)a.W + sx;
                    last = cell;
                    n = 0u;
                    u = __int2float_rn((int)sx);
                    v = __int2float_rn((int)sy);
                    z = __uint_as_float(st.y);
                    dx = __uint_as_float(st.z);
                    dy = __uint_as_float(st.w);
                    e = 0.f;
                    S = 1.f;
                    w = __ldg(a.weight + c);
                    fx = fy = h00 = h10 = h01 = h11 = 0.f;
                    Q = 0;
                    tmu = tk = smu = sk = acc_mu = acc_k = acc_w = 0.f;
                    ++traj;
                }
                advance(cur_ci, cur_j, take, a.N);
                cur_t += take;
            }
        }
        if (__ballot_sync(0xffffffffu, live) == 0u) {
            if (exhausted) break;
            continue;
        }
        // moves n and n + 1 from one Philox block: every live lane is at an even n
        const uint4 r = philox4x32_10(make_uint4(cell, j, n >> 1, 0u), a.keys);
        move(r.x, r.y);
        move(r.z, r.w);
    }
    flush();
    // FP64 reductions over the warp, then one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum_mu += __shfl_xor_sync(0xffffffffu, sum_mu, o);
        sum_k += __shfl_xor_sync(0xffffffffu, sum_k, o);
        steps += __shfl_xor_sync(0xffffffffu, steps, o);
        traj += __shfl_xor_sync(0xffffffffu, traj, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (GRAD) {
            atomicAdd(a.grad_theta + 0, sum_mu);
            atomicAdd(a.grad_theta + 1, sum_k);
        }
        if (a.stats) {
            if (steps) atomicAdd(a.stats + 0, steps);
            if (traj) atomicAdd(a.stats + 1, traj);
        }
    }
}

__global__ void k_to_float(const double* __restrict__ in, uint32_t n_max, const uint32_t* n_dev,
                           float* __restrict__ out)
{
    uint32_t n = n_max;
    if (n_dev) n = min(n, *n_dev);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void k_fixed_to_real(const long long* __restrict__ q, int64_t n, double scale, double* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)q[i] * scale;
}

struct SoftWs {
    unsigned long long stats[6];
    unsigned long long next_item;  // work counter of k_soft, in particles
    unsigned long long pad;
};
constexpr size_t SOFT_STARTS_OFF = 256;

static size_t soft_ws_bytes(uint32_t n_cells_max)
{
    return SOFT_STARTS_OFF + (size_t)n_cells_max * sizeof(CellStart) + (size_t)n_cells_max * sizeof(double) + 64;
}

static awo_status soft_setup(SoftArgs& a, const float* d_h, awo_grid g, const uint32_t* d_cells,
                             const uint32_t* d_n_cells, uint32_t n_cells_max, const float* d_weight,
                             const awo_sim_params* p, float tau, void* d_ws, size_t ws_bytes, cudaStream_t s)
{
    if (!d_h || !d_ws || !grid_ok(g) || !sim_params_ok(p, g.cell_size) || p->release_log2 != 0) return AWO_EINVAL;
    if (n_cells_max > 0 && (!d_cells || !d_weight)) return AWO_EINVAL;
    if (!(tau > 0.0f) || !(tau < 3.0e38f)) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0) return AWO_EINVAL;
    if (ws_bytes < soft_ws_bytes(n_cells_max)) return AWO_ENOMEM;
    memset(&a, 0, sizeof(a));
    const float D = p->step_scale * g.cell_size;
    a.h = d_h;
    a.W = g.width;
    a.H = g.height;
    a.Wm1 = (float)(g.width - 1);
    a.Hm1 = (float)(g.height - 1);
    a.P = p->persistence;
    a.oneP = 1.0f - p->persistence;
    a.R = p->randomness;
    a.s = p->step_scale;
    a.D = D;
    a.kD = p->drag_k * D;
    a.muD = p->mu * D;
    a.mu = p->mu;
    a.k = p->drag_k;
    a.inv_tau = 1.0f / tau;
    a.max_steps = p->max_steps;
    a.N = p->traj_per_cell;
    a.n_grid = (uint32_t)cells_of(g);
    uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.keys.k0[r] = k0;
        a.keys.k1[r] = k1;
        k0 += 0x9E3779B9u;  // Weyl key schedule of Philox4x32
        k1 += 0xBB67AE85u;
    }
    a.cells = d_cells;
    a.n_cells_dev = d_n_cells;
    a.n_cells_max = n_cells_max;
    a.weight = d_weight;
    SoftWs* ws = static_cast<SoftWs*>(d_ws);
    a.stats = ws->stats;
    a.next_item = &ws->next_item;
    a.starts = reinterpret_cast<CellStart*>(static_cast<char*>(d_ws) + SOFT_STARTS_OFF);
    a.grad_w = reinterpret_cast<double*>(static_cast<char*>(d_ws) + SOFT_STARTS_OFF +
                                         (size_t)n_cells_max * sizeof(CellStart));
    a.tex = dem_texture(d_h, g, s);
    return AWO_OK;
}

// Persistent grid of k_soft: the SMs times the resident blocks of the instance.
template <bool GRAD, bool TEX>
static unsigned soft_blocks()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_soft<GRAD, TEX>, SOFT_THREADS, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        cached[dev] = b;
    }
    return (unsigned)(sm_count() * cached[dev]);
}

}  // namespace awo

using namespace awo;

extern "C" size_t awo_soft_workspace_bytes(uint32_t n_cells_max) { return soft_ws_bytes(n_cells_max); }

extern "C" awo_status awo_soft_forward(const float* d_h, awo_grid g, const uint32_t* d_cells,
                                       const uint32_t* d_n_cells, uint32_t n_cells_max, const float* d_weight,
                                       const awo_sim_params* p, float tau, int64_t* d_deposit,
                                       awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream)
{
    SoftArgs a;
    awo_status st =
        soft_setup(a, d_h, g, d_cells, d_n_cells, n_cells_max, d_weight, p, tau, d_ws, ws_bytes, as_stream(stream));
    if (st != AWO_OK) return st;
    if (!d_deposit || (((uintptr_t)d_deposit) & 7u) != 0) return AWO_EINVAL;
    a.deposit = reinterpret_cast<unsigned long long*>(d_deposit);
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(a.stats, 0, sizeof(SoftWs), s) != cudaSuccess) return AWO_ECUDA;
    if (p->flags & AWO_SIM_CLEAR_OUTPUTS)
        if (cudaMemsetAsync(d_deposit, 0, (size_t)cells_of(g) * sizeof(int64_t), s) != cudaSuccess) return AWO_ECUDA;
    if (a.N > 0 && n_cells_max > 0) {
        k_soft_starts<<<stream_blocks((int64_t)n_cells_max, 256), 256, 0, s>>>(a);
        if (a.tex)
            k_soft<false, true><<<soft_blocks<false, true>(), SOFT_THREADS, 0, s>>>(a);
        else
            k_soft<false, false><<<soft_blocks<false, false>(), SOFT_THREADS, 0, s>>>(a);
        st = launch_status();
        if (st != AWO_OK) return st;
    }
    if (d_stats && cudaMemcpyAsync(d_stats, a.stats, sizeof(awo_sim_stats), cudaMemcpyDeviceToDevice, s) !=
                       cudaSuccess)
        return AWO_ECUDA;
    return AWO_OK;
}

extern "C" awo_status awo_soft_backward(const float* d_h, awo_grid g, const uint32_t* d_cells,
                                        const uint32_t* d_n_cells, uint32_t n_cells_max, const float* d_weight,
                                        const awo_sim_params* p, float tau, const float* d_grad_deposit,
                                        double* d_grad_theta, float* d_grad_weight, void* d_ws, size_t ws_bytes,
                                        void* stream)
{
    SoftArgs a;
    awo_status st =
        soft_setup(a, d_h, g, d_cells, d_n_cells, n_cells_max, d_weight, p, tau, d_ws, ws_bytes, as_stream(stream));
    if (st != AWO_OK) return st;
    if (!d_grad_deposit || !d_grad_theta || (n_cells_max > 0 && !d_grad_weight)) return AWO_EINVAL;
    a.grad = d_grad_deposit;
    a.grad_theta = d_grad_theta;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(a.stats, 0, sizeof(SoftWs), s) != cudaSuccess) return AWO_ECUDA;
    if (cudaMemsetAsync(d_grad_theta, 0, 2 * sizeof(double), s) != cudaSuccess) return AWO_ECUDA;
    if (n_cells_max > 0 && cudaMemsetAsync(a.grad_w, 0, (size_t)n_cells_max * sizeof(double), s) != cudaSuccess)
        return AWO_ECUDA;
    if (a.N > 0 && n_cells_max > 0) {
        k_soft_starts<<<stream_blocks((int64_t)n_cells_max, 256), 256, 0, s>>>(a);
        if (a.tex)
            k_soft<true, true><<<soft_blocks<true, true>(), SOFT_THREADS, 0, s>>>(a);
        else
            k_soft<true, false><<<soft_blocks<true, false>(), SOFT_THREADS, 0, s>>>(a);
    }
    if (n_cells_max > 0)
        k_to_float<<<stream_blocks((int64_t)n_cells_max, 256), 256, 0, s>>>(a.grad_w, n_cells_max, d_n_cells,
                                                                             d_grad_weight);
    return launch_status();
}

extern "C" awo_status awo_fixed_to_real(const int64_t* d_q, int64_t n, double* d_out, void* stream)
{
    if (!d_q || !d_out || n < 0) return AWO_EINVAL;
    if (n == 0) return AWO_OK;
    k_fixed_to_real<<<stream_blocks(n, 256), 256, 0, as_stream(stream)>>>(reinterpret_cast<const long long*>(d_q), n,
                                                                           1.0 / 4294967296.0, d_out);
    return launch_status();
}
