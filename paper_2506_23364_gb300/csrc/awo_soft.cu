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

__global__ void __launch_bounds__(256) k_soft_starts(const __grid_constant__ SoftArgs a)
{
    const uint32_t n_cells = soft_count(a);
    for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < n_cells; ci += gridDim.x * blockDim.x)
        a.starts[ci] = cell_start(a.h, a.W, a.H, a.n_grid, __ldg(a.cells + ci));
}

// One soft particle.  GRAD = false: deposits; GRAD = true: gradient sums.
// TEX: footprints by texture gather through a.tex (else by loads).
template <bool GRAD, bool TEX>
__device__ __forceinline__ void soft_particle(const SoftArgs& a, uint32_t ci, uint32_t j, double& sum_mu,
                                              double& sum_k, unsigned long long& steps, bool& rejected)
{
    const uint4 st = __ldg(reinterpret_cast<const uint4*>(a.starts) + ci);
    if (st.x == ~0u) {
        rejected = true;
        return;
    }
    const float w = __ldg(a.weight + ci);
    const uint32_t sx = st.x & 0xffffu, sy = st.x >> 16;
    const uint32_t cell = sy * (uint32_t)a.W + sx;
    float u = __int2float_rn((int)sx), v = __int2float_rn((int)sy);
    float z = __uint_as_float(st.y), dx = __uint_as_float(st.z), dy = __uint_as_float(st.w);
    float fx = 0.f, fy = 0.f, h00 = 0.f, h10 = 0.f, h01 = 0.f, h11 = 0.f;
    float e = 0.f, S = 1.f;
    uint32_t last = cell;
    // forward: cumulative fixed-point deposit; backward: tangents and sums
    long long Q = 0;
    float tmu = 0.f, tk = 0.f, smu = 0.f, sk = 0.f, acc_mu = 0.f, acc_k = 0.f, acc_w = 0.f;
    uint32_t n = 0;
    // the Philox block of moves n and n + 1 (words 0-1, then 2-3): computed at
    // even n only; the lanes of a warp start their particles together and
    // step in lock-step, so the branch is uniform across active lanes
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    while (n < a.max_steps) {
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
        const bool odd = (n & 1u) != 0u;
        if (!odd) r = philox4x32_10(make_uint4(cell, j, n >> 1, 0u), a.keys);
        const float xix = uniform_pm1(odd ? r.z : r.x);
        const float xiy = uniform_pm1(odd ? r.w : r.y);
        const float rx = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dx), __fmul_rn(a.oneP, gx)), __fmul_rn(a.R, xix));
        const float ry = __fadd_rn(__fadd_rn(__fmul_rn(a.P, dy), __fmul_rn(a.oneP, gy)), __fmul_rn(a.R, xiy));
        const float r2 = __fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry));
        if (r2 == 0.0f) break;
        const float rinv = rcp_sqrt_rn(r2);
        dx = __fmul_rn(rx, rinv);
        dy = __fmul_rn(ry, rinv);
        const float u1 = __fadd_rn(u, __fmul_rn(a.s, dx));
        const float v1 = __fadd_rn(v, __fmul_rn(a.s, dy));
        if (!(u1 >= 0.0f && u1 <= a.Wm1 && v1 >= 0.0f && v1 <= a.Hm1)) break;
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
        if (S1 < SOFT_S_MIN) break;
    }
    steps += n;
    if (GRAD) {
        const float G = __ldg(a.grad + last);
        acc_mu += G * smu;
        acc_k += G * sk;
        acc_w += G * S;
        sum_mu += (double)w * (double)acc_mu * (double)a.mu;  // d/dlog(mu) = mu d/dmu
        sum_k += (double)w * (double)acc_k * (double)a.k;
        atomicAdd(a.grad_w + ci, (double)acc_w);
    } else {
        const long long Wq = __float2ll_rn(w * FIX_SCALE);
        if (Wq != Q) atomicAdd(a.deposit + last, (unsigned long long)(Wq - Q));
    }
}

template <bool GRAD, bool TEX>
__global__ void __launch_bounds__(128) k_soft(const __grid_constant__ SoftArgs a)
{
    const uint64_t total = (uint64_t)soft_count(a) * a.N;
    double sum_mu = 0.0, sum_k = 0.0;
    unsigned long long steps = 0ull, traj = 0ull, bad = 0ull;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t ci = (uint32_t)(t / a.N), j = (uint32_t)(t - (uint64_t)ci * a.N);
        bool rejected = false;
        soft_particle<GRAD, TEX>(a, ci, j, sum_mu, sum_k, steps, rejected);
        bad += rejected ? 1ull : 0ull;
        traj += rejected ? 0ull : 1ull;
    }
    // FP64 reductions over the warp, then one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum_mu += __shfl_xor_sync(0xffffffffu, sum_mu, o);
        sum_k += __shfl_xor_sync(0xffffffffu, sum_k, o);
        steps += __shfl_xor_sync(0xffffffffu, steps, o);
        traj += __shfl_xor_sync(0xffffffffu, traj, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (GRAD) {
            atomicAdd(a.grad_theta + 0, sum_mu);
            atomicAdd(a.grad_theta + 1, sum_k);
        }
        if (a.stats) {
            if (steps) atomicAdd(a.stats + 0, steps);
            if (traj) atomicAdd(a.stats + 1, traj);
            if (bad) atomicAdd(a.stats + 5, bad);
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
    unsigned long long pad[2];
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
    a.starts = reinterpret_cast<CellStart*>(static_cast<char*>(d_ws) + SOFT_STARTS_OFF);
    a.grad_w = reinterpret_cast<double*>(static_cast<char*>(d_ws) + SOFT_STARTS_OFF +
                                         (size_t)n_cells_max * sizeof(CellStart));
    a.tex = dem_texture(d_h, g, s);
    return AWO_OK;
}

static unsigned soft_blocks(const SoftArgs& a)
{
    const int64_t total = (int64_t)a.n_cells_max * a.N;
    return stream_blocks(total, 128, 16);
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
            k_soft<false, true><<<soft_blocks(a), 128, 0, s>>>(a);
        else
            k_soft<false, false><<<soft_blocks(a), 128, 0, s>>>(a);
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
            k_soft<true, true><<<soft_blocks(a), 128, 0, s>>>(a);
        else
            k_soft<true, false><<<soft_blocks(a), 128, 0, s>>>(a);
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
