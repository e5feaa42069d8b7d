// awo_probe.cu -- L2 scattered-load and scattered-reduction throughput probes,
// the self-tests of the particle kernels' correctly rounded normalisation,
// visited cell and division, and their Philox words for given counters.
//
// A persistent grid (SMs x 8 blocks of 256 threads, enough warps to cover L2
// latency) issues independent, hashed 4-byte accesses into a buffer sized by
// the caller (an L2-resident size gives the L2 ceiling).  The hash is a
// multiply-xorshift of (thread, round), so accesses spread over all L2
// slices with no locality between lanes.
#include <algorithm>

#include "awo_internal.cuh"
#include "awo_particle.cuh"
#include "awo_probe.h"

namespace awo {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

__device__ __forceinline__ uint32_t mix(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_gather(const uint32_t* __restrict__ buf, uint32_t mask,
                                                                uint32_t iters, uint32_t* __restrict__ sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    uint32_t s = mix(tid * 0x9E3779B9u + 1u);
    for (uint32_t r = 0; r < iters; ++r) {
        uint32_t a0 = mix(s + 4u * r) & mask;
        uint32_t a1 = mix(s + 4u * r + 1u) & mask;
        uint32_t a2 = mix(s + 4u * r + 2u) & mask;
        uint32_t a3 = mix(s + 4u * r + 3u) & mask;
        acc += __ldg(buf + a0) ^ __ldg(buf + a1) ^ __ldg(buf + a2) ^ __ldg(buf + a3);
    }
    sink[tid] = acc;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_red(uint32_t* __restrict__ buf, uint32_t mask, uint32_t iters)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s = mix(tid * 0x9E3779B9u + 7u);
    for (uint32_t r = 0; r < iters; ++r) {
        uint32_t a0 = mix(s + 2u * r) & mask;
        uint32_t a1 = mix(s + 2u * r + 1u) & mask;
        atomicAdd(buf + a0, 1u);
        atomicMax(buf + a1, r);
    }
}

// Every bit pattern b of [first, first + count) (but +-0): rcp_sqrt_rn(x)
// against __frcp_rn(__fsqrt_rn(x)), bit for bit; one atomic per warp.
__global__ void __launch_bounds__(256) k_selftest_rcp_sqrt(uint32_t first, unsigned long long count,
                                                           unsigned long long* mismatches)
{
    unsigned long long bad = 0ull;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t bits = first + (uint32_t)i;
        if ((bits & 0x7fffffffu) == 0u) continue;
        const float x = __uint_as_float(bits);
        bad += __float_as_uint(rcp_sqrt_rn(x)) != __float_as_uint(__frcp_rn(__fsqrt_rn(x))) ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

// Every FP32 position u in [first bits, first bits + count) that is >= 0:
// visit_axis(u) against floor(u) + [u - floor(u) >= 1/2] in exact arithmetic
// (the fraction u - floor(u) of a float below 2^23 is exact).
__global__ void __launch_bounds__(256) k_selftest_visit(uint32_t first, unsigned long long count,
                                                        unsigned long long* mismatches)
{
    unsigned long long bad = 0ull;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float u = __uint_as_float(first + (uint32_t)i);
        if (!(u >= 0.0f && u < 8388608.0f)) continue;
        const float fl = floorf(u);
        const int want = (int)fl + (__fsub_rn(u, fl) >= 0.5f ? 1 : 0);
        bad += visit_axis(u) != want ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

// Philox4x32-10 words of the counters c[0 .. n), by the particle kernels'
// device function with round keys K (a table from the host or the Weyl
// schedule in registers, as the kernels take them).
template <class K>
__global__ void __launch_bounds__(256) k_probe_philox(const uint4* __restrict__ c, int64_t n, const K key,
                                                      uint4* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(__ldg(c + i), key);
}

}  // namespace awo

using namespace awo;

extern "C" awo_status awo_probe_philox(const uint32_t* d_counters, int64_t n, uint64_t seed, int32_t weyl_keys,
                                       uint32_t* d_out, void* stream)
{
    if (!d_counters || !d_out || n < 0) return AWO_EINVAL;
    if ((((uintptr_t)d_counters) & 15u) != 0 || (((uintptr_t)d_out) & 15u) != 0) return AWO_EINVAL;
    if (n == 0) return AWO_OK;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    const uint4* c = reinterpret_cast<const uint4*>(d_counters);
    uint4* o = reinterpret_cast<uint4*>(d_out);
    cudaStream_t s = as_stream(stream);
    if (weyl_keys) {
        KeysWeyl key;
        key.k0 = k0;
        key.k1 = k1;
        k_probe_philox<KeysWeyl><<<blocks, 256, 0, s>>>(c, n, key, o);
    } else {
        // the round-key table as the single-request kernel's host code fills it
        KeysTable key;
        uint32_t a = k0, b = k1;
        for (int r = 0; r < 10; ++r) {
            key.k0[r] = a;
            key.k1[r] = b;
            a += 0x9E3779B9u;
            b += 0xBB67AE85u;
        }
        k_probe_philox<KeysTable><<<blocks, 256, 0, s>>>(c, n, key, o);
    }
    return launch_status();
}

extern "C" awo_status awo_selftest_rcp_sqrt(uint32_t first, uint64_t count, uint64_t* d_mismatches, void* stream)
{
    if (!d_mismatches || (((uintptr_t)d_mismatches) & 7u) != 0) return AWO_EINVAL;
    if (count > (1ull << 32) - first) return AWO_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(d_mismatches, 0, sizeof(uint64_t), s) != cudaSuccess) return AWO_ECUDA;
    if (count == 0) return AWO_OK;
    k_selftest_rcp_sqrt<<<sm_count() * 8, 256, 0, s>>>(first, (unsigned long long)count,
                                                       reinterpret_cast<unsigned long long*>(d_mismatches));
    return launch_status();
}

// Every divisor b of the list (positive, finite) and every FP32 a with bits
// in [bits(b) - span, bits(b)] (at least +0): div_rn_by_rcp of a (unsigned and
// signed forms) and of -a (signed form) against the intrinsic.  The
// (divisor, offset) pairs are spread over the grid, so a long list of
// divisors with short spans runs as fast as a short list with long ones.
__global__ void __launch_bounds__(256) k_selftest_div(const float* __restrict__ divisors, uint32_t n_div,
                                                      uint32_t span, unsigned long long* mismatches)
{
    unsigned long long bad = 0ull;
    const unsigned long long per = (unsigned long long)span + 1ull, total = per * n_div;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t d = (uint32_t)(i / per), off = (uint32_t)(i - (unsigned long long)d * per);
        const float b = __ldg(divisors + d);
        if (!(b > 0.0f && b <= 3.4028234663852886e38f)) continue;
        const uint32_t bb = __float_as_uint(b);
        if (off > bb) continue;
        const float a = __uint_as_float(bb - off), y = __frcp_rn(b);
        const uint32_t want = __float_as_uint(__fdiv_rn(a, b)), want_neg = __float_as_uint(__fdiv_rn(-a, b));
        bad += __float_as_uint(div_rn_by_rcp<false>(a, b, y)) != want ? 1ull : 0ull;
        bad += __float_as_uint(div_rn_by_rcp<true>(a, b, y)) != want ? 1ull : 0ull;
        bad += __float_as_uint(div_rn_by_rcp<true>(-a, b, y)) != want_neg ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

extern "C" awo_status awo_selftest_div_rn(const float* d_divisors, uint32_t n_divisors, uint32_t span,
                                          uint64_t* d_mismatches, void* stream)
{
    if (!d_divisors || (((uintptr_t)d_divisors) & 3u) != 0 || n_divisors == 0) return AWO_EINVAL;
    if (!d_mismatches || (((uintptr_t)d_mismatches) & 7u) != 0) return AWO_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(d_mismatches, 0, sizeof(uint64_t), s) != cudaSuccess) return AWO_ECUDA;
    k_selftest_div<<<sm_count() * 8, 256, 0, s>>>(d_divisors, n_divisors, span,
                                                  reinterpret_cast<unsigned long long*>(d_mismatches));
    return launch_status();
}

extern "C" uint64_t awo_probe_threads(void)
{
    return (uint64_t)sm_count() * PROBE_BLOCKS_PER_SM * PROBE_THREADS;
}

static bool pow2_ok(uint32_t n) { return n >= 1024u && n <= (1u << 30) && (n & (n - 1u)) == 0u; }

extern "C" awo_status awo_probe_l2_gather(const uint32_t* d_buf, uint32_t n_words, uint32_t iters, uint32_t* d_sink,
                                          void* stream)
{
    if (!d_buf || !d_sink || !pow2_ok(n_words) || iters == 0) return AWO_EINVAL;
    k_probe_gather<<<sm_count() * PROBE_BLOCKS_PER_SM, PROBE_THREADS, 0, as_stream(stream)>>>(d_buf, n_words - 1u,
                                                                                              iters, d_sink);
    return launch_status();
}

extern "C" awo_status awo_probe_l2_red(uint32_t* d_buf, uint32_t n_words, uint32_t iters, void* stream)
{
    if (!d_buf || !pow2_ok(n_words) || iters == 0) return AWO_EINVAL;
    k_probe_red<<<sm_count() * PROBE_BLOCKS_PER_SM, PROBE_THREADS, 0, as_stream(stream)>>>(d_buf, n_words - 1u,
                                                                                           iters);
    return launch_status();
}

extern "C" awo_status awo_selftest_visit_cell(uint32_t first, uint64_t count, uint64_t* d_mismatches, void* stream)
{
    if (!d_mismatches || (((uintptr_t)d_mismatches) & 7u) != 0) return AWO_EINVAL;
    if (count > (1ull << 32) - first) return AWO_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(d_mismatches, 0, sizeof(uint64_t), s) != cudaSuccess) return AWO_ECUDA;
    if (count == 0) return AWO_OK;
    k_selftest_visit<<<sm_count() * 8, 256, 0, s>>>(first, (unsigned long long)count,
                                                    reinterpret_cast<unsigned long long*>(d_mismatches));
    return launch_status();
}
