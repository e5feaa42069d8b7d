// awo_overlay.cu -- velocity indicator and overlay mipmap (Sec. 3, Fig. 4).
//
// Both are streaming passes.  The mipmap is built level by level: each thread
// reduces 2x2 blocks of the level above (two output texels from 16-byte rows
// when the level allows it; counts summed in 64 bits and saturated,
// velocities by max), so every level reads its parent once.
#include "awo_internal.cuh"

namespace awo {

// vel = sqrt((2 g) maxe); float4 loads and stores when both rasters are
// 16-byte aligned, then a scalar tail.  A thread issues the loads of
// STREAM_UNROLL float4 (each coalesced across the grid) before their stores,
// so that enough bytes are in flight per SM to keep HBM busy.
constexpr int STREAM_UNROLL = 4;

__global__ void k_finalize(const float* __restrict__ maxe, int64_t n, float g2, float* __restrict__ vel, bool vec4)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n4 = vec4 ? n / 4 : 0;
    for (int64_t q = tid; q < n4; q += STREAM_UNROLL * stride) {
        float4 m[STREAM_UNROLL];
#pragma unroll
        for (int u = 0; u < STREAM_UNROLL; ++u) {
            const int64_t k = q + u * stride;
            m[u] = k < n4 ? __ldg(reinterpret_cast<const float4*>(maxe) + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < STREAM_UNROLL; ++u) {
            const int64_t k = q + u * stride;
            if (k < n4)
                reinterpret_cast<float4*>(vel)[k] =
                    make_float4(__fsqrt_rn(__fmul_rn(g2, m[u].x)), __fsqrt_rn(__fmul_rn(g2, m[u].y)),
                                __fsqrt_rn(__fmul_rn(g2, m[u].z)), __fsqrt_rn(__fmul_rn(g2, m[u].w)));
        }
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += stride) vel[i] = __fsqrt_rn(__fmul_rn(g2, maxe[i]));
}

__device__ __forceinline__ uint32_t sat_sum4(uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    const unsigned long long s = (unsigned long long)a + b + c + d;
    return s > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)s;
}

// One mipmap level.  Fast form (w % 4 == 0, h even, 16-byte-aligned inputs,
// 8-byte-aligned outputs): a thread makes two output texels from a uint4 /
// float4 of each of the two parent rows.  General form: one output texel,
// missing children ignored.  Items are indexed in 32 bits (W * H < 2^31).
__global__ void k_lod_level(const uint32_t* __restrict__ c_in, const float* __restrict__ v_in, int w, int h,
                            uint32_t* __restrict__ c_out, float* __restrict__ v_out, int w2, int h2, bool vec)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    if (vec) {
        const uint32_t pairs = (uint32_t)(w2 / 2), items = pairs * (uint32_t)h2;
        for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += stride) {
            const uint32_t y = it / pairs, xp = it - y * pairs;
            const int64_t r0 = (int64_t)(2 * y) * w + 4 * xp, r1 = r0 + w;
            const uint4 a = __ldg(reinterpret_cast<const uint4*>(c_in + r0));
            const uint4 b = __ldg(reinterpret_cast<const uint4*>(c_in + r1));
            const float4 p = __ldg(reinterpret_cast<const float4*>(v_in + r0));
            const float4 q = __ldg(reinterpret_cast<const float4*>(v_in + r1));
            const int64_t o = (int64_t)y * w2 + 2 * xp;
            reinterpret_cast<uint2*>(c_out + o)[0] = make_uint2(sat_sum4(a.x, a.y, b.x, b.y), sat_sum4(a.z, a.w, b.z, b.w));
            reinterpret_cast<float2*>(v_out + o)[0] =
                make_float2(fmaxf(fmaxf(p.x, p.y), fmaxf(q.x, q.y)), fmaxf(fmaxf(p.z, p.w), fmaxf(q.z, q.w)));
        }
        return;
    }
    const uint32_t n = (uint32_t)w2 * (uint32_t)h2;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int y = (int)(i / (uint32_t)w2);
        int x = (int)(i - (uint32_t)y * (uint32_t)w2);
        int sx = 2 * x, sy = 2 * y;
        bool hx = sx + 1 < w, hy = sy + 1 < h;
        const int64_t r0 = (int64_t)sy * w, r1 = (int64_t)(sy + 1) * w;
        unsigned long long sum = c_in[r0 + sx];
        float m = v_in[r0 + sx];
        if (hx) {
            sum += c_in[r0 + sx + 1];
            m = fmaxf(m, v_in[r0 + sx + 1]);
        }
        if (hy) {
            sum += c_in[r1 + sx];
            m = fmaxf(m, v_in[r1 + sx]);
            if (hx) {
                sum += c_in[r1 + sx + 1];
                m = fmaxf(m, v_in[r1 + sx + 1]);
            }
        }
        c_out[i] = sum > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)sum;
        v_out[i] = m;
    }
}

}  // namespace awo

using namespace awo;

extern "C" awo_status awo_finalize(const float* d_maxe, awo_grid g, float gravity, float* d_vel, void* stream)
{
    if (!d_maxe || !d_vel || !grid_ok(g) || !(gravity > 0.0f) || !(gravity < 1.0e38f)) return AWO_EINVAL;
    const int64_t n = cells_of(g);
    const bool vec4 = ((((uintptr_t)d_maxe) | ((uintptr_t)d_vel)) & 15u) == 0;
    k_finalize<<<stream_blocks(vec4 ? n / 4 + 1 : n, 256), 256, 0, as_stream(stream)>>>(d_maxe, n, 2.0f * gravity,
                                                                                        d_vel, vec4);
    return launch_status();
}

extern "C" awo_status awo_overlay_lod(const uint32_t* d_count, const float* d_vel, awo_grid g, int32_t levels,
                                      uint32_t* const* d_count_lv, float* const* d_vel_lv, void* stream)
{
    if (!d_count || !d_vel || !grid_ok(g) || levels < 1 || levels > 16) return AWO_EINVAL;
    if (levels > 1 && (!d_count_lv || !d_vel_lv)) return AWO_EINVAL;
    for (int l = 0; l + 1 < levels; ++l)
        if (!d_count_lv[l] || !d_vel_lv[l]) return AWO_EINVAL;
    cudaStream_t s = as_stream(stream);
    const uint32_t* ci = d_count;
    const float* vi = d_vel;
    int w = g.width, h = g.height;
    for (int l = 1; l < levels; ++l) {
        int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
        const bool vec = w % 4 == 0 && h % 2 == 0 && ((((uintptr_t)ci) | ((uintptr_t)vi)) & 15u) == 0 &&
                         ((((uintptr_t)d_count_lv[l - 1]) | ((uintptr_t)d_vel_lv[l - 1])) & 7u) == 0;
        const int64_t items = vec ? (int64_t)(w2 / 2) * h2 : (int64_t)w2 * h2;
        k_lod_level<<<stream_blocks(items, 256), 256, 0, s>>>(ci, vi, w, h, d_count_lv[l - 1], d_vel_lv[l - 1], w2,
                                                              h2, vec);
        awo_status st = launch_status();
        if (st != AWO_OK) return st;
        ci = d_count_lv[l - 1];
        vi = d_vel_lv[l - 1];
        w = w2;
        h = h2;
    }
    return AWO_OK;
}
