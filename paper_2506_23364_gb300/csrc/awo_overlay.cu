// awo_overlay.cu -- velocity indicator and overlay mipmap (Sec. 3, Fig. 4).
//
// Both are streaming passes.  Levels 1-6 of the mipmap come from one kernel:
// a block reduces its 64 x 64 tile of level 0 to level 1 and then, in shared
// memory, to each further level (counts summed in 64 bits and saturated,
// velocities by max), so level 0 is read once and every level written once;
// deeper levels are built one launch per level from their parent.  The
// workflow's call also makes the velocity from the maximum energy inside the
// same pass (awo_finalize_lod).
#include <string.h>

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

// Levels 1 .. 1 + LOD_FUSED - 1 of the mipmap in one pass over level 0.  A
// block owns a 32 x 32 tile of level 1 (a 64 x 64 tile of level 0) and all
// its descendants: 16 x 16 of level 2, ... 1 x 1 of level 6, since the tiles
// of every level nest.  Level 1 is reduced from level 0 in global memory,
// each further level from the previous one in shared memory; every texel is
// the saturating count sum and the velocity maximum of its existing children
// (children past a level's edge are ignored), as in k_lod_level.  One read of
// level 0 and one write of each level, instead of a read and a write per
// level with a launch each.  FROM_MAXE: level 0's velocity is not read but
// made from the maximum energy as it is needed, vel = sqrt((2 g) maxe), and
// written (awo_finalize fused in): each level-0 cell is the child of exactly
// one level-1 texel, so each is computed and written once.
constexpr int LOD_TILE = 32;   // level-1 tile side
constexpr int LOD_FUSED = 6;   // levels a block can finish: 32, 16, 8, 4, 2, 1

struct LodArgs {
    const uint32_t* c0;
    const float* v0;  // level-0 velocity, or the maximum energy when FROM_MAXE
    float* vel0;      // FROM_MAXE: level-0 velocity out (may alias v0)
    float g2;         // FROM_MAXE: 2 g
    int w[LOD_FUSED + 1], h[LOD_FUSED + 1];  // level sizes 0 .. LOD_FUSED
    uint32_t* c[LOD_FUSED];                  // outputs of levels 1 .. LOD_FUSED
    float* v[LOD_FUSED];
    int n_out;                               // levels written, 1 .. LOD_FUSED
    bool vec2;                               // level-0 child pairs as uint2 / float2
};

template <bool FROM_MAXE>
__device__ __forceinline__ float lod_vel0(const LodArgs& a, uint32_t i)
{
    const float x = __ldg(a.v0 + i);
    if (!FROM_MAXE) return x;
    const float v = __fsqrt_rn(__fmul_rn(a.g2, x));
    a.vel0[i] = v;
    return v;
}

template <bool FROM_MAXE>
__device__ __forceinline__ float2 lod_vel0_pair(const LodArgs& a, uint32_t i)
{
    const float2 x = __ldg(reinterpret_cast<const float2*>(a.v0 + i));
    if (!FROM_MAXE) return x;
    const float2 v = make_float2(__fsqrt_rn(__fmul_rn(a.g2, x.x)), __fsqrt_rn(__fmul_rn(a.g2, x.y)));
    *reinterpret_cast<float2*>(a.vel0 + i) = v;
    return v;
}

template <bool FROM_MAXE>
__global__ void __launch_bounds__(256) k_lod_fused(const __grid_constant__ LodArgs a)
{
    __shared__ uint32_t sc[2][LOD_TILE][LOD_TILE + 1];
    __shared__ float sv[2][LOD_TILE][LOD_TILE + 1];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int bx = blockIdx.x, by = blockIdx.y;
    // level 1 from level 0: four texels per thread, rows ty, ty + 8, ...
    {
        const int w0 = a.w[0], h0 = a.h[0], w1 = a.w[1], h1 = a.h[1];
        const int X = bx * LOD_TILE + tx;
#pragma unroll
        for (int k = 0; k < LOD_TILE / 8; ++k) {
            const int y = ty + 8 * k, Y = by * LOD_TILE + y;
            if (X < w1 && Y < h1) {
                const int sx = 2 * X, sy = 2 * Y;
                const bool hx = sx + 1 < w0, hy = sy + 1 < h0;
                const uint32_t r0 = (uint32_t)sy * (uint32_t)w0 + (uint32_t)sx, r1 = r0 + (uint32_t)w0;
                unsigned long long sum;
                float m;
                if (a.vec2) {  // w0 even: both columns exist and the pair is 8-byte aligned
                    const uint2 c_0 = __ldg(reinterpret_cast<const uint2*>(a.c0 + r0));
                    const float2 v_0 = lod_vel0_pair<FROM_MAXE>(a, r0);
                    sum = (unsigned long long)c_0.x + c_0.y;
                    m = fmaxf(v_0.x, v_0.y);
                    if (hy) {
                        const uint2 c_1 = __ldg(reinterpret_cast<const uint2*>(a.c0 + r1));
                        const float2 v_1 = lod_vel0_pair<FROM_MAXE>(a, r1);
                        sum += (unsigned long long)c_1.x + c_1.y;
                        m = fmaxf(m, fmaxf(v_1.x, v_1.y));
                    }
                } else {
                    sum = __ldg(a.c0 + r0);
                    m = lod_vel0<FROM_MAXE>(a, r0);
                    if (hx) {
                        sum += __ldg(a.c0 + r0 + 1);
                        m = fmaxf(m, lod_vel0<FROM_MAXE>(a, r0 + 1));
                    }
                    if (hy) {
                        sum += __ldg(a.c0 + r1);
                        m = fmaxf(m, lod_vel0<FROM_MAXE>(a, r1));
                        if (hx) {
                            sum += __ldg(a.c0 + r1 + 1);
                            m = fmaxf(m, lod_vel0<FROM_MAXE>(a, r1 + 1));
                        }
                    }
                }
                const uint32_t c = sum > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)sum;
                const uint32_t o = (uint32_t)Y * (uint32_t)w1 + (uint32_t)X;
                a.c[0][o] = c;
                a.v[0][o] = m;
                sc[0][y][tx] = c;
                sv[0][y][tx] = m;
            }
        }
    }
    // levels 2 .. n_out from the previous level in shared memory
    int t = LOD_TILE, src = 0;
    for (int l = 2; l <= a.n_out; ++l) {
        __syncthreads();
        const int t2 = t >> 1;
        if (tid < t2 * t2) {
            const int x = tid % t2, y = tid / t2;
            const int X = bx * t2 + x, Y = by * t2 + y;
            if (X < a.w[l] && Y < a.h[l]) {
                const int wp = a.w[l - 1], hp = a.h[l - 1];
                const bool hx = 2 * X + 1 < wp, hy = 2 * Y + 1 < hp;
                unsigned long long sum = sc[src][2 * y][2 * x];
                float m = sv[src][2 * y][2 * x];
                if (hx) {
                    sum += sc[src][2 * y][2 * x + 1];
                    m = fmaxf(m, sv[src][2 * y][2 * x + 1]);
                }
                if (hy) {
                    sum += sc[src][2 * y + 1][2 * x];
                    m = fmaxf(m, sv[src][2 * y + 1][2 * x]);
                    if (hx) {
                        sum += sc[src][2 * y + 1][2 * x + 1];
                        m = fmaxf(m, sv[src][2 * y + 1][2 * x + 1]);
                    }
                }
                const uint32_t c = sum > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)sum;
                const uint32_t o = (uint32_t)Y * (uint32_t)a.w[l] + (uint32_t)X;
                a.c[l - 1][o] = c;
                a.v[l - 1][o] = m;
                sc[src ^ 1][y][x] = c;
                sv[src ^ 1][y][x] = m;
            }
        }
        src ^= 1;
        t = t2;
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

// Levels 1 .. levels-1 from level 0 = (d_count, v0): one fused launch for
// levels 1 .. LOD_FUSED, then one launch per further level.  from_maxe: v0
// is the maximum energy and level 0's velocity is written to d_vel (g2 = 2 g).
static awo_status lod_levels(const uint32_t* d_count, const float* v0, bool from_maxe, float g2, float* d_vel,
                             awo_grid g, int32_t levels, uint32_t* const* d_count_lv, float* const* d_vel_lv,
                             cudaStream_t s)
{
    LodArgs a;
    memset(&a, 0, sizeof(a));
    a.c0 = d_count;
    a.v0 = v0;
    a.vel0 = d_vel;
    a.g2 = g2;
    a.n_out = levels - 1 < LOD_FUSED ? levels - 1 : LOD_FUSED;
    a.w[0] = g.width;
    a.h[0] = g.height;
    for (int k = 1; k <= a.n_out; ++k) {
        a.w[k] = (a.w[k - 1] + 1) / 2;
        a.h[k] = (a.h[k - 1] + 1) / 2;
        a.c[k - 1] = d_count_lv[k - 1];
        a.v[k - 1] = d_vel_lv[k - 1];
    }
    a.vec2 = g.width % 2 == 0 &&
             ((((uintptr_t)d_count) | ((uintptr_t)v0) | (from_maxe ? (uintptr_t)d_vel : (uintptr_t)0)) & 7u) == 0;
    const dim3 grid((unsigned)((a.w[1] + LOD_TILE - 1) / LOD_TILE), (unsigned)((a.h[1] + LOD_TILE - 1) / LOD_TILE));
    if (from_maxe)
        k_lod_fused<true><<<grid, 256, 0, s>>>(a);
    else
        k_lod_fused<false><<<grid, 256, 0, s>>>(a);
    awo_status st = launch_status();
    if (st != AWO_OK) return st;
    const uint32_t* ci = d_count_lv[a.n_out - 1];
    const float* vi = d_vel_lv[a.n_out - 1];
    int w = a.w[a.n_out], h = a.h[a.n_out];
    for (int l = 1 + a.n_out; l < levels; ++l) {
        int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
        const bool vec = w % 4 == 0 && h % 2 == 0 && ((((uintptr_t)ci) | ((uintptr_t)vi)) & 15u) == 0 &&
                         ((((uintptr_t)d_count_lv[l - 1]) | ((uintptr_t)d_vel_lv[l - 1])) & 7u) == 0;
        const int64_t items = vec ? (int64_t)(w2 / 2) * h2 : (int64_t)w2 * h2;
        k_lod_level<<<stream_blocks(items, 256), 256, 0, s>>>(ci, vi, w, h, d_count_lv[l - 1], d_vel_lv[l - 1], w2,
                                                              h2, vec);
        st = launch_status();
        if (st != AWO_OK) return st;
        ci = d_count_lv[l - 1];
        vi = d_vel_lv[l - 1];
        w = w2;
        h = h2;
    }
    return AWO_OK;
}

extern "C" awo_status awo_overlay_lod(const uint32_t* d_count, const float* d_vel, awo_grid g, int32_t levels,
                                      uint32_t* const* d_count_lv, float* const* d_vel_lv, void* stream)
{
    if (!d_count || !d_vel || !grid_ok(g) || levels < 1 || levels > 16) return AWO_EINVAL;
    if (levels > 1 && (!d_count_lv || !d_vel_lv)) return AWO_EINVAL;
    for (int l = 0; l + 1 < levels; ++l)
        if (!d_count_lv[l] || !d_vel_lv[l]) return AWO_EINVAL;
    if (levels == 1) return AWO_OK;
    return lod_levels(d_count, d_vel, false, 0.0f, nullptr, g, levels, d_count_lv, d_vel_lv, as_stream(stream));
}

extern "C" awo_status awo_finalize_lod(const float* d_maxe, const uint32_t* d_count, awo_grid g, float gravity,
                                       int32_t levels, float* d_vel, uint32_t* const* d_count_lv,
                                       float* const* d_vel_lv, void* stream)
{
    if (!d_maxe || !d_count || !d_vel || !grid_ok(g) || levels < 1 || levels > 16) return AWO_EINVAL;
    if (!(gravity > 0.0f) || !(gravity < 1.0e38f)) return AWO_EINVAL;
    if (levels > 1 && (!d_count_lv || !d_vel_lv)) return AWO_EINVAL;
    for (int l = 0; l + 1 < levels; ++l)
        if (!d_count_lv[l] || !d_vel_lv[l]) return AWO_EINVAL;
    if (levels == 1) return awo_finalize(d_maxe, g, gravity, d_vel, stream);
    return lod_levels(d_count, d_maxe, true, 2.0f * gravity, d_vel, g, levels, d_count_lv, d_vel_lv,
                      as_stream(stream));
}
