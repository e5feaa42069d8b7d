// awo_compose.cu -- overlay colouring / alpha blending and the snow-cover mask.
//
// Both are per-texel streaming passes (HBM-bound) over rasters the rest of the
// library produces: the velocity and count overlay (Sec. 3 compose pass,
// Fig. 4 colour scale) and the normals (Sec. 5.1 snow cover).  FP32 with
// explicit round-to-nearest intrinsics; 8-bit outputs rounded half to even.
#include <math.h>

#include "awo_internal.cuh"

namespace awo {

// Round half to even into [0, 255]: non-positive and NaN give 0, values
// above 255 give 255 (the saturating conversion of fmaxf(x, 0), capped).
__device__ __forceinline__ uint32_t to_u8(float x) { return min(__float2uint_rn(fmaxf(x, 0.0f)), 255u); }

// The colour ramp in shared memory, per segment k: its start value, width
// v[k+1] - v[k], start colour and colour step c[k+1] - c[k] (the same
// roundings the per-texel formula makes; the colour step of 8-bit colours is
// exact) -- two 16-byte loads per texel -- and RN(1 / width) for the division.
struct RampSmem {
    float4 seg[15][2];  // {v0, dv, c0.r, c0.g}, {c0.b, dc.r, dc.g, dc.b}
    float rcp[15];
};

// One texel: colour of value x, opacity from its count, over base texel b
// (packed RGBA, little-endian bytes) when HAS_BASE.  The segment is the
// number of interior stops at or below x (stops strictly increase): NS - 2
// compares against the stop values in the kernel's parameter bank.
template <int NS, bool HAS_BASE>
__device__ __forceinline__ uint32_t compose_one(const RampSmem& r, const awo_colormap& cm, float x, uint32_t count,
                                                uint32_t b)
{
    if (!(x > cm.value[0])) x = cm.value[0];
    if (x > cm.value[NS - 1]) x = cm.value[NS - 1];
    int k = 0;
#pragma unroll
    for (int j = 1; j < NS - 1; ++j) k += x >= cm.value[j] ? 1 : 0;
    const float4 s0 = r.seg[k][0], s1 = r.seg[k][1];
    const float t = div_rn_by_rcp<false>(__fsub_rn(x, s0.x), s0.y, r.rcp[k]);  // = __fdiv_rn(x - v0, dv)
    const float a = count >= cm.count_min ? cm.alpha : 0.0f;
    const float col[3] = {__fadd_rn(s0.z, __fmul_rn(t, s1.y)), __fadd_rn(s0.w, __fmul_rn(t, s1.z)),
                          __fadd_rn(s1.x, __fmul_rn(t, s1.w))};
    const float na = __fsub_rn(1.0f, a);
    uint32_t o = 0u;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float bc = (float)((b >> (8 * c)) & 0xffu);
        const uint32_t ch = HAS_BASE ? to_u8(__fadd_rn(__fmul_rn(a, col[c]), __fmul_rn(na, bc))) : to_u8(col[c]);
        o |= ch << (8 * c);
    }
    const uint32_t oa = HAS_BASE ? (b >> 24) : to_u8(__fmul_rn(255.0f, a));
    return o | (oa << 24);
}

// Four texels per thread (float4 / uint4 loads, uint4 store) when every
// buffer is 16-byte aligned, then a scalar tail.  One instance per stop count
// and base / no base: the stop compares unroll, and no texel selects between
// the two blends.
template <int NS, bool HAS_BASE>
__global__ void k_compose(const float* __restrict__ value, const uint32_t* __restrict__ count, int64_t n,
                          const __grid_constant__ awo_colormap cm, const uint8_t* __restrict__ base,
                          uint8_t* __restrict__ out, bool vec4)
{
    __shared__ RampSmem ramp;
    for (int i = threadIdx.x; i < NS - 1; i += blockDim.x) {
        const float c0r = (float)cm.rgb[i][0], c0g = (float)cm.rgb[i][1], c0b = (float)cm.rgb[i][2];
        const float dv = __fsub_rn(cm.value[i + 1], cm.value[i]);
        ramp.seg[i][0] = make_float4(cm.value[i], dv, c0r, c0g);
        ramp.seg[i][1] = make_float4(c0b, __fsub_rn((float)cm.rgb[i + 1][0], c0r),
                                     __fsub_rn((float)cm.rgb[i + 1][1], c0g), __fsub_rn((float)cm.rgb[i + 1][2], c0b));
        ramp.rcp[i] = __frcp_rn(dv);
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t* base32 = reinterpret_cast<const uint32_t*>(base);
    uint32_t* out32 = reinterpret_cast<uint32_t*>(out);
    const int64_t n4 = vec4 ? n / 4 : 0;
    for (int64_t q = tid; q < n4; q += stride) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(value) + q);
        const uint4 c = __ldg(reinterpret_cast<const uint4*>(count) + q);
        const uint4 b = HAS_BASE ? __ldg(reinterpret_cast<const uint4*>(base32) + q) : make_uint4(0u, 0u, 0u, 0u);
        reinterpret_cast<uint4*>(out32)[q] =
            make_uint4(compose_one<NS, HAS_BASE>(ramp, cm, v.x, c.x, b.x),
                       compose_one<NS, HAS_BASE>(ramp, cm, v.y, c.y, b.y),
                       compose_one<NS, HAS_BASE>(ramp, cm, v.z, c.z, b.z),
                       compose_one<NS, HAS_BASE>(ramp, cm, v.w, c.w, b.w));
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += stride)
        out32[i] = compose_one<NS, HAS_BASE>(ramp, cm, value[i], count[i], HAS_BASE ? base32[i] : 0u);
}

template <int NS>
static void launch_compose(const float* v, const uint32_t* c, int64_t n, const awo_colormap& cm, const uint8_t* b,
                           uint8_t* o, bool vec4, cudaStream_t s)
{
    const unsigned blocks = stream_blocks(vec4 ? n / 4 + 1 : n, 256);
    if (b)
        k_compose<NS, true><<<blocks, 256, 0, s>>>(v, c, n, cm, b, o, vec4);
    else
        k_compose<NS, false><<<blocks, 256, 0, s>>>(v, c, n, cm, b, o, vec4);
}

__device__ __forceinline__ float smooth_step(float e0, float e1, float x)
{
    if (e1 == e0) return x >= e0 ? 1.0f : 0.0f;
    float t = __fdiv_rn(__fsub_rn(x, e0), __fsub_rn(e1, e0));
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    return __fmul_rn(__fmul_rn(t, t), __fsub_rn(3.0f, __fmul_rn(2.0f, t)));
}

__device__ __forceinline__ uint32_t snow_rgba(float a) { return 0x00ffffffu | (to_u8(__fmul_rn(255.0f, a)) << 24); }

// Four texels per thread when every buffer is 16-byte aligned, then a scalar tail.
__global__ void k_snow(const float* __restrict__ h, const float* __restrict__ nz, int64_t n, float a0, float a1,
                       float c0, float c1, float* __restrict__ alpha, uint8_t* __restrict__ rgba, bool vec4)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t* rgba32 = reinterpret_cast<uint32_t*>(rgba);
    const int64_t n4 = vec4 ? n / 4 : 0;
    for (int64_t q = tid; q < n4; q += stride) {
        const float4 hv = __ldg(reinterpret_cast<const float4*>(h) + q);
        const float4 zv = __ldg(reinterpret_cast<const float4*>(nz) + q);
        const float4 a = make_float4(__fmul_rn(smooth_step(a0, a1, hv.x), smooth_step(c0, c1, zv.x)),
                                     __fmul_rn(smooth_step(a0, a1, hv.y), smooth_step(c0, c1, zv.y)),
                                     __fmul_rn(smooth_step(a0, a1, hv.z), smooth_step(c0, c1, zv.z)),
                                     __fmul_rn(smooth_step(a0, a1, hv.w), smooth_step(c0, c1, zv.w)));
        if (alpha) reinterpret_cast<float4*>(alpha)[q] = a;
        if (rgba)
            reinterpret_cast<uint4*>(rgba32)[q] = make_uint4(snow_rgba(a.x), snow_rgba(a.y), snow_rgba(a.z),
                                                             snow_rgba(a.w));
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += stride) {
        const float a = __fmul_rn(smooth_step(a0, a1, h[i]), smooth_step(c0, c1, nz[i]));
        if (alpha) alpha[i] = a;
        if (rgba) rgba32[i] = snow_rgba(a);
    }
}

}  // namespace awo

using namespace awo;

static_assert(sizeof(awo_colormap) == 128, "awo_colormap layout (C ABI)");

extern "C" awo_status awo_compose(const float* d_value, const uint32_t* d_count, awo_grid g, const awo_colormap* cm,
                                  const uint8_t* d_base_rgba, uint8_t* d_out_rgba, void* stream)
{
    if (!d_value || !d_count || !cm || !d_out_rgba || !grid_ok(g)) return AWO_EINVAL;
    if (cm->n_stops < 2 || cm->n_stops > 16 || !(cm->alpha >= 0.0f && cm->alpha <= 1.0f)) return AWO_EINVAL;
    for (int k = 0; k + 1 < cm->n_stops; ++k)
        if (!(cm->value[k] < cm->value[k + 1])) return AWO_EINVAL;
    if ((((uintptr_t)d_out_rgba) & 3u) != 0 || (((uintptr_t)d_base_rgba) & 3u) != 0) return AWO_EINVAL;
    const int64_t n = cells_of(g);
    const bool vec4 = ((((uintptr_t)d_value) | ((uintptr_t)d_count) | ((uintptr_t)d_base_rgba) |
                        ((uintptr_t)d_out_rgba)) & 15u) == 0;
    const cudaStream_t s = as_stream(stream);
    switch (cm->n_stops) {
#define AWO_COMPOSE_NS(K)                                                                              \
    case K:                                                                                            \
        launch_compose<K>(d_value, d_count, n, *cm, d_base_rgba, d_out_rgba, vec4, s);                 \
        break;
        AWO_COMPOSE_NS(2) AWO_COMPOSE_NS(3) AWO_COMPOSE_NS(4) AWO_COMPOSE_NS(5) AWO_COMPOSE_NS(6)
        AWO_COMPOSE_NS(7) AWO_COMPOSE_NS(8) AWO_COMPOSE_NS(9) AWO_COMPOSE_NS(10) AWO_COMPOSE_NS(11)
        AWO_COMPOSE_NS(12) AWO_COMPOSE_NS(13) AWO_COMPOSE_NS(14) AWO_COMPOSE_NS(15) AWO_COMPOSE_NS(16)
#undef AWO_COMPOSE_NS
        default: return AWO_EINVAL;
    }
    return launch_status();
}

extern "C" awo_status awo_snow_cover(const float* d_h, const float* d_nz, awo_grid g, const awo_snow_params* p,
                                     float* d_alpha, uint8_t* d_rgba, void* stream)
{
    if (!d_h || !d_nz || !p || !grid_ok(g) || (!d_alpha && !d_rgba)) return AWO_EINVAL;
    if (!(p->blend_alt_m >= 0.0f) || !(p->blend_slope_deg >= 0.0f) || !(p->max_slope_deg >= 0.0f) ||
        !(p->max_slope_deg <= 90.0f) || !(p->snow_line_m > -1.0e30f && p->snow_line_m < 1.0e30f))
        return AWO_EINVAL;
    if ((((uintptr_t)d_rgba) & 3u) != 0) return AWO_EINVAL;
    const double r = 3.14159265358979323846 / 180.0;
    const double L = p->snow_line_m, b = p->blend_alt_m;
    const float a0 = (float)(L - 0.5 * b), a1 = (float)(L + 0.5 * b);
    double s_lo = (double)p->max_slope_deg + 0.5 * (double)p->blend_slope_deg;
    double s_hi = (double)p->max_slope_deg - 0.5 * (double)p->blend_slope_deg;
    if (s_lo > 90.0) s_lo = 90.0;
    if (s_hi < 0.0) s_hi = 0.0;
    const float c0 = (float)cos(s_lo * r), c1 = (float)cos(s_hi * r);
    const int64_t n = cells_of(g);
    const bool vec4 = ((((uintptr_t)d_h) | ((uintptr_t)d_nz) | ((uintptr_t)d_alpha) | ((uintptr_t)d_rgba)) & 15u) == 0;
    k_snow<<<stream_blocks(vec4 ? n / 4 + 1 : n, 256), 256, 0, as_stream(stream)>>>(d_h, d_nz, n, a0, a1, c0, c1,
                                                                                     d_alpha, d_rgba, vec4);
    return launch_status();
}
