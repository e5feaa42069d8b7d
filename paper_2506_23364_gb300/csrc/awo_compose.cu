// awo_compose.cu -- overlay colouring / alpha blending and the snow-cover mask.
//
// Both are per-texel streaming passes (HBM-bound) over rasters the rest of the
// library produces: the velocity and count overlay (Sec. 3 compose pass,
// Fig. 4 colour scale) and the normals (Sec. 5.1 snow cover).  FP32 with
// explicit round-to-nearest intrinsics; 8-bit outputs rounded half to even.
#include <math.h>

#include "awo_internal.cuh"

namespace awo {

__device__ __forceinline__ uint8_t to_u8(float x)
{
    if (!(x > 0.0f)) return 0;
    if (x > 255.0f) return 255;
    return (uint8_t)__float2uint_rn(x);
}

__global__ void k_compose(const float* __restrict__ value, const uint32_t* __restrict__ count, int64_t n,
                          const awo_colormap cm, const uint8_t* __restrict__ base, uint8_t* __restrict__ out)
{
    const int last = cm.n_stops - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float x = value[i];
        if (!(x > cm.value[0])) x = cm.value[0];
        if (x > cm.value[last]) x = cm.value[last];
        int k = 0;
        while (k + 1 < last && x >= cm.value[k + 1]) ++k;
        const float t = __fdiv_rn(__fsub_rn(x, cm.value[k]), __fsub_rn(cm.value[k + 1], cm.value[k]));
        const float a = count[i] >= cm.count_min ? cm.alpha : 0.0f;
        uchar4 o;
        uint8_t ch[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float c0 = (float)cm.rgb[k][c], c1 = (float)cm.rgb[k + 1][c];
            const float col = __fadd_rn(c0, __fmul_rn(t, __fsub_rn(c1, c0)));
            ch[c] = base ? to_u8(__fadd_rn(__fmul_rn(a, col), __fmul_rn(__fsub_rn(1.0f, a), (float)base[4 * i + c])))
                         : to_u8(col);
        }
        o.x = ch[0];
        o.y = ch[1];
        o.z = ch[2];
        o.w = base ? base[4 * i + 3] : to_u8(__fmul_rn(255.0f, a));
        reinterpret_cast<uchar4*>(out)[i] = o;
    }
}

__device__ __forceinline__ float smooth_step(float e0, float e1, float x)
{
    if (e1 == e0) return x >= e0 ? 1.0f : 0.0f;
    float t = __fdiv_rn(__fsub_rn(x, e0), __fsub_rn(e1, e0));
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    return __fmul_rn(__fmul_rn(t, t), __fsub_rn(3.0f, __fmul_rn(2.0f, t)));
}

__global__ void k_snow(const float* __restrict__ h, const float* __restrict__ nz, int64_t n, float a0, float a1,
                       float c0, float c1, float* __restrict__ alpha, uint8_t* __restrict__ rgba)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = __fmul_rn(smooth_step(a0, a1, h[i]), smooth_step(c0, c1, nz[i]));
        if (alpha) alpha[i] = a;
        if (rgba) reinterpret_cast<uchar4*>(rgba)[i] = make_uchar4(255, 255, 255, to_u8(__fmul_rn(255.0f, a)));
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
    k_compose<<<stream_blocks(n, 256), 256, 0, as_stream(stream)>>>(d_value, d_count, n, *cm, d_base_rgba,
                                                                     d_out_rgba);
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
    k_snow<<<stream_blocks(n, 256), 256, 0, as_stream(stream)>>>(d_h, d_nz, n, a0, a1, c0, c1, d_alpha, d_rgba);
    return launch_status();
}
