// awo_overlay.cu -- velocity indicator and overlay mipmap (Sec. 3, Fig. 4).
//
// Both are streaming passes.  The mipmap is built level by level: each thread
// reduces one 2x2 block of the level above (counts summed in 64 bits and
// saturated, velocities by max), so every level reads its parent once.
#include "awo_internal.cuh"

namespace awo {

__global__ void k_finalize(const float* __restrict__ maxe, int64_t n, float g2, float* __restrict__ vel)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        vel[i] = __fsqrt_rn(__fmul_rn(g2, maxe[i]));
}

__global__ void k_lod_level(const uint32_t* __restrict__ c_in, const float* __restrict__ v_in, int w, int h,
                            uint32_t* __restrict__ c_out, float* __restrict__ v_out, int w2, int h2)
{
    const int64_t n = (int64_t)w2 * h2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int y = (int)(i / w2);
        int x = (int)(i - (int64_t)y * w2);
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
    k_finalize<<<stream_blocks(n, 256), 256, 0, as_stream(stream)>>>(d_maxe, n, 2.0f * gravity, d_vel);
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
        k_lod_level<<<stream_blocks((int64_t)w2 * h2, 256), 256, 0, s>>>(ci, vi, w, h, d_count_lv[l - 1],
                                                                         d_vel_lv[l - 1], w2, h2);
        awo_status st = launch_status();
        if (st != AWO_OK) return st;
        ci = d_count_lv[l - 1];
        vi = d_vel_lv[l - 1];
        w = w2;
        h = h2;
    }
    return AWO_OK;
}
