// awo_internal.cuh -- helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "awo.h"

namespace awo {

// Validates a grid: 1 <= W, H <= 65536, W*H < 2^31, finite positive cell size.
inline bool grid_ok(awo_grid g)
{
    if (g.width < 1 || g.height < 1 || g.width > 65536 || g.height > 65536) return false;
    if ((int64_t)g.width * (int64_t)g.height >= ((int64_t)1 << 31)) return false;
    if (!(g.cell_size > 0.0f) || !(g.cell_size < 3.0e38f)) return false;
    return true;
}

inline int64_t cells_of(awo_grid g) { return (int64_t)g.width * (int64_t)g.height; }

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Status after enqueueing: any pending launch error becomes AWO_ECUDA.
inline awo_status launch_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AWO_OK : AWO_ECUDA;
}

// Number of SMs of the current device (cached per device ordinal).
int sm_count();

// Grid size for a grid-stride streaming kernel: a multiple of the SM count,
// capped by the work available.
inline unsigned stream_blocks(int64_t work_items, int threads, int per_sm = 8)
{
    int64_t want = (work_items + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (unsigned)want;
}

// Validates particle parameters for a grid of cell size cs (see awo.h).
inline bool sim_params_ok(const awo_sim_params* p, float cs)
{
    if (!p) return false;
    if (!(p->persistence >= 0.0f && p->persistence <= 1.0f)) return false;
    if (!(p->randomness >= 0.0f) || !(p->randomness < 3.0e38f)) return false;
    if (!(p->mu >= 0.0f) || !(p->mu < 3.0e38f)) return false;
    if (!(p->drag_k >= 0.0f) || !(p->drag_k < 3.0e38f)) return false;
    if (!(p->step_scale > 0.0f) || !(p->step_scale <= 1.0f)) return false;
    if (!(p->gravity > 0.0f) || !(p->gravity < 3.0e38f)) return false;
    const float D = p->step_scale * cs;
    const float kD = p->drag_k * D;
    if (!(kD < 1.0f)) return false;
    if ((p->flags & ~AWO_SIM_CLEAR_OUTPUTS) != 0u) return false;
    return true;
}

// Size of the release texture at 2^r times the resolution of grid g
// (awo_release_texture); false when r or the size is out of range.
inline bool release_texture_dims(awo_grid g, int32_t r, int64_t* wr, int64_t* hr)
{
    if (!grid_ok(g) || r < -AWO_RELEASE_LOG2_MAX || r > AWO_RELEASE_LOG2_MAX) return false;
    if (r >= 0) {
        *wr = (int64_t)g.width << r;
        *hr = (int64_t)g.height << r;
    } else {
        const int64_t q = (int64_t)1 << (-r);
        *wr = ((int64_t)g.width + q - 1) / q;
        *hr = ((int64_t)g.height + q - 1) / q;
    }
    return *wr * *hr < ((int64_t)1 << 31);
}

// Parameters and the release texture they name are valid for grid g.
inline bool sim_params_ok(const awo_sim_params* p, awo_grid g)
{
    int64_t wr, hr;
    return sim_params_ok(p, g.cell_size) && release_texture_dims(g, p->release_log2, &wr, &hr);
}

#ifdef __CUDACC__
// a / b rounded to nearest (the value of __fdiv_rn(a, b)) from y = RN(1 / b),
// the correctly rounded reciprocal, by two corrections of the quotient with
// exact FMA remainders, q' = q + (a - b q) y: the first takes q0 = RN(a y) to
// a faithful quotient (relative error about 2^-47 before its rounding), and
// the second turns a faithful quotient into the correctly rounded one
// (Markstein's theorem: P. Markstein, IBM J. Res. Dev. 34 (1990) 111-119;
// M. Cornea, J. Harrison, P. T. P. Tang, Scientific Computing on
// Itanium-based Systems, 2002).  The theorem needs every intermediate value
// normal and every remainder exact: |a| = 0 or in [2^-60, 2^60], b in
// [2^-60, 2^60]; elsewhere the intrinsic gives the value.  SIGNED: a of
// either sign (rounding to nearest is symmetric: the quotient of |a| takes
// a's sign); otherwise negative a and -0 take the intrinsic.
// awo_selftest_div_rn compares this function with the intrinsic on the
// running GPU.
template <bool SIGNED = false>
__device__ __forceinline__ float div_rn_by_rcp(float a, float b, float y)
{
    const uint32_t ab = __float_as_uint(a) & (SIGNED ? 0x7fffffffu : 0xffffffffu);
    const bool fast = (ab == 0u || (ab >= 0x21800000u && ab <= 0x5d800000u)) &&  // |a|: 0 or [2^-60, 2^60]
                      (b >= 0x1p-60f && b <= 0x1p60f);
    if (!fast) return __fdiv_rn(a, b);
    const float m = __uint_as_float(ab);
    const float q0 = __fmul_rn(m, y);
    const float q1 = __fmaf_rn(__fmaf_rn(-b, q0, m), y, q0);
    const float q2 = __fmaf_rn(__fmaf_rn(-b, q1, m), y, q1);
    return SIGNED ? __uint_as_float(__float_as_uint(q2) | (__float_as_uint(a) & 0x80000000u)) : q2;
}
#endif

// Texture view of the DEM buffer d_h of grid g for the particle kernels'
// footprint gathers, or 0 when the grid is small, the buffer or row pitch is
// not texture-aligned, the view table is full, or a new view would be needed
// while stream s is capturing (awo_simulate.cu).
cudaTextureObject_t dem_texture(const float* d_h, awo_grid g, cudaStream_t s);

}  // namespace awo
