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

// Texture view of the DEM buffer d_h of grid g for the particle kernels'
// footprint gathers, or 0 when the grid is small, the buffer or row pitch is
// not texture-aligned, the view table is full, or a new view would be needed
// while stream s is capturing (awo_simulate.cu).
cudaTextureObject_t dem_texture(const float* d_h, awo_grid g, cudaStream_t s);

}  // namespace awo
