// awo_terrain.cu -- DEM decode, normals/steepness and release-cell selection.
//
// These are streaming passes over the W x H grid (HBM-bound).  Each kernel is
// a grid-stride loop sized in multiples of the SM count.  Arithmetic uses
// explicit round-to-nearest intrinsics so no multiply-add is ever fused.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "awo_internal.cuh"

namespace awo {

int sm_count()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

// ---------------------------------------------------------------------------
// a0. decode: h = (float)q * scale
// ---------------------------------------------------------------------------
__global__ void k_decode_u16(const uint16_t* __restrict__ q, int64_t n, float scale, float* __restrict__ h)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        h[i] = __fmul_rn(__uint2float_rn((unsigned)q[i]), scale);
}

// ---------------------------------------------------------------------------
// a1. normals + tan^2 + optional slope in degrees.  One thread per cell of a
// row segment; neighbours come through L1/L2 (each height is read by <= 5
// threads of nearby warps).
// ---------------------------------------------------------------------------
__global__ void k_normals(const float* __restrict__ h, int W, int H, float cs, float* __restrict__ nrm,
                          float* __restrict__ tan2, float* __restrict__ slope_deg)
{
    const int64_t plane = (int64_t)W * H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += stride) {
        int y = (int)(i / W);
        int x = (int)(i - (int64_t)y * W);
        int xl = x > 0 ? x - 1 : 0, xr = x < W - 1 ? x + 1 : W - 1;
        int yl = y > 0 ? y - 1 : 0, yr = y < H - 1 ? y + 1 : H - 1;
        float gx = 0.0f, gy = 0.0f;
        if (xr > xl) {
            float den = __fmul_rn(cs, (float)(xr - xl));
            gx = __fdiv_rn(__fsub_rn(__ldg(h + (int64_t)y * W + xr), __ldg(h + (int64_t)y * W + xl)), den);
        }
        if (yr > yl) {
            float den = __fmul_rn(cs, (float)(yr - yl));
            gy = __fdiv_rn(__fsub_rn(__ldg(h + (int64_t)yr * W + x), __ldg(h + (int64_t)yl * W + x)), den);
        }
        float t2 = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
        if (nrm) {
            float inv = __frcp_rn(__fsqrt_rn(__fadd_rn(t2, 1.0f)));
            nrm[i] = __fmul_rn(-gx, inv);
            nrm[plane + i] = __fmul_rn(-gy, inv);
            nrm[2 * plane + i] = inv;
        }
        if (tan2) tan2[i] = t2;
        if (slope_deg) slope_deg[i] = atanf(sqrtf(t2)) * 57.295779513082320876f;
    }
}

// ---------------------------------------------------------------------------
// b. release selection: three passes, deterministic and ordered.
//   1. mask + per-tile count   (tile = RT_THREADS * RT_CELLS cells)
//   2. exclusive scan of the tile counts (one block)
//   3. scatter of the selected indices in increasing order
// ---------------------------------------------------------------------------
constexpr int RT_THREADS = 256;
constexpr int RT_CELLS = 16;
constexpr int RT_TILE = RT_THREADS * RT_CELLS;

__device__ __forceinline__ int block_exclusive_scan(int v, int* total)
{
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    int base = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + incl - v;
}

__global__ void __launch_bounds__(RT_THREADS) k_release_mask(const float* __restrict__ tan2, int64_t n, float t_lo,
                                                             float t_hi, uint8_t* __restrict__ mask,
                                                             uint32_t* __restrict__ tile_count)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    int cnt = 0;
    uint32_t packed[RT_CELLS / 4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < RT_CELLS; ++k) {
        int64_t i = base + k;
        if (i < n) {
            float t = __ldg(tan2 + i);
            uint32_t sel = (t_lo <= t && t <= t_hi) ? 1u : 0u;
            cnt += (int)sel;
            packed[k >> 2] |= sel << (8 * (k & 3));
        }
    }
    if (mask) {
        if (base + RT_CELLS <= n && (((uintptr_t)(mask + base)) & 15u) == 0) {
            *reinterpret_cast<uint4*>(mask + base) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        } else {
            for (int k = 0; k < RT_CELLS; ++k)
                if (base + k < n) mask[base + k] = (uint8_t)((packed[k >> 2] >> (8 * (k & 3))) & 0xffu);
        }
    }
    int total;
    block_exclusive_scan(cnt, &total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = (uint32_t)total;
}

// Exclusive scan of tile counts in one block of 1024 threads; also writes the
// total to *d_n.  Each thread scans a contiguous run of tiles.
__global__ void __launch_bounds__(1024) k_release_scan(const uint32_t* __restrict__ tile_count, int n_tiles,
                                                       uint32_t* __restrict__ tile_offset, uint32_t* __restrict__ d_n)
{
    const int per = (n_tiles + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, n_tiles);
    int s = 0;
    for (int t = lo; t < hi; ++t) s += (int)tile_count[t];
    int total;
    int run = block_exclusive_scan(s, &total);
    for (int t = lo; t < hi; ++t) {
        tile_offset[t] = (uint32_t)run;
        run += (int)tile_count[t];
    }
    if (threadIdx.x == 0) *d_n = (uint32_t)total;
}

__global__ void __launch_bounds__(RT_THREADS) k_release_scatter(const float* __restrict__ tan2, int64_t n, float t_lo,
                                                                float t_hi, const uint32_t* __restrict__ tile_offset,
                                                                uint32_t* __restrict__ cells)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < RT_CELLS; ++k) {
        int64_t i = base + k;
        if (i < n) {
            float t = __ldg(tan2 + i);
            if (t_lo <= t && t <= t_hi) bits |= 1u << k;
        }
    }
    int total;
    int off = block_exclusive_scan(__popc(bits), &total) + (int)tile_offset[blockIdx.x];
    while (bits) {
        int k = __ffs(bits) - 1;
        bits &= bits - 1;
        cells[off++] = (uint32_t)(base + k);
    }
}

// Release cells given by a caller's mask (known release areas, Sec. 5.2:
// "known release points encoded in a pre-computed texture"): per-tile counts
// and ordered scatter of the cells whose mask byte is non-zero.
__global__ void __launch_bounds__(RT_THREADS) k_mask_count(const uint8_t* __restrict__ mask, int64_t n,
                                                           uint32_t* __restrict__ tile_count)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < RT_CELLS; ++k)
        if (base + k < n) cnt += __ldg(mask + base + k) != 0 ? 1 : 0;
    int total;
    block_exclusive_scan(cnt, &total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = (uint32_t)total;
}

__global__ void __launch_bounds__(RT_THREADS) k_mask_scatter(const uint8_t* __restrict__ mask, int64_t n,
                                                             const uint32_t* __restrict__ tile_offset,
                                                             uint32_t* __restrict__ cells)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < RT_CELLS; ++k)
        if (base + k < n && __ldg(mask + base + k) != 0) bits |= 1u << k;
    int total;
    int off = block_exclusive_scan(__popc(bits), &total) + (int)tile_offset[blockIdx.x];
    while (bits) {
        int k = __ffs(bits) - 1;
        bits &= bits - 1;
        cells[off++] = (uint32_t)(base + k);
    }
}

// Release points on a texture at 2^r times the DEM resolution
// (awo_release_texture): per tile of RT_TILE texels, the mask and its count.
// A texel's steepness is the bilinear interpolation of tan^2 at its centre,
// with the footprint rule and FP32 weights of the particles' height sampling.
__device__ __forceinline__ float texel_centre(uint32_t a, float scale, float n_m1)
{
    const float c = __fsub_rn(__fmul_rn(__fadd_rn(__uint2float_rn(a), 0.5f), scale), 0.5f);
    return fminf(fmaxf(c, 0.0f), n_m1);
}

__global__ void __launch_bounds__(RT_THREADS) k_release_texture_mask(const float* __restrict__ tan2, int W, int H,
                                                                     uint32_t Wr, int64_t n, float scale,
                                                                     float t_lo, float t_hi,
                                                                     uint8_t* __restrict__ mask,
                                                                     uint32_t* __restrict__ tile_count)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    const float wm1 = __int2float_rn(W - 1), hm1 = __int2float_rn(H - 1);
    uint32_t b = 0u, a = 0u;
    if (base < n) {
        b = (uint32_t)(base / Wr);
        a = (uint32_t)(base - (int64_t)b * Wr);
    }
    float v = texel_centre(b, scale, hm1);
    int cnt = 0;
    uint32_t packed[RT_CELLS / 4] = {0u, 0u, 0u, 0u};
#pragma unroll 4
    for (int k = 0; k < RT_CELLS; ++k) {
        if (base + k < n) {
            const float u = texel_centre(a, scale, wm1);
            const int i0 = __float2int_rd(u), j0 = __float2int_rd(v);
            const float fx = __fsub_rn(u, __int2float_rn(i0)), fy = __fsub_rn(v, __int2float_rn(j0));
            const int di = i0 + 1 < W ? 1 : 0;
            const int dj = j0 + 1 < H ? W : 0;
            const int o = j0 * W + i0;
            const float t00 = __ldg(tan2 + o), t10 = __ldg(tan2 + o + di);
            const float t01 = __ldg(tan2 + o + dj), t11 = __ldg(tan2 + o + dj + di);
            const float ox = __fsub_rn(1.0f, fx), oy = __fsub_rn(1.0f, fy);
            const float top = __fadd_rn(__fmul_rn(t00, ox), __fmul_rn(t10, fx));
            const float bot = __fadd_rn(__fmul_rn(t01, ox), __fmul_rn(t11, fx));
            const float T = __fadd_rn(__fmul_rn(top, oy), __fmul_rn(bot, fy));
            const uint32_t sel = (t_lo <= T && T <= t_hi) ? 1u : 0u;
            cnt += (int)sel;
            packed[k >> 2] |= sel << (8 * (k & 3));
            if (++a == Wr) {
                a = 0u;
                ++b;
                v = texel_centre(b, scale, hm1);
            }
        }
    }
    if (base + RT_CELLS <= n && (((uintptr_t)(mask + base)) & 15u) == 0) {
        *reinterpret_cast<uint4*>(mask + base) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    } else {
        for (int k = 0; k < RT_CELLS; ++k)
            if (base + k < n) mask[base + k] = (uint8_t)((packed[k >> 2] >> (8 * (k & 3))) & 0xffu);
    }
    int total;
    block_exclusive_scan(cnt, &total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = (uint32_t)total;
}

static float tan2_of_degrees(double deg)
{
    double t = tan(deg * (3.14159265358979323846 / 180.0));
    return (float)(t * t);
}

}  // namespace awo

using namespace awo;

extern "C" const char* awo_status_string(awo_status s)
{
    switch (s) {
        case AWO_OK: return "ok";
        case AWO_EINVAL: return "invalid argument";
        case AWO_ENOMEM: return "workspace too small";
        case AWO_ECUDA: return "CUDA error";
        case AWO_ETIMEOUT: return "bounded device wait timed out";
        case AWO_EOVERFLOW: return "32-bit count overflow";
        case AWO_ECANCELLED: return "cancelled";
    }
    return "unknown status";
}

extern "C" int32_t awo_version(void) { return 10000; }

extern "C" awo_status awo_decode_u16(const uint16_t* d_q, awo_grid g, float scale, float* d_h, void* stream)
{
    if (!d_q || !d_h || !grid_ok(g) || !(scale > 0.0f) || !(scale < 3.0e38f)) return AWO_EINVAL;
    const int64_t n = cells_of(g);
    k_decode_u16<<<stream_blocks(n, 256), 256, 0, as_stream(stream)>>>(d_q, n, scale, d_h);
    return launch_status();
}

extern "C" awo_status awo_normals(const float* d_h, awo_grid g, float* d_normal, float* d_tan2,
                                  float* d_slope_deg, void* stream)
{
    if (!d_h || !grid_ok(g)) return AWO_EINVAL;
    if (!d_normal && !d_tan2 && !d_slope_deg) return AWO_OK;
    const int64_t n = cells_of(g);
    k_normals<<<stream_blocks(n, 256), 256, 0, as_stream(stream)>>>(d_h, g.width, g.height, g.cell_size, d_normal,
                                                                     d_tan2, d_slope_deg);
    return launch_status();
}

extern "C" size_t awo_release_workspace_bytes(awo_grid g)
{
    if (!grid_ok(g)) return 0;
    int64_t tiles = (cells_of(g) + RT_TILE - 1) / RT_TILE;
    return (size_t)(2 * tiles * sizeof(uint32_t) + 256);
}

extern "C" awo_status awo_release(const float* d_tan2, awo_grid g, double slope_lo_deg, double slope_hi_deg,
                                  uint8_t* d_mask, uint32_t* d_cells, uint32_t* d_n, void* d_ws, size_t ws_bytes,
                                  void* stream)
{
    if (!d_tan2 || !d_cells || !d_n || !d_ws || !grid_ok(g)) return AWO_EINVAL;
    if (!(slope_lo_deg >= 0.0) || !(slope_hi_deg < 90.0) || slope_lo_deg > slope_hi_deg) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0) return AWO_EINVAL;
    if (ws_bytes < awo_release_workspace_bytes(g)) return AWO_ENOMEM;
    const int64_t n = cells_of(g);
    const int tiles = (int)((n + RT_TILE - 1) / RT_TILE);
    uint32_t* tile_count = static_cast<uint32_t*>(d_ws);
    uint32_t* tile_offset = tile_count + tiles;
    const float t_lo = tan2_of_degrees(slope_lo_deg), t_hi = tan2_of_degrees(slope_hi_deg);
    cudaStream_t s = as_stream(stream);
    k_release_mask<<<tiles, RT_THREADS, 0, s>>>(d_tan2, n, t_lo, t_hi, d_mask, tile_count);
    k_release_scan<<<1, 1024, 0, s>>>(tile_count, tiles, tile_offset, d_n);
    k_release_scatter<<<tiles, RT_THREADS, 0, s>>>(d_tan2, n, t_lo, t_hi, tile_offset, d_cells);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Release selection with a scratch array inside the library, for callers that
// cannot pass a workspace (see awo_release_noalloc in awo.h).  The array holds
// the tile counts and tile offsets of the three passes for grids up to
// AWO_RELEASE_NOALLOC_MAX_CELLS cells.
// ---------------------------------------------------------------------------
namespace awo {

constexpr int NOALLOC_MAX_TILES = (int)(AWO_RELEASE_NOALLOC_MAX_CELLS / RT_TILE);
static __device__ __align__(256) uint32_t g_release_scratch[2 * NOALLOC_MAX_TILES];

// Device address of g_release_scratch for the current device.  In host code
// the symbol name is only a host-side stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress while that device is current.
static awo_status noalloc_scratch(uint32_t** out)
{
    static std::mutex mu;
    static std::vector<uint32_t*> addr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AWO_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_release_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return AWO_ECUDA;
        }
        addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = addr[dev];
    return AWO_OK;
}

}  // namespace awo

extern "C" awo_status awo_release_noalloc(const float* d_tan2, awo_grid g, double slope_lo_deg, double slope_hi_deg,
                                          uint8_t* d_mask, uint32_t* d_cells, uint32_t* d_n, void* stream)
{
    if (!d_tan2 || !d_cells || !d_n || !grid_ok(g)) return AWO_EINVAL;
    if (!(slope_lo_deg >= 0.0) || !(slope_hi_deg < 90.0) || slope_lo_deg > slope_hi_deg) return AWO_EINVAL;
    const int64_t n = cells_of(g);
    if (n > AWO_RELEASE_NOALLOC_MAX_CELLS) return AWO_ENOMEM;
    uint32_t* scratch = nullptr;
    awo_status st = noalloc_scratch(&scratch);
    if (st != AWO_OK) return st;
    const int tiles = (int)((n + RT_TILE - 1) / RT_TILE);
    uint32_t* tile_count = scratch;
    uint32_t* tile_offset = scratch + NOALLOC_MAX_TILES;
    const float t_lo = tan2_of_degrees(slope_lo_deg), t_hi = tan2_of_degrees(slope_hi_deg);
    cudaStream_t s = as_stream(stream);
    k_release_mask<<<tiles, RT_THREADS, 0, s>>>(d_tan2, n, t_lo, t_hi, d_mask, tile_count);
    k_release_scan<<<1, 1024, 0, s>>>(tile_count, tiles, tile_offset, d_n);
    k_release_scatter<<<tiles, RT_THREADS, 0, s>>>(d_tan2, n, t_lo, t_hi, tile_offset, d_cells);
    return launch_status();
}

extern "C" awo_status awo_release_from_mask(const uint8_t* d_mask, awo_grid g, uint32_t* d_cells, uint32_t* d_n,
                                            void* d_ws, size_t ws_bytes, void* stream)
{
    if (!d_mask || !d_cells || !d_n || !d_ws || !grid_ok(g)) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0) return AWO_EINVAL;
    if (ws_bytes < awo_release_workspace_bytes(g)) return AWO_ENOMEM;
    const int64_t n = cells_of(g);
    const int tiles = (int)((n + RT_TILE - 1) / RT_TILE);
    uint32_t* tile_count = static_cast<uint32_t*>(d_ws);
    uint32_t* tile_offset = tile_count + tiles;
    cudaStream_t s = as_stream(stream);
    k_mask_count<<<tiles, RT_THREADS, 0, s>>>(d_mask, n, tile_count);
    k_release_scan<<<1, 1024, 0, s>>>(tile_count, tiles, tile_offset, d_n);
    k_mask_scatter<<<tiles, RT_THREADS, 0, s>>>(d_mask, n, tile_offset, d_cells);
    return launch_status();
}

// ---------------------------------------------------------------------------
// b''. Release points on a texture of chosen resolution: mask and tile counts
// in one pass, then the scan and the ordered scatter of the mask's texels.
// ---------------------------------------------------------------------------
extern "C" awo_status awo_release_texture_dims(awo_grid g, int32_t release_log2, int32_t* width, int32_t* height)
{
    int64_t wr, hr;
    if (!width || !height || !release_texture_dims(g, release_log2, &wr, &hr)) return AWO_EINVAL;
    *width = (int32_t)wr;
    *height = (int32_t)hr;
    return AWO_OK;
}

extern "C" size_t awo_release_texture_workspace_bytes(awo_grid g, int32_t release_log2)
{
    int64_t wr, hr;
    if (!release_texture_dims(g, release_log2, &wr, &hr)) return 0;
    const int64_t tiles = (wr * hr + RT_TILE - 1) / RT_TILE;
    return (size_t)(2 * tiles * sizeof(uint32_t) + 256);
}

extern "C" awo_status awo_release_texture(const float* d_tan2, awo_grid g, int32_t release_log2, double slope_lo_deg,
                                          double slope_hi_deg, uint8_t* d_mask, uint32_t* d_texels, uint32_t* d_n,
                                          void* d_ws, size_t ws_bytes, void* stream)
{
    int64_t wr, hr;
    if (!d_tan2 || !d_mask || !d_texels || !d_n || !d_ws || !release_texture_dims(g, release_log2, &wr, &hr))
        return AWO_EINVAL;
    if (!(slope_lo_deg >= 0.0) || !(slope_hi_deg < 90.0) || slope_lo_deg > slope_hi_deg) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0) return AWO_EINVAL;
    if (ws_bytes < awo_release_texture_workspace_bytes(g, release_log2)) return AWO_ENOMEM;
    const int64_t n = wr * hr;
    const int tiles = (int)((n + RT_TILE - 1) / RT_TILE);
    uint32_t* tile_count = static_cast<uint32_t*>(d_ws);
    uint32_t* tile_offset = tile_count + tiles;
    const float t_lo = tan2_of_degrees(slope_lo_deg), t_hi = tan2_of_degrees(slope_hi_deg);
    const float scale = ldexpf(1.0f, -release_log2);
    cudaStream_t s = as_stream(stream);
    k_release_texture_mask<<<tiles, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr, n, scale, t_lo,
                                                        t_hi, d_mask, tile_count);
    k_release_scan<<<1, 1024, 0, s>>>(tile_count, tiles, tile_offset, d_n);
    k_mask_scatter<<<tiles, RT_THREADS, 0, s>>>(d_mask, n, tile_offset, d_texels);
    return launch_status();
}
