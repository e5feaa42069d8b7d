// awo_terrain.cu -- DEM decode, normals/steepness and release-cell selection.
//
// These are streaming passes over the W x H grid (HBM-bound).  Each kernel is
// a grid-stride loop sized in multiples of the SM count, moving 16-byte
// vectors when its buffers are aligned (a general path covers ragged sizes
// and offsets).  Arithmetic uses explicit round-to-nearest intrinsics so no
// multiply-add is ever fused.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "awo_internal.cuh"
#include "awo_particle.cuh"  // rcp_sqrt_rn

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
// Four heights per thread (8-byte load, float4 store) when both buffers allow
// it, then a scalar tail.
// A thread issues the loads of DECODE_UNROLL groups of four heights (each
// coalesced across the grid) before their stores, so that enough bytes are
// in flight per SM to keep HBM busy.
constexpr int DECODE_UNROLL = 4;

__global__ void k_decode_u16(const uint16_t* __restrict__ q, int64_t n, float scale, float* __restrict__ h, bool vec4)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n4 = vec4 ? n / 4 : 0;
    for (int64_t k0 = tid; k0 < n4; k0 += DECODE_UNROLL * stride) {
        uint2 w[DECODE_UNROLL];
#pragma unroll
        for (int u = 0; u < DECODE_UNROLL; ++u) {
            const int64_t k = k0 + u * stride;
            w[u] = k < n4 ? __ldg(reinterpret_cast<const uint2*>(q) + k) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < DECODE_UNROLL; ++u) {
            const int64_t k = k0 + u * stride;
            if (k < n4)
                reinterpret_cast<float4*>(h)[k] = make_float4(__fmul_rn(__uint2float_rn(w[u].x & 0xffffu), scale),
                                                              __fmul_rn(__uint2float_rn(w[u].x >> 16), scale),
                                                              __fmul_rn(__uint2float_rn(w[u].y & 0xffffu), scale),
                                                              __fmul_rn(__uint2float_rn(w[u].y >> 16), scale));
        }
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += stride) h[i] = __fmul_rn(__uint2float_rn((unsigned)q[i]), scale);
}

// ---------------------------------------------------------------------------
// a1. normals + tan^2 + optional slope in degrees.  One thread per run of 4
// cells of a row (no 64-bit division: a 32-bit item index splits into row and
// run).  When rows are 16-byte aligned (W % 4 == 0 and aligned buffers) the
// run's heights, the rows above and below and the outputs move as float4;
// the two horizontal neighbours outside the run are scalar loads (L1 hits).
// Otherwise each cell is handled alone with the same arithmetic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void normal_of(float gx, float gy, float& nx, float& ny, float& nz, float& t2)
{
    t2 = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
    const float inv = rcp_sqrt_rn(__fadd_rn(t2, 1.0f));  // = __frcp_rn(__fsqrt_rn(.)) bit for bit, one branch
    nx = __fmul_rn(-gx, inv);
    ny = __fmul_rn(-gy, inv);
    nz = inv;
}

__device__ __forceinline__ float slope_deg_of(float t2) { return atanf(sqrtf(t2)) * 57.295779513082320876f; }

// Heights for k_normals: FP32 metres, or (FROM_U16) uint16 words decoded
// exactly as k_decode_u16 does, h = (float)q * scale.
template <bool FROM_U16>
struct HeightSrc {
    const void* p;
    float scale;
    __device__ __forceinline__ float at(int64_t i) const
    {
        if (FROM_U16) return __fmul_rn(__uint2float_rn((unsigned)__ldg(static_cast<const uint16_t*>(p) + i)), scale);
        return __ldg(static_cast<const float*>(p) + i);
    }
    // four consecutive heights from i (16-byte aligned floats / 8-byte aligned words)
    __device__ __forceinline__ float4 at4(int64_t i) const
    {
        if (FROM_U16) {
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(p) + i));
            return make_float4(__fmul_rn(__uint2float_rn(w.x & 0xffffu), scale),
                               __fmul_rn(__uint2float_rn(w.x >> 16), scale),
                               __fmul_rn(__uint2float_rn(w.y & 0xffffu), scale),
                               __fmul_rn(__uint2float_rn(w.y >> 16), scale));
        }
        return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + i));
    }
};

// FROM_U16: the heights are decoded from uint16 words and also written to
// h_out (each thread writes the cells of its run), so a0 and a1 take one
// pass: awo_decode_u16 followed by awo_normals, without re-reading h.
template <bool FROM_U16>
__global__ void __launch_bounds__(256) k_normals(const HeightSrc<FROM_U16> h, int W, int H, float cs,
                                                 float* __restrict__ nrm, float* __restrict__ tan2,
                                                 float* __restrict__ slope_deg, float* __restrict__ h_out, bool vec4)
{
    const int64_t plane = (int64_t)W * H;
    const uint32_t runs = (uint32_t)((W + 3) >> 2);
    const uint32_t items = runs * (uint32_t)H;
    const float den1 = cs, den2 = __fmul_rn(cs, 2.0f);
    const float rden1 = __frcp_rn(den1), rden2 = __frcp_rn(den2);  // the divisions: div_rn_by_rcp, = __fdiv_rn
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        const int y = (int)(it / runs);
        const int x0 = (int)(it - (uint32_t)y * runs) * 4;
        const int yl = y > 0 ? y - 1 : 0, yr = y < H - 1 ? y + 1 : H - 1;
        const float deny = yr - yl == 2 ? den2 : den1, rdeny = yr - yl == 2 ? rden2 : rden1;
        const int64_t row = (int64_t)y * W;
        if (vec4) {
            const float4 c = h.at4(row + x0);
            const float4 up = h.at4((int64_t)yl * W + x0);
            const float4 dn = h.at4((int64_t)yr * W + x0);
            const float left = x0 > 0 ? h.at(row + x0 - 1) : c.x;
            const float right = x0 + 4 < W ? h.at(row + x0 + 4) : c.w;
            if (FROM_U16) *reinterpret_cast<float4*>(h_out + row + x0) = c;
            const float hc[6] = {left, c.x, c.y, c.z, c.w, right};
            const float hu[4] = {up.x, up.y, up.z, up.w}, hd[4] = {dn.x, dn.y, dn.z, dn.w};
            float o_nx[4], o_ny[4], o_nz[4], o_t2[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = x0 + k;
                const int xl = x > 0 ? x - 1 : 0, xr = x < W - 1 ? x + 1 : W - 1;
                float gx = 0.0f, gy = 0.0f;
                const float h_r = x < W - 1 ? hc[k + 2] : hc[k + 1];
                const float h_l = x > 0 ? hc[k] : hc[k + 1];
                if (xr > xl)
                    gx = xr - xl == 2 ? div_rn_by_rcp<true>(__fsub_rn(h_r, h_l), den2, rden2)
                                      : div_rn_by_rcp<true>(__fsub_rn(h_r, h_l), den1, rden1);
                if (yr > yl) gy = div_rn_by_rcp<true>(__fsub_rn(hd[k], hu[k]), deny, rdeny);
                normal_of(gx, gy, o_nx[k], o_ny[k], o_nz[k], o_t2[k]);
            }
            if (nrm) {
                *reinterpret_cast<float4*>(nrm + row + x0) = make_float4(o_nx[0], o_nx[1], o_nx[2], o_nx[3]);
                *reinterpret_cast<float4*>(nrm + plane + row + x0) = make_float4(o_ny[0], o_ny[1], o_ny[2], o_ny[3]);
                *reinterpret_cast<float4*>(nrm + 2 * plane + row + x0) =
                    make_float4(o_nz[0], o_nz[1], o_nz[2], o_nz[3]);
            }
            if (tan2) *reinterpret_cast<float4*>(tan2 + row + x0) = make_float4(o_t2[0], o_t2[1], o_t2[2], o_t2[3]);
            if (slope_deg)
                *reinterpret_cast<float4*>(slope_deg + row + x0) =
                    make_float4(slope_deg_of(o_t2[0]), slope_deg_of(o_t2[1]), slope_deg_of(o_t2[2]),
                                slope_deg_of(o_t2[3]));
        } else {
            const int x_end = x0 + 4 < W ? x0 + 4 : W;
            for (int x = x0; x < x_end; ++x) {
                const int xl = x > 0 ? x - 1 : 0, xr = x < W - 1 ? x + 1 : W - 1;
                float gx = 0.0f, gy = 0.0f;
                if (xr > xl)
                    gx = div_rn_by_rcp<true>(__fsub_rn(h.at(row + xr), h.at(row + xl)), xr - xl == 2 ? den2 : den1,
                                             xr - xl == 2 ? rden2 : rden1);
                if (yr > yl)
                    gy = div_rn_by_rcp<true>(__fsub_rn(h.at((int64_t)yr * W + x), h.at((int64_t)yl * W + x)), deny,
                                             rdeny);
                float nx, ny, nz, t2;
                normal_of(gx, gy, nx, ny, nz, t2);
                const int64_t i = row + x;
                if (FROM_U16) h_out[i] = h.at(i);
                if (nrm) {
                    nrm[i] = nx;
                    nrm[plane + i] = ny;
                    nrm[2 * plane + i] = nz;
                }
                if (tan2) tan2[i] = t2;
                if (slope_deg) slope_deg[i] = slope_deg_of(t2);
            }
        }
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

// Selection bits of the RT_CELLS consecutive cells from `base` (bit k: cell
// base + k is in [t_lo, t_hi]; cells past n are not).  Full, 16-byte-aligned
// runs load as four float4.
__device__ __forceinline__ uint32_t select_bits(const float* __restrict__ tan2, int64_t base, int64_t n, float t_lo,
                                                float t_hi)
{
    uint32_t bits = 0u;
    if (base + RT_CELLS <= n && (((uintptr_t)(tan2 + base)) & 15u) == 0) {
        const float4* p = reinterpret_cast<const float4*>(tan2 + base);
#pragma unroll
        for (int q = 0; q < RT_CELLS / 4; ++q) {
            const float4 t = __ldg(p + q);
            bits |= ((t_lo <= t.x && t.x <= t_hi) ? 1u : 0u) << (4 * q);
            bits |= ((t_lo <= t.y && t.y <= t_hi) ? 1u : 0u) << (4 * q + 1);
            bits |= ((t_lo <= t.z && t.z <= t_hi) ? 1u : 0u) << (4 * q + 2);
            bits |= ((t_lo <= t.w && t.w <= t_hi) ? 1u : 0u) << (4 * q + 3);
        }
    } else {
#pragma unroll
        for (int k = 0; k < RT_CELLS; ++k) {
            if (base + k < n) {
                const float t = __ldg(tan2 + base + k);
                if (t_lo <= t && t <= t_hi) bits |= 1u << k;
            }
        }
    }
    return bits;
}

// Bits of the non-zero bytes among the RT_CELLS mask bytes from `base`.
__device__ __forceinline__ uint32_t mask_bits(const uint8_t* __restrict__ mask, int64_t base, int64_t n)
{
    uint32_t bits = 0u;
    if (base + RT_CELLS <= n && (((uintptr_t)(mask + base)) & 15u) == 0) {
        const uint4 m = __ldg(reinterpret_cast<const uint4*>(mask + base));
        const uint32_t w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int k = 0; k < RT_CELLS; ++k) bits |= (((w[k >> 2] >> (8 * (k & 3))) & 0xffu) != 0u ? 1u : 0u) << k;
    } else {
#pragma unroll
        for (int k = 0; k < RT_CELLS; ++k)
            if (base + k < n && __ldg(mask + base + k) != 0) bits |= 1u << k;
    }
    return bits;
}

// Writes the selection bits as 0/1 bytes (one uint4 when full and aligned).
__device__ __forceinline__ void store_mask(uint8_t* __restrict__ mask, int64_t base, int64_t n, uint32_t bits)
{
    uint32_t packed[RT_CELLS / 4];
#pragma unroll
    for (int q = 0; q < RT_CELLS / 4; ++q)
        packed[q] = ((bits >> (4 * q)) & 1u) | (((bits >> (4 * q + 1)) & 1u) << 8) |
                    (((bits >> (4 * q + 2)) & 1u) << 16) | (((bits >> (4 * q + 3)) & 1u) << 24);
    if (base + RT_CELLS <= n && (((uintptr_t)(mask + base)) & 15u) == 0) {
        *reinterpret_cast<uint4*>(mask + base) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    } else {
        for (int k = 0; k < RT_CELLS; ++k)
            if (base + k < n) mask[base + k] = (uint8_t)((bits >> k) & 1u);
    }
}

// Ordered scatter of the selected indices of this thread's run, after the
// block's exclusive scan of the per-thread counts.
__device__ __forceinline__ void scatter_bits(uint32_t bits, int64_t base, const uint32_t* __restrict__ tile_offset,
                                            uint32_t* __restrict__ cells)
{
    int total;
    int off = block_exclusive_scan(__popc(bits), &total) + (int)tile_offset[blockIdx.x];
    while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1;
        cells[off++] = (uint32_t)(base + k);
    }
}

__global__ void __launch_bounds__(RT_THREADS) k_release_mask(const float* __restrict__ tan2, int64_t n, float t_lo,
                                                             float t_hi, uint8_t* __restrict__ mask,
                                                             uint32_t* __restrict__ tile_count)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    const uint32_t bits = select_bits(tan2, base, n, t_lo, t_hi);
    if (mask) store_mask(mask, base, n, bits);
    int total;
    block_exclusive_scan(__popc(bits), &total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = (uint32_t)total;
}

// Exclusive scan of tile counts in one block of 1024 threads; also writes the
// total to *d_n.  Each thread scans a contiguous run of tiles.  Up to 16 tiles
// per thread (grids up to 2^26 cells) the run is held in registers and read
// and written as uint4 when the buffers allow, so the scan costs one round
// trip to memory; larger grids read their runs twice (measured on GB300, the
// three release passes at 8192^2: 0.106 -> 0.096 ms).
__global__ void __launch_bounds__(1024) k_release_scan(const uint32_t* __restrict__ tile_count, int n_tiles,
                                                       uint32_t* __restrict__ tile_offset, uint32_t* __restrict__ d_n)
{
    const int per = (n_tiles + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, n_tiles);
    int total;
    if (per <= 16) {
        uint32_t c[16];
        const bool vec = (per & 3) == 0 && (((uintptr_t)tile_count) & 15u) == 0 && (((uintptr_t)tile_offset) & 15u) == 0 &&
                         hi - lo == per;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (vec && 4 * q < per) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(tile_count + lo) + q);
                c[4 * q] = v.x, c[4 * q + 1] = v.y, c[4 * q + 2] = v.z, c[4 * q + 3] = v.w;
            } else {
#pragma unroll
                for (int k = 4 * q; k < 4 * q + 4; ++k) c[k] = lo + k < hi ? __ldg(tile_count + lo + k) : 0u;
            }
        }
        int s = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) s += (int)c[k];
        uint32_t run = (uint32_t)block_exclusive_scan(s, &total);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t here = run;
            run += c[k];
            c[k] = here;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (vec && 4 * q < per) {
                reinterpret_cast<uint4*>(tile_offset + lo)[q] = make_uint4(c[4 * q], c[4 * q + 1], c[4 * q + 2],
                                                                           c[4 * q + 3]);
            } else {
#pragma unroll
                for (int k = 4 * q; k < 4 * q + 4; ++k)
                    if (lo + k < hi) tile_offset[lo + k] = c[k];
            }
        }
    } else {
        // more than 16 tiles a thread (release textures): two passes over the
        // thread's range, 16-byte loads unrolled so that several are in flight
        const bool vec = (per & 3) == 0 && (((uintptr_t)tile_count) & 15u) == 0 &&
                         (((uintptr_t)tile_offset) & 15u) == 0 && hi - lo == per;
        const uint4* src = reinterpret_cast<const uint4*>(tile_count + lo);
        uint32_t s = 0u;
        if (vec) {
#pragma unroll 2
            for (int q = 0; q < per / 4; ++q) {
                const uint4 v = __ldg(src + q);
                s += v.x + v.y + v.z + v.w;
            }
        } else {
            for (int t = lo; t < hi; ++t) s += tile_count[t];
        }
        uint32_t run = (uint32_t)block_exclusive_scan((int)s, &total);
        if (vec) {
            uint4* dst = reinterpret_cast<uint4*>(tile_offset + lo);
#pragma unroll 2
            for (int q = 0; q < per / 4; ++q) {
                const uint4 v = __ldg(src + q);
                uint4 o;
                o.x = run;
                o.y = o.x + v.x;
                o.z = o.y + v.y;
                o.w = o.z + v.z;
                run = o.w + v.w;
                dst[q] = o;
            }
        } else {
            for (int t = lo; t < hi; ++t) {
                tile_offset[t] = run;
                run += tile_count[t];
            }
        }
    }
    if (threadIdx.x == 0) *d_n = (uint32_t)total;
}

__global__ void __launch_bounds__(RT_THREADS) k_release_scatter(const float* __restrict__ tan2, int64_t n, float t_lo,
                                                                float t_hi, const uint32_t* __restrict__ tile_offset,
                                                                uint32_t* __restrict__ cells)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    scatter_bits(select_bits(tan2, base, n, t_lo, t_hi), base, tile_offset, cells);
}

// Release cells given by a mask -- a caller's (known release areas, Sec. 5.2:
// "known release points encoded in a pre-computed texture") or the one the
// first release pass wrote: per-tile counts and ordered scatter of the cells
// whose mask byte is non-zero.
__global__ void __launch_bounds__(RT_THREADS) k_mask_count(const uint8_t* __restrict__ mask, int64_t n,
                                                           uint32_t* __restrict__ tile_count)
{
    const int64_t base = (int64_t)blockIdx.x * RT_TILE + (int64_t)threadIdx.x * RT_CELLS;
    int total;
    block_exclusive_scan(__popc(mask_bits(mask, base, n)), &total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = (uint32_t)total;
}

// The scatter pass takes SC_RUNS consecutive runs per thread, so a block
// covers SC_RUNS release tiles and starts at the offset of the first: four
// mask loads in flight per thread and a quarter of the blocks and block scans
// (measured on GB300, the three release passes at 8192^2: 0.111 -> 0.106 ms).
constexpr int SC_RUNS = 4;
constexpr int SC_TILE = RT_TILE * SC_RUNS;

__global__ void __launch_bounds__(RT_THREADS) k_mask_scatter(const uint8_t* __restrict__ mask, int64_t n,
                                                             const uint32_t* __restrict__ tile_offset,
                                                             uint32_t* __restrict__ cells)
{
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * (RT_CELLS * SC_RUNS);
    uint32_t bits[SC_RUNS];
    int count = 0;
#pragma unroll
    for (int r = 0; r < SC_RUNS; ++r) {
        bits[r] = mask_bits(mask, base + r * RT_CELLS, n);
        count += __popc(bits[r]);
    }
    int total;
    int off = block_exclusive_scan(count, &total) + (int)tile_offset[(int64_t)blockIdx.x * SC_RUNS];
#pragma unroll
    for (int r = 0; r < SC_RUNS; ++r) {
        uint32_t b = bits[r];
        while (b) {
            const int k = __ffs(b) - 1;
            b &= b - 1;
            cells[off++] = (uint32_t)(base + r * RT_CELLS + k);
        }
    }
}

// Launch of the scatter pass over `tiles` release tiles.
static inline void launch_mask_scatter(const uint8_t* mask, int64_t n, int tiles, const uint32_t* tile_offset,
                                       uint32_t* cells, cudaStream_t s)
{
    k_mask_scatter<<<(tiles + SC_RUNS - 1) / SC_RUNS, RT_THREADS, 0, s>>>(mask, n, tile_offset, cells);
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

// A run of RT_CELLS texels of a texture at 2^R times the DEM resolution
// (R >= 0) whose first texel index a along the row is a multiple of 2^R (every
// run of the kernel below: runs start at multiples of RT_CELLS and rows have
// W 2^R texels).  Texel a + k is centred at u = A + (2k + 1 - 2^R) / 2^(R+1)
// with A = a / 2^R, so its footprint column is A + delta(k) and its weight
// frac(k), both fixed for the run -- exactly what texel_centre and the floor
// give when no clamping occurs.
template <int R>
struct TexRun {
    static constexpr int S = 1 << R;
    __host__ __device__ static constexpr int num(int k) { return 2 * k + 1 - S; }
    __host__ __device__ static constexpr int fdiv(int x, int d) { return x >= 0 ? x / d : -((-x + d - 1) / d); }
    __host__ __device__ static constexpr int delta(int k) { return fdiv(num(k), 2 * S); }
    __host__ __device__ static constexpr float frac(int k) { return (float)(num(k) - delta(k) * 2 * S) / (float)(2 * S); }
    __host__ __device__ static constexpr float one_minus_frac(int k) { return 1.0f - frac(k); }  // exact: frac has <= 4 bits
    static constexpr int DMIN = delta(0), DMAX = delta(RT_CELLS - 1);
    static constexpr int NC = DMAX - DMIN + 2;  // footprint columns the run reads
};

// Selection bits of a run in one texture row, away from both row ends: the
// two tan^2 rows under it are loaded once (NC values each) and every texel
// interpolates with compile-time weights.  Same arithmetic as the general
// path, texel by texel.  VEC: tan2 + row + A is 16-byte aligned (tan2
// aligned, W and A multiples of 4), so the aligned groups of four among the
// NC columns are read as float4 -- a quarter of the load instructions, which
// bound this pass through the L1 otherwise.
template <int R, bool VEC>
__device__ __forceinline__ uint32_t texel_run_bits(const float* __restrict__ tan2, int row, int dj, int A, float oy,
                                                   float fy, float t_lo, float t_hi)
{
    using T = TexRun<R>;
    float top[T::NC], bot[T::NC];
    const float* p = tan2 + row + A;
#pragma unroll
    for (int i = T::DMIN; i <= T::DMAX + 1; ++i) {
        const int g = i & ~3;  // start of i's aligned group of four (relative to A)
        const bool whole = VEC && g >= T::DMIN && g + 3 <= T::DMAX + 1;
        if (whole && i == g) {
            const float4 qt = __ldg(reinterpret_cast<const float4*>(p + i));
            const float4 qb = __ldg(reinterpret_cast<const float4*>(p + dj + i));
            top[i - T::DMIN] = qt.x, top[i - T::DMIN + 1] = qt.y, top[i - T::DMIN + 2] = qt.z,
                          top[i - T::DMIN + 3] = qt.w;
            bot[i - T::DMIN] = qb.x, bot[i - T::DMIN + 1] = qb.y, bot[i - T::DMIN + 2] = qb.z,
                          bot[i - T::DMIN + 3] = qb.w;
        } else if (!whole) {
            top[i - T::DMIN] = __ldg(p + i);
            bot[i - T::DMIN] = __ldg(p + dj + i);
        }
    }
    uint32_t bits = 0u;
#pragma unroll
    for (int k = 0; k < RT_CELLS; ++k) {
        const int c = T::delta(k) - T::DMIN;
        const float fx = T::frac(k), ox = T::one_minus_frac(k);
        const float tp = __fadd_rn(__fmul_rn(top[c], ox), __fmul_rn(top[c + 1], fx));
        const float bt = __fadd_rn(__fmul_rn(bot[c], ox), __fmul_rn(bot[c + 1], fx));
        const float Tk = __fadd_rn(__fmul_rn(tp, oy), __fmul_rn(bt, fy));
        bits |= ((t_lo <= Tk && Tk <= t_hi) ? 1u : 0u) << k;
    }
    return bits;
}

// R >= 0: runs in one row away from the row ends take texel_run_bits; the
// rest (and every run when R < 0, written R = -1) the general per-texel path.
// VEC as in texel_run_bits (host-checked alignment of tan2 and W; R <= 2).
template <int R, bool VEC>
__global__ void __launch_bounds__(RT_THREADS) k_release_texture_mask(const float* __restrict__ tan2, int W, int H,
                                                                     uint32_t Wr, int64_t n, float scale,
                                                                     float t_lo, float t_hi,
                                                                     uint8_t* __restrict__ mask,
                                                                     uint32_t* __restrict__ tile_count,
                                                                     uint32_t tile0)
{
    // the texture has fewer than 2^31 texels: 32-bit indices throughout
    const uint32_t tile = tile0 + blockIdx.x;
    const uint32_t base = tile * (uint32_t)RT_TILE + threadIdx.x * (uint32_t)RT_CELLS;
    const uint32_t n32 = (uint32_t)n;
    const float wm1 = __int2float_rn(W - 1), hm1 = __int2float_rn(H - 1);
    uint32_t b = 0u, a = 0u;
    if (base < n32) {
        b = base / Wr;
        a = base - b * Wr;
    }
    // row terms, recomputed when the run wraps to the next texture row
    float v = texel_centre(b, scale, hm1);
    int j0 = __float2int_rd(v);
    float fy = __fsub_rn(v, __int2float_rn(j0)), oy = __fsub_rn(1.0f, fy);
    int row = j0 * W, dj = j0 + 1 < H ? W : 0;
    uint32_t bits = 0u;
    bool done = false;
    if (R >= 0 && base + RT_CELLS <= n32 && a + RT_CELLS <= Wr) {
        const int A = (int)(a >> (R >= 0 ? R : 0));
        if (A + TexRun<(R >= 0 ? R : 0)>::DMIN >= 0 && A + TexRun<(R >= 0 ? R : 0)>::DMAX + 1 <= W - 2) {
            bits = texel_run_bits<(R >= 0 ? R : 0), VEC>(tan2, row, dj, A, oy, fy, t_lo, t_hi);
            done = true;
        }
    }
    if (!done) {
        // footprint of the previous texel: on a finer texture 2^r consecutive
        // texels share one, so its four values are loaded once
        int o_prev = -1;
        float t00 = 0.0f, t10 = 0.0f, t01 = 0.0f, t11 = 0.0f;
#pragma unroll
        for (int k = 0; k < RT_CELLS; ++k) {
            if (base + k < n32) {
                const float u = texel_centre(a, scale, wm1);
                const int i0 = __float2int_rd(u);
                const float fx = __fsub_rn(u, __int2float_rn(i0));
                const int o = row + i0;
                if (o != o_prev) {
                    const int di = i0 + 1 < W ? 1 : 0;
                    t00 = __ldg(tan2 + o);
                    t10 = __ldg(tan2 + o + di);
                    t01 = __ldg(tan2 + o + dj);
                    t11 = __ldg(tan2 + o + dj + di);
                    o_prev = o;
                }
                const float ox = __fsub_rn(1.0f, fx);
                const float top = __fadd_rn(__fmul_rn(t00, ox), __fmul_rn(t10, fx));
                const float bot = __fadd_rn(__fmul_rn(t01, ox), __fmul_rn(t11, fx));
                const float T = __fadd_rn(__fmul_rn(top, oy), __fmul_rn(bot, fy));
                bits |= ((t_lo <= T && T <= t_hi) ? 1u : 0u) << k;
                if (++a == Wr) {
                    a = 0u;
                    ++b;
                    v = texel_centre(b, scale, hm1);
                    j0 = __float2int_rd(v);
                    fy = __fsub_rn(v, __int2float_rn(j0));
                    oy = __fsub_rn(1.0f, fy);
                    row = j0 * W;
                    dj = j0 + 1 < H ? W : 0;
                }
            }
        }
    }
    store_mask(mask, base, n, bits);
    int total;
    block_exclusive_scan(__popc(bits), &total);
    if (threadIdx.x == 0) tile_count[tile] = (uint32_t)total;
}

// Rows that share their tan^2 rows (R = 1, 2): texture rows b = 2^R j + 2^(R-1)
// ... 2^R j + 2^(R-1) + 2^R - 1 all have their centres between DEM rows j and
// j + 1, so their texels at one column interpolate the same two horizontal
// interpolations, with their own vertical weights.  A block takes one tile
// column (RT_TILE texels of a row; rows are whole tiles) of the 2^R rows of
// group j = blockIdx.y, each thread a run of RT_CELLS texels in every row:
// the tan^2 values and the horizontal interpolations are computed once for
// the group, the vertical combination per row (the same operations, in the
// same order, as k_release_texture_mask).  The 2^(R-1) rows above the first
// group and below the last clamp their centres to the grid and take
// k_release_texture_mask.
template <int R, bool VEC>
__global__ void __launch_bounds__(RT_THREADS) k_release_texture_rows(const float* __restrict__ tan2, int W, int H,
                                                                     uint32_t Wr, int64_t n, float scale,
                                                                     float t_lo, float t_hi,
                                                                     uint8_t* __restrict__ mask,
                                                                     uint32_t* __restrict__ tile_count)
{
    using T = TexRun<R>;
    constexpr int ROWS = 1 << R;
    const uint32_t tiles_per_row = Wr / (uint32_t)RT_TILE;
    const int j = (int)blockIdx.y;
    const uint32_t b0 = (uint32_t)j * ROWS + (ROWS >> 1);  // first texture row of the group
    const uint32_t a = blockIdx.x * (uint32_t)RT_TILE + threadIdx.x * (uint32_t)RT_CELLS;
    const float hm1 = __int2float_rn(H - 1), wm1 = __int2float_rn(W - 1);
    float oy[ROWS], fy[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const float v = texel_centre(b0 + r, scale, hm1);  // in [j, j + 1): floor j, no clamp
        fy[r] = __fsub_rn(v, __int2float_rn(j));
        oy[r] = __fsub_rn(1.0f, fy[r]);
    }
    const int row = j * W;  // dj = W: j + 1 <= H - 1
    uint32_t bits[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) bits[r] = 0u;
    const int A = (int)(a >> R);
    if (A + T::DMIN >= 0 && A + T::DMAX + 1 <= W - 2) {
        float top[T::NC], bot[T::NC];
        const float* p = tan2 + row + A;
#pragma unroll
        for (int i = T::DMIN; i <= T::DMAX + 1; ++i) {
            const int g = i & ~3;
            const bool whole = VEC && g >= T::DMIN && g + 3 <= T::DMAX + 1;
            if (whole && i == g) {
                const float4 qt = __ldg(reinterpret_cast<const float4*>(p + i));
                const float4 qb = __ldg(reinterpret_cast<const float4*>(p + W + i));
                top[i - T::DMIN] = qt.x, top[i - T::DMIN + 1] = qt.y, top[i - T::DMIN + 2] = qt.z,
                              top[i - T::DMIN + 3] = qt.w;
                bot[i - T::DMIN] = qb.x, bot[i - T::DMIN + 1] = qb.y, bot[i - T::DMIN + 2] = qb.z,
                              bot[i - T::DMIN + 3] = qb.w;
            } else if (!whole) {
                top[i - T::DMIN] = __ldg(p + i);
                bot[i - T::DMIN] = __ldg(p + W + i);
            }
        }
#pragma unroll
        for (int k = 0; k < RT_CELLS; ++k) {
            const int c = T::delta(k) - T::DMIN;
            const float fx = T::frac(k), ox = T::one_minus_frac(k);
            const float tp = __fadd_rn(__fmul_rn(top[c], ox), __fmul_rn(top[c + 1], fx));
            const float bt = __fadd_rn(__fmul_rn(bot[c], ox), __fmul_rn(bot[c + 1], fx));
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const float Tk = __fadd_rn(__fmul_rn(tp, oy[r]), __fmul_rn(bt, fy[r]));
                bits[r] |= ((t_lo <= Tk && Tk <= t_hi) ? 1u : 0u) << k;
            }
        }
    } else {
        // the run touches a row end: texel by texel, columns clamped as in the general path
#pragma unroll 1
        for (int k = 0; k < RT_CELLS; ++k) {
            const float u = texel_centre(a + (uint32_t)k, scale, wm1);
            const int i0 = __float2int_rd(u);
            const float fx = __fsub_rn(u, __int2float_rn(i0));
            const int o = row + i0, di = i0 + 1 < W ? 1 : 0;
            const float t00 = __ldg(tan2 + o), t10 = __ldg(tan2 + o + di);
            const float t01 = __ldg(tan2 + o + W), t11 = __ldg(tan2 + o + W + di);
            const float ox = __fsub_rn(1.0f, fx);
            const float tp = __fadd_rn(__fmul_rn(t00, ox), __fmul_rn(t10, fx));
            const float bt = __fadd_rn(__fmul_rn(t01, ox), __fmul_rn(t11, fx));
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const float Tk = __fadd_rn(__fmul_rn(tp, oy[r]), __fmul_rn(bt, fy[r]));
                bits[r] |= ((t_lo <= Tk && Tk <= t_hi) ? 1u : 0u) << k;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        store_mask(mask, (int64_t)(b0 + r) * Wr + a, n, bits[r]);
        int total;
        block_exclusive_scan(__popc(bits[r]), &total);
        if (threadIdx.x == 0) tile_count[(b0 + r) * tiles_per_row + blockIdx.x] = (uint32_t)total;
    }
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

extern "C" int32_t awo_version(void) { return 10300; }

extern "C" awo_status awo_decode_u16(const uint16_t* d_q, awo_grid g, float scale, float* d_h, void* stream)
{
    if (!d_q || !d_h || !grid_ok(g) || !(scale > 0.0f) || !(scale < 3.0e38f)) return AWO_EINVAL;
    const int64_t n = cells_of(g);
    const bool vec4 = (((uintptr_t)d_q) & 7u) == 0 && (((uintptr_t)d_h) & 15u) == 0;
    k_decode_u16<<<stream_blocks(vec4 ? n / 4 + 1 : n, 256), 256, 0, as_stream(stream)>>>(d_q, n, scale, d_h, vec4);
    return launch_status();
}

extern "C" awo_status awo_normals(const float* d_h, awo_grid g, float* d_normal, float* d_tan2,
                                  float* d_slope_deg, void* stream)
{
    if (!d_h || !grid_ok(g)) return AWO_EINVAL;
    if (!d_normal && !d_tan2 && !d_slope_deg) return AWO_OK;
    const int64_t items = (int64_t)((g.width + 3) / 4) * g.height;
    auto a16 = [](const void* p) { return p == nullptr || (((uintptr_t)p) & 15u) == 0; };
    const bool vec4 = (g.width % 4) == 0 && a16(d_h) && a16(d_normal) && a16(d_tan2) && a16(d_slope_deg);
    k_normals<false><<<stream_blocks(items, 256), 256, 0, as_stream(stream)>>>(
        HeightSrc<false>{d_h, 1.0f}, g.width, g.height, g.cell_size, d_normal, d_tan2, d_slope_deg, nullptr, vec4);
    return launch_status();
}

extern "C" awo_status awo_normals_u16(const uint16_t* d_q, awo_grid g, float scale, float* d_h, float* d_normal,
                                      float* d_tan2, float* d_slope_deg, void* stream)
{
    if (!d_q || !d_h || !grid_ok(g) || !(scale > 0.0f) || !(scale < 3.0e38f)) return AWO_EINVAL;
    if (!d_normal && !d_tan2 && !d_slope_deg) return awo_decode_u16(d_q, g, scale, d_h, stream);
    const int64_t items = (int64_t)((g.width + 3) / 4) * g.height;
    auto a16 = [](const void* p) { return p == nullptr || (((uintptr_t)p) & 15u) == 0; };
    const bool vec4 = (g.width % 4) == 0 && (((uintptr_t)d_q) & 7u) == 0 && a16(d_h) && a16(d_normal) &&
                      a16(d_tan2) && a16(d_slope_deg);
    k_normals<true><<<stream_blocks(items, 256), 256, 0, as_stream(stream)>>>(
        HeightSrc<true>{d_q, scale}, g.width, g.height, g.cell_size, d_normal, d_tan2, d_slope_deg, d_h, vec4);
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
    if (d_mask)  // 1 byte per cell instead of 4
        launch_mask_scatter(d_mask, n, tiles, tile_offset, d_cells, s);
    else
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
    if (d_mask)  // 1 byte per cell instead of 4
        launch_mask_scatter(d_mask, n, tiles, tile_offset, d_cells, s);
    else
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
    launch_mask_scatter(d_mask, n, tiles, tile_offset, d_cells, s);
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
    // float4 reads of tan2 rows: base 16-byte aligned and W a multiple of 4,
    // so that every row and every run start (a multiple of 16 / 2^r cells) is
    const bool vec = (((uintptr_t)d_tan2) & 15u) == 0 && (g.width & 3) == 0;
    auto kern = release_log2 == 0   ? (vec ? k_release_texture_mask<0, true> : k_release_texture_mask<0, false>)
                : release_log2 == 1 ? (vec ? k_release_texture_mask<1, true> : k_release_texture_mask<1, false>)
                : release_log2 == 2 ? (vec ? k_release_texture_mask<2, true> : k_release_texture_mask<2, false>)
                : release_log2 == 3 ? k_release_texture_mask<3, false>
                                    : k_release_texture_mask<-1, false>;
    if ((release_log2 == 1 || release_log2 == 2) && g.height >= 2 && wr % RT_TILE == 0) {
        // rows are whole tiles: the row groups that share their tan^2 rows in
        // one kernel, the 2^(r-1) clamped rows at each end in the other
        const uint32_t tpr = (uint32_t)(wr / RT_TILE), edge = 1u << (release_log2 - 1);
        const uint32_t last = edge + ((uint32_t)(g.height - 1) << release_log2);  // first bottom edge row
        kern<<<edge * tpr, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr, n, scale, t_lo, t_hi, d_mask,
                                                tile_count, 0u);
        kern<<<edge * tpr, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr, n, scale, t_lo, t_hi, d_mask,
                                                tile_count, last * tpr);
        const dim3 grid(tpr, (unsigned)(g.height - 1));
        if (release_log2 == 1) {
            if (vec)
                k_release_texture_rows<1, true><<<grid, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr,
                                                                           n, scale, t_lo, t_hi, d_mask, tile_count);
            else
                k_release_texture_rows<1, false><<<grid, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr,
                                                                            n, scale, t_lo, t_hi, d_mask, tile_count);
        } else {
            if (vec)
                k_release_texture_rows<2, true><<<grid, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr,
                                                                           n, scale, t_lo, t_hi, d_mask, tile_count);
            else
                k_release_texture_rows<2, false><<<grid, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr,
                                                                            n, scale, t_lo, t_hi, d_mask, tile_count);
        }
    } else {
        kern<<<tiles, RT_THREADS, 0, s>>>(d_tan2, g.width, g.height, (uint32_t)wr, n, scale, t_lo, t_hi, d_mask,
                                          tile_count, 0u);
    }
    k_release_scan<<<1, 1024, 0, s>>>(tile_count, tiles, tile_offset, d_n);
    launch_mask_scatter(d_mask, n, tiles, tile_offset, d_texels, s);
    return launch_status();
}
