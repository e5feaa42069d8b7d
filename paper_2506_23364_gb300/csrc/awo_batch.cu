// awo_batch.cu -- many avalanche-overlay requests in one persistent launch.
//
// Requests (each a DEM, a release list, parameters and rasters) travel in the
// kernel's parameter block, so a launch needs no host-to-device copy and can
// be captured in a CUDA graph.  Three kernels:
//   k_batch_prepare  one block: release counts (possibly on the device), the
//                    chunk size, the prefix sums of cells and of particle
//                    chunks over requests, zeroed counters;
//   k_batch_starts   per release cell of every request: its start record (in
//                    the processing order of awo_particle.cuh) and
//                    the release visits of its particles;
//   k_batch_simulate persistent: warps take chunks of consecutive particles
//                    from one global counter over all requests.  A warp
//                    runs one request at a time; it switches only when all
//                    its lanes are idle, which happens at request
//                    boundaries only, so the request's constants are
//                    warp-uniform.  Lanes refill as in the single-request
//                    kernel (AWO_REFILL_LANE) or start 32 particles together
//                    (AWO_REFILL_WARP); each iteration makes two moves from
//                    one Philox block, as there.
// The per-move arithmetic is the one of awo_particle.cuh, so every request's
// rasters equal those of awo_simulate on that request alone.
#include <math.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "awo_particle.cuh"

namespace awo {

struct BatchReq {
    // request constants (names read by AWO_MOVE_WORDS)
    const float* h;
    uint32_t* count;
    float* maxe;
    int W, H;
    float Wm1, Hm1, P, oneP, R, s, kD, muD;
    uint32_t max_steps;
    // work
    const uint32_t* cells;
    const uint32_t* n_cells_dev;
    uint32_t n_cells_max, n_grid, N;
    uint32_t k0, k1;      // Philox key (seed words)
    uint32_t starts_off;  // index of this request's first start record
    uint32_t texel;       // 1: the release list holds texels of the release texture
    TexelGeom tg;
    cudaTextureObject_t tex;  // texture view of h for the footprint gathers, or 0 (loads)
};

struct BatchHeader {
    unsigned long long next_chunk;                     // global work counter, in chunks
    unsigned long long chunk_prefix[AWO_BATCH_MAX + 1];  // chunks before each request
    uint32_t cell_prefix[AWO_BATCH_MAX + 1];           // start records before each request
    uint32_t n_cells[AWO_BATCH_MAX];
    uint32_t chunk;                                    // particles per chunk
    uint32_t pad;
    unsigned long long stats[AWO_BATCH_MAX][6];
    uint32_t order_sinv[AWO_BATCH_MAX];                // processing order of each request's entries
};
constexpr size_t BATCH_HEADER_BYTES = ((sizeof(BatchHeader) + 255) / 256) * 256;
// Lane refill once idle lanes add up to this many idle lane-iterations (as
// in awo_simulate.cu; 64 regions 512^2..4096^2 on GB300: 12 -> 486.8 ms,
// 8 -> 485.6 ms, 4 -> 482.7 ms per batched launch).
constexpr uint32_t BATCH_REFILL_IDLE = 4;

static_assert(sizeof(awo_sim_request) == 112, "awo_sim_request layout (C ABI)");
static_assert(offsetof(awo_sim_request, params) == 48, "awo_sim_request layout (C ABI)");
static_assert(sizeof(awo_tuning) == 16, "awo_tuning layout (C ABI)");

struct BatchArgs {
    BatchReq r[AWO_BATCH_MAX];
    KeysTable keys;  // round keys when every request has the same seed
    uint32_t n_req;
    uint32_t group;      // particles per chunk (0 = chosen by k_batch_prepare)
    uint32_t sim_warps;  // warps of the k_batch_simulate grid
    BatchHeader* hdr;
    TexelStart* starts;  // one 32-byte slot per release-list entry (a CellStart fills the first half)
};
static_assert(sizeof(BatchArgs) <= 32764, "the request table must fit the kernel parameter block");

// Warp-register copy of the current request's constants.
struct ReqRegs {
    const float* h;
    uint32_t* count;
    float* maxe;
    int W, H;
    float Wm1, Hm1, P, oneP, R, s, kD, muD;
    uint32_t max_steps, N;
    const TexelStart* starts;
    uint32_t k0, k1;
    bool texel;
    cudaTextureObject_t tex;
};

__device__ __forceinline__ ReqRegs load_req(const BatchArgs& a, int r)
{
    const BatchReq& b = a.r[r];
    ReqRegs q;
    q.h = b.h;
    q.count = b.count;
    q.maxe = b.maxe;
    q.W = b.W;
    q.H = b.H;
    q.Wm1 = b.Wm1;
    q.Hm1 = b.Hm1;
    q.P = b.P;
    q.oneP = b.oneP;
    q.R = b.R;
    q.s = b.s;
    q.kD = b.kD;
    q.muD = b.muD;
    q.max_steps = b.max_steps;
    q.N = b.N;
    q.starts = a.starts + b.starts_off;
    q.k0 = b.k0;
    q.k1 = b.k1;
    q.texel = b.texel != 0u;
    q.tex = b.tex;
    return q;
}

// Index r with prefix[r] <= g < prefix[r+1] (prefix has n + 1 entries).
template <typename T>
__device__ __forceinline__ int find_request(const T* prefix, int n, T g)
{
    int lo = 0, hi = n;  // invariant: prefix[lo] <= g < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Chunk size when the caller names none: a multiple of 32 in [32, 1024],
// about total / (warps * 16), so that every warp gets many chunks (as in
// awo_simulate.cu).
__device__ __forceinline__ uint32_t adaptive_chunk(unsigned long long total, uint32_t warps)
{
    unsigned long long c = total / ((unsigned long long)max(warps, 1u) * 16ull);
    c = c < 32ull ? 32ull : (c > 1024ull ? 1024ull : c);
    return (uint32_t)(c & ~31ull);
}

__global__ void __launch_bounds__(AWO_BATCH_MAX) k_batch_prepare(const __grid_constant__ BatchArgs a)
{
    __shared__ uint32_t s_nc[AWO_BATCH_MAX];
    __shared__ unsigned long long s_np[AWO_BATCH_MAX];
    const int t = threadIdx.x;
    uint32_t nc = 0u;
    if (t < (int)a.n_req) {
        const BatchReq& q = a.r[t];
        nc = q.n_cells_max;
        if (q.n_cells_dev) nc = min(nc, *q.n_cells_dev);
        if (q.N == 0u) nc = 0u;  // no particles, no release visits
        a.hdr->n_cells[t] = nc;
        a.hdr->order_sinv[t] = order_stride_inverse(nc / order_block(q.N));
    }
    s_nc[t] = nc;
    // particles for the particle kernel: none for a request with max_steps = 0
    // (every particle capped at its release visit, counted by k_batch_starts)
    s_np[t] = (t < (int)a.n_req && a.r[t].max_steps != 0u) ? (unsigned long long)nc * a.r[t].N : 0ull;
    for (int i = t; i < (int)a.n_req * 6; i += blockDim.x) (&a.hdr->stats[0][0])[i] = 0ull;
    __syncthreads();
    if (t == 0) {
        unsigned long long total = 0ull;
        for (int r = 0; r < (int)a.n_req; ++r) total += s_np[r];
        const uint32_t chunk = a.group ? a.group : adaptive_chunk(total, a.sim_warps);
        uint32_t cs = 0u;
        unsigned long long gs = 0ull;
        for (int r = 0; r < (int)a.n_req; ++r) {
            a.hdr->cell_prefix[r] = cs;
            a.hdr->chunk_prefix[r] = gs;
            cs += s_nc[r];
            gs += (s_np[r] + chunk - 1u) / chunk;
        }
        a.hdr->cell_prefix[a.n_req] = cs;
        a.hdr->chunk_prefix[a.n_req] = gs;
        a.hdr->chunk = chunk;
        a.hdr->next_chunk = 0ull;
    }
}

__global__ void __launch_bounds__(256) k_batch_starts(const __grid_constant__ BatchArgs a)
{
    __shared__ uint32_t s_cp[AWO_BATCH_MAX + 1];
    const int n = (int)a.n_req;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) s_cp[i] = a.hdr->cell_prefix[i];
    __syncthreads();
    const uint32_t total = s_cp[n];
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const int r = find_request<uint32_t>(s_cp, n, g);
        const BatchReq& q = a.r[r];
        const uint32_t ci = g - s_cp[r];
        const uint32_t entry = __ldg(q.cells + ci);
        const uint32_t B = order_block(q.N);
        const uint32_t slot = order_slot(ci, B, (s_cp[r + 1] - s_cp[r]) / B, a.hdr->order_sinv[r]);
        bool ok;
        if (q.texel) {
            const TexelStart st = texel_start(q.h, q.W, q.H, q.tg, entry);
            ok = st.t != ~0u;
            if (ok) atomicAdd(q.count + st.vcell, q.N);
            a.starts[q.starts_off + slot] = st;
        } else {
            const CellStart st = cell_start(q.h, q.W, q.H, q.n_grid, entry);
            ok = st.xy != ~0u;
            if (ok) atomicAdd(q.count + entry, q.N);
            *reinterpret_cast<CellStart*>(a.starts + q.starts_off + slot) = st;
        }
        // particles of entries outside the grid are rejected; with max_steps = 0
        // every particle is capped at its release visit (no particle kernel work)
        unsigned long long* st6 = a.hdr->stats[r];
        if (!ok) atomicAdd(st6 + 5, (unsigned long long)q.N);
        if (ok && q.max_steps == 0u) {
            atomicAdd(st6 + 1, (unsigned long long)q.N);
            atomicAdd(st6 + 3, (unsigned long long)q.N);
        }
    }
}

template <int THREADS, bool WARP_REFILL, bool TABLE_KEYS>
__global__ void __launch_bounds__(THREADS) k_batch_simulate(const __grid_constant__ BatchArgs a)
{
    constexpr int kGather = 2;  // footprints by texture gather where the request has a view (AWO_MOVE_WORDS)
    __shared__ unsigned long long s_gp[AWO_BATCH_MAX + 1];
    const int n_req = (int)a.n_req;
    for (int i = threadIdx.x; i <= n_req; i += blockDim.x) s_gp[i] = a.hdr->chunk_prefix[i];
    __syncthreads();
    const unsigned long long total_chunks = s_gp[n_req];
    const uint32_t chunk = a.hdr->chunk;

    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;

    int cr = -1;  // request of the warp (uniform)
    ReqRegs q = load_req(a, 0);
    // warp-uniform cursor: next particle of the request (t, and as (entry, j))
    // and the end of the chunk
    unsigned long long cur_t = 0ull, end_t = 0ull;
    uint32_t cur_ci = 0u, cur_j = 0u;
    bool exhausted = (total_chunks == 0ull);
    bool have_p = false;  // fetched chunk waiting for the warp to drain
    uint32_t idle_acc = 0u;  // idle lane-iterations since the last lane refill (warp-uniform)
    int p_r = 0;
    unsigned long long p_t = 0ull, p_end = 0ull;

    AWO_LANE_STATE

    while (true) {
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        idle_acc += (uint32_t)__popc(idle);
        // lane refill waits for BATCH_REFILL_IDLE idle lane-iterations (as in
        // the single-request kernel); warp refill for all 32 lanes
        const bool can_refill =
            idle != 0u && (WARP_REFILL ? idle == 0xffffffffu : idle_acc >= BATCH_REFILL_IDLE);
        if (can_refill) idle_acc = 0u;
        if (can_refill && cur_t >= end_t && !exhausted && !have_p) {
            unsigned long long g = 0;
            if (lane == 0) g = atomicAdd(&a.hdr->next_chunk, 1ull);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= total_chunks) {
                exhausted = true;
            } else {
                p_r = find_request<unsigned long long>(s_gp, n_req, g);
                const unsigned long long n_part = (unsigned long long)a.hdr->n_cells[p_r] * a.r[p_r].N;
                p_t = (g - s_gp[p_r]) * chunk;
                p_end = min(p_t + chunk, n_part);
                have_p = true;
            }
        }
        if (have_p && cur_t >= end_t && (p_r == cr || idle == 0xffffffffu)) {
            if (p_r != cr) {
                // all lanes are idle here; their positions are reset so that
                // the loads of dead lanes stay inside the new request's grid
                if (cr >= 0) {
                    AWO_FOLD_LANE(true, q.max_steps);
                    AWO_FLUSH_COUNTERS(a.hdr->stats[cr]);
                }
                cr = p_r;
                q = load_req(a, cr);
                u = v = 0.0f;  // (fx .. h11 are not read before the first move)
            }
            cur_t = p_t;
            end_t = p_end;
            cur_ci = (uint32_t)(p_t / q.N);  // one division per chunk
            cur_j = (uint32_t)(p_t - (unsigned long long)cur_ci * q.N);
            have_p = false;
        }
        if (can_refill && cur_t < end_t) {
            const unsigned long long left = end_t - cur_t;
            const unsigned avail = left < 32ull ? (unsigned)left : 32u;
            const unsigned want = (unsigned)__popc(idle);
            const unsigned take = want < avail ? want : avail;
            const unsigned rank = (unsigned)__popc(idle & lane_lt);
            const bool mine = ((idle >> lane) & 1u) && rank < take;
            uint32_t ci = cur_ci, jj = cur_j;
            advance(ci, jj, rank < take ? rank : 0u, q.N);
            uint4 st = make_uint4(~0u, 0u, 0u, 0u), st1 = make_uint4(0u, 0u, 0u, 0u);
            if (mine) st = __ldg(reinterpret_cast<const uint4*>(q.starts) + 2u * ci);
            if (mine && q.texel) st1 = __ldg(reinterpret_cast<const uint4*>(q.starts) + 2u * ci + 1u);
            const bool ok = mine && st.x != ~0u;  // entries outside the grid: counted by k_batch_starts
            AWO_FOLD_LANE(mine, q.max_steps);
            if (q.texel)  // warp-uniform
                AWO_LANE_START_TEXEL(ok, st, st1, jj);
            else
                AWO_LANE_START(ok, st, jj, q.W);
            my_traj += ok ? 1u : 0u;  // particles are counted when they start
            live = live || ok;
            advance(cur_ci, cur_j, take, q.N);
            cur_t += take;
        }
        if (__ballot_sync(0xffffffffu, live) == 0u) {
            if (exhausted && !have_p) break;
            continue;
        }
        if (TABLE_KEYS)
            AWO_MOVE_PAIR(q, a.keys);
        else
            AWO_MOVE_PAIR(q, (KeysWeyl{q.k0, q.k1}));
    }
    if (cr >= 0) {
        AWO_FOLD_LANE(true, q.max_steps);
        AWO_FLUSH_COUNTERS(a.hdr->stats[cr]);
    }
}

using BatchKernel = void (*)(BatchArgs);

static BatchKernel pick_kernel(int threads, int refill, bool table_keys)
{
#define AWO_K(T, W) (table_keys ? (BatchKernel)k_batch_simulate<T, W, true> : (BatchKernel)k_batch_simulate<T, W, false>)
    const bool w = refill == AWO_REFILL_WARP;
    if (threads == 64) return w ? AWO_K(64, true) : AWO_K(64, false);
    if (threads == 256) return w ? AWO_K(256, true) : AWO_K(256, false);
    return w ? AWO_K(128, true) : AWO_K(128, false);
#undef AWO_K
}

static int blocks_per_sm(BatchKernel k, int threads)
{
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, const void*>, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : cache)
        if (e.first.first == dev && e.first.second == (const void*)k) return e.second;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, threads, 0) != cudaSuccess || b < 1) b = 1;
    cache.push_back({{dev, (const void*)k}, b});
    return b;
}

static bool tuning_ok(const awo_tuning* t)
{
    if (!t) return true;
    if (t->threads_per_block != 0 && t->threads_per_block != 64 && t->threads_per_block != 128 &&
        t->threads_per_block != 256)
        return false;
    if (t->group_particles != 0 && (t->group_particles < 32 || t->group_particles > 65536)) return false;
    if (t->refill != AWO_REFILL_LANE && t->refill != AWO_REFILL_WARP) return false;
    return true;
}

static bool requests_ok(const awo_sim_request* reqs, int32_t n_req, uint64_t* total_cells)
{
    if (!reqs || n_req < 1 || n_req > AWO_BATCH_MAX) return false;
    uint64_t tot = 0;
    for (int i = 0; i < n_req; ++i) {
        const awo_sim_request& q = reqs[i];
        if (!q.d_h || !q.d_count || !q.d_maxe || !grid_ok(q.grid)) return false;
        if (q.n_cells_max > 0 && !q.d_cells) return false;
        if (!sim_params_ok(&q.params, q.grid)) return false;
        if ((((uintptr_t)q.d_count) & 3u) != 0 || (((uintptr_t)q.d_maxe) & 3u) != 0) return false;
        tot += q.n_cells_max;
    }
    if (tot >= ((uint64_t)1 << 31)) return false;
    *total_cells = tot;
    return true;
}

}  // namespace awo

using namespace awo;

extern "C" size_t awo_simulate_batched_workspace_bytes(const awo_sim_request* reqs, int32_t n_req)
{
    uint64_t tot = 0;
    if (!requests_ok(reqs, n_req, &tot)) return 0;
    return BATCH_HEADER_BYTES + (size_t)tot * sizeof(TexelStart);
}

extern "C" awo_status awo_simulate_batched(const awo_sim_request* reqs, int32_t n_req, const awo_tuning* tuning,
                                           awo_sim_stats* d_stats, void* d_ws, size_t ws_bytes, void* stream)
{
    uint64_t total = 0;
    if (!requests_ok(reqs, n_req, &total) || !tuning_ok(tuning) || !d_ws) return AWO_EINVAL;
    if ((((uintptr_t)d_ws) & 15u) != 0) return AWO_EINVAL;
    if (ws_bytes < BATCH_HEADER_BYTES + (size_t)total * sizeof(TexelStart)) return AWO_ENOMEM;
    const int threads = (tuning && tuning->threads_per_block) ? tuning->threads_per_block : 128;
    const uint32_t group = tuning ? (uint32_t)tuning->group_particles : 0u;
    const int refill = tuning ? tuning->refill : AWO_REFILL_LANE;
    cudaStream_t s = as_stream(stream);

    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.n_req = (uint32_t)n_req;
    a.hdr = static_cast<BatchHeader*>(d_ws);
    a.starts = reinterpret_cast<TexelStart*>(static_cast<char*>(d_ws) + BATCH_HEADER_BYTES);
    bool same_seed = true;
    uint32_t off = 0;
    for (int i = 0; i < n_req; ++i) {
        const awo_sim_request& q = reqs[i];
        const awo_sim_params* p = &q.params;
        const float D = p->step_scale * q.grid.cell_size;  // one FP32 rounding each, as in awo_simulate
        BatchReq& b = a.r[i];
        b.h = q.d_h;
        b.count = q.d_count;
        b.maxe = q.d_maxe;
        b.W = q.grid.width;
        b.H = q.grid.height;
        b.Wm1 = (float)(q.grid.width - 1);
        b.Hm1 = (float)(q.grid.height - 1);
        b.P = p->persistence;
        b.oneP = 1.0f - p->persistence;
        b.R = p->randomness;
        b.s = p->step_scale;
        b.kD = p->drag_k * D;
        b.muD = p->mu * D;
        b.max_steps = p->max_steps;
        b.cells = q.d_cells;
        b.n_cells_dev = q.d_n_cells;
        b.n_cells_max = q.n_cells_max;
        b.n_grid = (uint32_t)cells_of(q.grid);
        b.N = p->traj_per_cell;
        b.k0 = (uint32_t)(p->seed & 0xffffffffu);
        b.k1 = (uint32_t)(p->seed >> 32);
        b.starts_off = off;
        off += q.n_cells_max;
        int64_t wr = 0, hr = 0;
        release_texture_dims(q.grid, p->release_log2, &wr, &hr);  // checked by requests_ok
        b.texel = p->release_log2 != 0 ? 1u : 0u;
        b.tg.Wr = (uint32_t)wr;
        b.tg.n_tex = (uint32_t)(wr * hr);
        b.tg.scale = ldexpf(1.0f, -p->release_log2);
        b.tex = dem_texture(q.d_h, q.grid, s);
        if (p->seed != reqs[0].params.seed) same_seed = false;
        if (p->flags & AWO_SIM_CLEAR_OUTPUTS) {
            const size_t bytes = (size_t)cells_of(q.grid) * sizeof(uint32_t);
            if (cudaMemsetAsync(q.d_count, 0, bytes, s) != cudaSuccess) return AWO_ECUDA;
            if (cudaMemsetAsync(q.d_maxe, 0, bytes, s) != cudaSuccess) return AWO_ECUDA;
        }
    }
    uint32_t k0 = a.r[0].k0, k1 = a.r[0].k1;
    for (int r = 0; r < 10; ++r) {
        a.keys.k0[r] = k0;
        a.keys.k1[r] = k1;
        k0 += 0x9E3779B9u;  // Weyl key schedule of Philox4x32
        k1 += 0xBB67AE85u;
    }

    BatchKernel k = pick_kernel(threads, refill, same_seed);
    const unsigned blocks = (unsigned)(sm_count() * blocks_per_sm(k, threads));
    a.group = group;
    a.sim_warps = blocks * (unsigned)(threads / 32);
    k_batch_prepare<<<1, AWO_BATCH_MAX, 0, s>>>(a);
    if (total > 0) k_batch_starts<<<stream_blocks((int64_t)total, 256), 256, 0, s>>>(a);
    k<<<blocks, threads, 0, s>>>(a);
    awo_status st = launch_status();
    if (st != AWO_OK) return st;
    if (d_stats) {
        if (cudaMemcpyAsync(d_stats, a.hdr->stats, (size_t)n_req * sizeof(awo_sim_stats), cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return AWO_ECUDA;
    }
    return AWO_OK;
}

extern "C" awo_status awo_tune_batched(const awo_sim_request* reqs, int32_t n_req, void* d_ws, size_t ws_bytes,
                                       void* stream, awo_tuning* best, float* best_ms)
{
    uint64_t total = 0;
    if (!requests_ok(reqs, n_req, &total) || !best) return AWO_EINVAL;
    std::vector<awo_sim_request> rq(reqs, reqs + n_req);
    for (auto& q : rq) q.params.flags |= AWO_SIM_CLEAR_OUTPUTS;
    cudaStream_t s = as_stream(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return AWO_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return AWO_ECUDA;
    }
    const int threads[] = {64, 128, 256};
    const int groups[] = {0, 256, 1024, 4096};  // 0: chosen from the particle count
    const int refills[] = {AWO_REFILL_LANE, AWO_REFILL_WARP};
    float best_t = 3.0e38f;
    awo_tuning best_cfg = {128, 0, AWO_REFILL_LANE, 0};
    awo_status result = AWO_OK;
    for (int rf : refills)
        for (int th : threads)
            for (int gp : groups) {
                awo_tuning t = {th, gp, rf, 0};
                float t_min = 3.0e38f;
                for (int rep = 0; rep < 2 && result == AWO_OK; ++rep) {
                    if (cudaEventRecord(e0, s) != cudaSuccess) result = AWO_ECUDA;
                    if (result == AWO_OK)
                        result = awo_simulate_batched(rq.data(), n_req, &t, nullptr, d_ws, ws_bytes, stream);
                    if (result == AWO_OK && cudaEventRecord(e1, s) != cudaSuccess) result = AWO_ECUDA;
                    if (result == AWO_OK && cudaEventSynchronize(e1) != cudaSuccess) result = AWO_ECUDA;
                    float ms = 0.f;
                    if (result == AWO_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) result = AWO_ECUDA;
                    if (result == AWO_OK) t_min = std::min(t_min, ms);
                }
                if (result != AWO_OK) break;
                if (t_min < best_t) {
                    best_t = t_min;
                    best_cfg = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != AWO_OK) return result;
    *best = best_cfg;
    if (best_ms) *best_ms = best_t;
    return AWO_OK;
}
