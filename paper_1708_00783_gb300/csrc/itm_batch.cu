// Batched per-frame core: many (scene, frame) items -- rigid submaps that one
// frame is fused into at their relative poses (InfiniTAM v3 Sec. 7.2), or
// independent scenes of different sizes -- go through allocation,
// integration and raycast with one launch per stage for the whole batch.
//
// Every stage is a persistent kernel (a fixed number of CTAs per SM) walking
// one virtual work space that concatenates the items' work: 32x8-pixel tiles
// for enumeration and raycast (sizes known on the host), and requests,
// allocated blocks and visible blocks for the other stages, whose per-item
// counts live on the device and are prefix-summed by each CTA at start.  A
// virtual index is mapped back to its item by binary search, and the item's
// work runs through the same bodies as the single-scene kernels (itm_ops.cuh),
// so each scene gets bit-identical arithmetic.  Because no launch depends on
// the work sizes, the eight launches are captured once into a CUDA graph and
// replayed for any item set up to the batch's capacity: per frame the host
// only uploads the item table (pinned ring buffer, one async copy) and
// launches the graph.
//
// Launch shapes are tunable per stage (CTAs per SM; itm_batch_set_tuning),
// and so is the schedule (itm_batch_set_schedule): the number of blocks an
// integration CTA updates at once (64 threads per block), and whether the
// enumeration and raycast CTAs walk the virtual 32x8 tiles in order or
// scattered (tile v taken as v * P mod total with P coprime to the total, so
// the items' tiles, whose costs differ by item, interleave over the grid).
// The autotuner in paper_1708_00783_gb300/autotune.py searches both.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "itm_ops.cuh"

namespace itm {

namespace {

constexpr int kMaxItems = 256;
constexpr int kRing = 4;
enum Stage { ST_ENUM = 0, ST_COMMIT, ST_VISIBLE, ST_INTEGRATE, ST_RANGE, ST_RAYCAST, ST_COUNT };

struct ItemDev {
    SceneDev s;
    const float *depth;
    float4 *vtx, *nrm;
    Intr in;
    Mat34 T, M;
    float inv_b, tB_m, inv_sv, zc;
    int max_iter;
    int cta_tiles_x;  // 32x8-pixel tiles per row
    int cta_begin;    // first virtual 32x8 tile of this item
    int rtiles_x, rtiles_y;
    int raycast;
};

struct BatchHead {
    int n, cta_total;
    int scatter_p;  // multiplier of the scattered tile order (coprime to cta_total)
    int pad;
};

// knobs of itm_batch_set_schedule
enum Knob { K_INTEG_BLOCKS = 0, K_ENUM_SCATTER, K_RAY_SCATTER, K_COUNT };

// virtual tile v in the walk order of a stage: in order, or scattered
__device__ __forceinline__ int walk_tile(int v, int total, int p, bool scatter)
{
    return scatter ? (int)(((long long)v * p) % total) : v;
}

// last index i in [0, n) with prefix[i] <= v (prefix ascending, prefix[0] = 0)
__device__ __forceinline__ int find_item(const int *prefix, int n, int v)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// prefix[i] = sum of count(item j) for j < i, prefix[n] = total (whole CTA)
template <class Count>
__device__ __forceinline__ int cta_prefix(const ItemDev *__restrict__ items, int n, int *prefix, Count count)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) prefix[i + 1] = count(items[i]);
    __syncthreads();
    if (threadIdx.x == 0) {
        prefix[0] = 0;
        for (int i = 1; i <= n; ++i) prefix[i] += prefix[i - 1];
    }
    __syncthreads();
    return prefix[n];
}

__global__ void __launch_bounds__(256) batch_begin_kernel(const ItemDev *__restrict__ items, const BatchHead *head)
{
    const int n = head->n;
    if ((int)blockIdx.x >= n) return;
    const ItemDev &it = items[blockIdx.x];
    if (threadIdx.x < kFrameCountersBytes / 4)
        reinterpret_cast<int *>(reinterpret_cast<char *>(it.s.ctr) + kFrameCountersOffset)[threadIdx.x] = 0;
    const int tiles = it.rtiles_x * it.rtiles_y;
    for (int i = threadIdx.x; i < tiles; i += blockDim.x) {
        it.s.range_min[i] = 0xffffffffu;
        it.s.range_max[i] = 0u;
    }
}

__global__ void __launch_bounds__(256) batch_enumerate_kernel(const ItemDev *__restrict__ items, const BatchHead *head,
                                                                bool scatter)
{
    __shared__ int begin[kMaxItems + 1];
    const int n = head->n, total = head->cta_total, p = head->scatter_p;
    for (int i = threadIdx.x; i < n; i += blockDim.x) begin[i] = items[i].cta_begin;
    __syncthreads();
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int vt = walk_tile(v, total, p, scatter);
        const int k = find_item(begin, n, vt);
        const ItemDev &it = items[k];
        const int local = vt - begin[k];
        enumerate_tile(it.s, it.depth, it.in, it.T, it.inv_b, local % it.cta_tiles_x, local / it.cta_tiles_x);
    }
}

__global__ void __launch_bounds__(256) batch_commit_kernel(const ItemDev *__restrict__ items, const BatchHead *head)
{
    __shared__ int prefix[kMaxItems + 1];
    const int n = head->n;
    const int total = cta_prefix(items, n, prefix, [](const ItemDev &it) {
        return min(__ldcg(&it.s.ctr->n_req), it.s.nb);
    });
    for (int i0 = blockIdx.x * blockDim.x; i0 < total; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        if (i >= total) continue;
        const int k = find_item(prefix, n, i);
        commit_request(items[k].s, i - prefix[k]);
    }
}

__global__ void __launch_bounds__(kOvfThreads) batch_overflow_kernel(const ItemDev *__restrict__ items,
                                                                     const BatchHead *head)
{
    __shared__ int remaining;
    if ((int)blockIdx.x >= head->n) return;
    overflow_scene(items[blockIdx.x].s, remaining);
}

__global__ void __launch_bounds__(256) batch_visible_kernel(const ItemDev *__restrict__ items, const BatchHead *head)
{
    __shared__ int prefix[kMaxItems + 1];
    const int n = head->n;
    const int total = cta_prefix(items, n, prefix, [](const ItemDev &it) {
        return min(__ldcg(&it.s.ctr->block_head), it.s.nv);
    });
    for (int i0 = blockIdx.x * blockDim.x; i0 < total; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        if (i >= total) continue;
        const int k = find_item(prefix, n, i);
        const ItemDev &it = items[k];
        visible_block(it.s, it.M, it.in, visible_zfar(it.s), i - prefix[k]);
    }
}

__global__ void __launch_bounds__(256) batch_integrate_kernel(const ItemDev *__restrict__ items, const BatchHead *head,
                                                              float2 nz)
{
    __shared__ int prefix[kMaxItems + 1];
    __shared__ float2 rcp_w[256];
    fill_rcp_w(rcp_w);  // read after cta_prefix's barrier
    const int n = head->n;
    const int total = cta_prefix(items, n, prefix, [](const ItemDev &it) {
        return min(__ldcg(&it.s.ctr->n_visible), it.s.nv);
    });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) {
            atomicAdd(&items[k].s.ctr->visited, (unsigned long long)(prefix[k + 1] - prefix[k]) * kBlockVoxels);
            atomicAdd(&items[k].s.ctr->frames, 1ull);
        }
    }
    // blockDim.x / 64 blocks at once, 64 threads each
    const int t = threadIdx.x & 63, per = blockDim.x >> 6;
    for (int vb = blockIdx.x * per + (threadIdx.x >> 6); vb < total; vb += gridDim.x * per) {
        const int k = find_item(prefix, n, vb);
        const ItemDev &it = items[k];
        const int ptr = vis_ptr(__ldg(&it.s.visible[vb - prefix[k]]));
        const short4 b = __ldg(&it.s.block_pos[ptr]);
        unsigned updated = 0;
        const RowData row = load_row<0>(it.s, ptr, t);
        integrate_block<0>(it.s, it.depth, nullptr, it.in, it.M, ptr, b, t, updated, row, rcp_w, nz);
        for (int o = 16; o > 0; o >>= 1) updated += __shfl_xor_sync(kFull, updated, o);
        if ((t & 31) == 0 && updated) atomicAdd(&it.s.ctr->updated, (unsigned long long)updated);
    }
}

__global__ void __launch_bounds__(256) batch_range_kernel(const ItemDev *__restrict__ items, const BatchHead *head)
{
    __shared__ int prefix[kMaxItems + 1];
    const int n = head->n;
    // work unit: a chunk of 32 allocated blocks of one item (one warp)
    const int total = cta_prefix(items, n, prefix, [](const ItemDev &it) {
        return it.raycast ? (min(__ldcg(&it.s.ctr->block_head), it.s.nv) + 31) / 32 : 0;
    });
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < total; c += warps) {
        const int k = find_item(prefix, n, c);
        const ItemDev &it = items[k];
        const int nb = min(__ldcg(&it.s.ctr->block_head), it.s.nv);
        const int i = (c - prefix[k]) * 32 + lane;
        TileRange r{0, -1, 0, -1, 0.f, 0.f};
        bool ok = false;
        if (i < nb) {
            const int ptr = __ldg(&it.s.block_free[i]);
            const short4 b = __ldg(&it.s.block_pos[ptr]);
            if (b.w) ok = block_tile_range(b, it.M, it.in, it.s.voxel_size, it.zc, it.rtiles_x, it.rtiles_y, r);
        }
        range_rasterize(ok, r, it.rtiles_x, it.s.range_min, it.s.range_max);
    }
}

__global__ void __launch_bounds__(256, 4) batch_raycast_kernel(const ItemDev *__restrict__ items, const BatchHead *head,
                                                                   bool scatter)
{
    __shared__ int begin[kMaxItems + 1];
    const int n = head->n, total = head->cta_total, p = head->scatter_p;
    for (int i = threadIdx.x; i < n; i += blockDim.x) begin[i] = items[i].cta_begin;
    __syncthreads();
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int vt = walk_tile(v, total, p, scatter);
        const int k = find_item(begin, n, vt);
        const ItemDev &it = items[k];
        if (!it.raycast) continue;
        const int local = vt - begin[k];
        raycast_tile<0, true, 1>(it.s, it.in, it.T, it.vtx, it.nrm, it.max_iter, it.tB_m, it.inv_sv,
                                 it.s.range_min, it.s.range_max, it.rtiles_x, it.rtiles_y, local % it.cta_tiles_x,
                                 local / it.cta_tiles_x);
    }
}

// The raycast's second phase over the same tiles: refinement, hit point and
// normal of the rays the march (batch_raycast_kernel) left behind the surface.
__global__ void __launch_bounds__(256, 4) batch_finish_kernel(const ItemDev *__restrict__ items, const BatchHead *head,
                                                                  bool scatter)
{
    __shared__ int begin[kMaxItems + 1];
    const int n = head->n, total = head->cta_total, p = head->scatter_p;
    for (int i = threadIdx.x; i < n; i += blockDim.x) begin[i] = items[i].cta_begin;
    __syncthreads();
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int vt = walk_tile(v, total, p, scatter);
        const int k = find_item(begin, n, vt);
        const ItemDev &it = items[k];
        if (!it.raycast) continue;
        const int local = vt - begin[k];
        raycast_tile<0, false, 2>(it.s, it.in, it.T, it.vtx, it.nrm, it.max_iter, it.tB_m, it.inv_sv, nullptr,
                                  nullptr, it.rtiles_x, it.rtiles_y, local % it.cta_tiles_x, local / it.cta_tiles_x);
    }
}

const void *stage_kernel(int st)
{
    switch (st) {
    case ST_ENUM: return (const void *)batch_enumerate_kernel;
    case ST_COMMIT: return (const void *)batch_commit_kernel;
    case ST_VISIBLE: return (const void *)batch_visible_kernel;
    case ST_INTEGRATE: return (const void *)batch_integrate_kernel;
    case ST_RANGE: return (const void *)batch_range_kernel;
    default: return (const void *)batch_raycast_kernel;
    }
}

const int kStageThreads[ST_COUNT] = {256, 256, 256, 64, 256, 256};

}  // namespace

}  // namespace itm

using namespace itm;

struct itm_batch {
    int max_items;
    ItemDev *d_items;
    BatchHead *d_head;
    unsigned char *h_stage[kRing];
    cudaEvent_t ev[kRing];
    int ring;
    int sms;
    int per_sm[ST_COUNT];  // 0: as many as fit
    int grid[ST_COUNT];
    int knob[K_COUNT];     // itm_batch_set_schedule
    int use_graph;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int have_graph;
};

static int stage_threads(const itm_batch *b, int st)
{
    return st == ST_INTEGRATE ? 64 * b->knob[K_INTEG_BLOCKS] : kStageThreads[st];
}

static void batch_grids(itm_batch *b)
{
    for (int st = 0; st < ST_COUNT; ++st) {
        int fit = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, stage_kernel(st), stage_threads(b, st), 0);
        if (fit < 1) fit = 1;
        int per = b->per_sm[st] > 0 && b->per_sm[st] < fit ? b->per_sm[st] : fit;
        b->grid[st] = b->sms * per;
    }
}

static int gcd(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// a multiplier coprime to total near 0.618 total (consecutive tiles land far
// apart in the scattered order); 1 for total <= 2
static int scatter_multiplier(int total)
{
    if (total <= 2) return 1;
    for (int p = (int)(0.6180339887 * total); p > 1; --p)
        if (gcd(p, total) == 1) return p;
    return 1;
}

static void drop_graph(itm_batch *b)
{
    if (b->have_graph) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->have_graph = 0;
    }
}

static cudaError_t launch_stages(itm_batch *b, cudaStream_t st)
{
    const ItemDev *it = b->d_items;
    const BatchHead *h = b->d_head;
    batch_begin_kernel<<<b->max_items, 256, 0, st>>>(it, h);
    batch_enumerate_kernel<<<b->grid[ST_ENUM], 256, 0, st>>>(it, h, b->knob[K_ENUM_SCATTER] != 0);
    batch_commit_kernel<<<b->grid[ST_COMMIT], 256, 0, st>>>(it, h);
    batch_overflow_kernel<<<b->max_items, kOvfThreads, 0, st>>>(it, h);
    batch_visible_kernel<<<b->grid[ST_VISIBLE], 256, 0, st>>>(it, h);
    batch_integrate_kernel<<<b->grid[ST_INTEGRATE], stage_threads(b, ST_INTEGRATE), 0, st>>>(it, h,
                                                                                        make_float2(-0.0f, -0.0f));
    batch_range_kernel<<<b->grid[ST_RANGE], 256, 0, st>>>(it, h);
    batch_raycast_kernel<<<b->grid[ST_RAYCAST], 256, 0, st>>>(it, h, b->knob[K_RAY_SCATTER] != 0);
    batch_finish_kernel<<<b->grid[ST_RAYCAST], 256, 0, st>>>(it, h, b->knob[K_RAY_SCATTER] != 0);
    return cudaGetLastError();
}

extern "C" {

int itm_batch_create(int max_items, itm_batch **out)
{
    if (!out || max_items < 1 || max_items > kMaxItems) return ITM_ERR_ARG;
    *out = nullptr;
    itm_batch *b = (itm_batch *)calloc(1, sizeof(itm_batch));
    if (!b) return ITM_ERR_ARG;
    b->max_items = max_items;
    b->use_graph = 1;
    b->knob[K_INTEG_BLOCKS] = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms < 1) b->sms = 1;
    const size_t stage_bytes = sizeof(BatchHead) + sizeof(ItemDev) * (size_t)max_items;
    cudaError_t e = cudaMalloc((void **)&b->d_head, stage_bytes);
    if (e == cudaSuccess) b->d_items = reinterpret_cast<ItemDev *>(b->d_head + 1);
    for (int r = 0; r < kRing && e == cudaSuccess; ++r) {
        e = cudaMallocHost((void **)&b->h_stage[r], stage_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev[r], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        cudaMemset(b->d_head, 0, sizeof(BatchHead));
        batch_grids(b);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        for (int r = 0; r < kRing; ++r) {
            if (b->h_stage[r]) cudaFreeHost(b->h_stage[r]);
            if (b->ev[r]) cudaEventDestroy(b->ev[r]);
        }
        if (b->d_head) cudaFree(b->d_head);
        free(b);
        cudaGetLastError();
        return ITM_ERR_CUDA;
    }
    *out = b;
    return ITM_OK;
}

int itm_batch_destroy(itm_batch *b)
{
    if (!b) return ITM_ERR_ARG;
    cudaDeviceSynchronize();
    drop_graph(b);
    for (int r = 0; r < kRing; ++r) {
        cudaFreeHost(b->h_stage[r]);
        cudaEventDestroy(b->ev[r]);
    }
    cudaFree(b->d_head);
    free(b);
    return ITM_OK;
}

int itm_batch_set_tuning(itm_batch *b, const int *ctas_per_sm, int n)
{
    if (!b || !ctas_per_sm || n != ST_COUNT) return ITM_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (ctas_per_sm[i] < 0 || ctas_per_sm[i] > 64) return ITM_ERR_ARG;
    cudaDeviceSynchronize();
    for (int i = 0; i < n; ++i) b->per_sm[i] = ctas_per_sm[i];
    batch_grids(b);
    drop_graph(b);
    return ITM_OK;
}

int itm_batch_get_tuning(itm_batch *b, int *grid_ctas, int n)
{
    if (!b || !grid_ctas || n != ST_COUNT) return ITM_ERR_ARG;
    for (int i = 0; i < n; ++i) grid_ctas[i] = b->grid[i];
    return ITM_OK;
}

int itm_batch_set_schedule(itm_batch *b, const int *knobs, int n)
{
    if (!b || !knobs || n != K_COUNT) return ITM_ERR_ARG;
    const int kb = knobs[K_INTEG_BLOCKS];
    if (!(kb == 1 || kb == 2 || kb == 4)) return ITM_ERR_ARG;
    if ((knobs[K_ENUM_SCATTER] & ~1) || (knobs[K_RAY_SCATTER] & ~1)) return ITM_ERR_ARG;
    cudaDeviceSynchronize();
    for (int i = 0; i < n; ++i) b->knob[i] = knobs[i];
    batch_grids(b);
    drop_graph(b);
    return ITM_OK;
}

int itm_batch_get_schedule(itm_batch *b, int *knobs, int n)
{
    if (!b || !knobs || n != K_COUNT) return ITM_ERR_ARG;
    for (int i = 0; i < n; ++i) knobs[i] = b->knob[i];
    return ITM_OK;
}

int itm_batch_set_graph(itm_batch *b, int use_graph)
{
    if (!b) return ITM_ERR_ARG;
    cudaDeviceSynchronize();
    b->use_graph = use_graph ? 1 : 0;
    drop_graph(b);
    return ITM_OK;
}

int itm_batch_run(itm_batch *b, const itm_batch_item *items, int n, itm_stream stream)
{
    if (!b || n < 1 || n > b->max_items || !items) return ITM_ERR_ARG;
    // validate everything before touching the device
    for (int i = 0; i < n; ++i) {
        const itm_batch_item &x = items[i];
        if (!x.scene || !x.depth_dev || !valid_intr(&x.intr)) return ITM_ERR_ARG;
        if (x.scene->d.weight_mode != 0) return ITM_ERR_ARG;
        if (x.scene->d.swap_state || x.scene->d.rgbw) return ITM_ERR_ARG;  // swapping / colour: per-scene calls
        if (x.intr.width > kRangeMaxW || x.intr.height > kRangeMaxH) return ITM_ERR_ARG;
        if ((x.vertex_dev != nullptr) != (x.normal_dev != nullptr)) return ITM_ERR_ARG;
        if ((reinterpret_cast<uintptr_t>(x.vertex_dev) & 15) || (reinterpret_cast<uintptr_t>(x.normal_dev) & 15))
            return ITM_ERR_ARG;
        for (int k = 0; k < 16; ++k)
            if (!isfinite(x.T_wc[k])) return ITM_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (items[j].scene == x.scene) return ITM_ERR_ARG;  // one frame per scene per batch
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int slot = b->ring;
    b->ring = (b->ring + 1) % kRing;
    if (cudaEventSynchronize(b->ev[slot]) != cudaSuccess) return ITM_ERR_CUDA;  // the slot's last copy is done
    BatchHead *h = reinterpret_cast<BatchHead *>(b->h_stage[slot]);
    ItemDev *it = reinterpret_cast<ItemDev *>(h + 1);
    int cta_total = 0;
    for (int i = 0; i < n; ++i) {
        const itm_batch_item &x = items[i];
        ItemDev &d = it[i];
        memset(&d, 0, sizeof(d));
        d.s = x.scene->d;
        d.depth = x.depth_dev;
        d.vtx = reinterpret_cast<float4 *>(x.vertex_dev);
        d.nrm = reinterpret_cast<float4 *>(x.normal_dev);
        d.raycast = x.vertex_dev != nullptr;
        d.in = to_intr(&x.intr);
        pose_rows(x.T_wc, d.T);
        rigid_inverse_rows(x.T_wc, d.M);
        const SceneDev &s = x.scene->d;
        d.inv_b = (float)(1.0 / (8.0 * (double)s.voxel_size));
        // the same host-side float steps as launch_raycast
        volatile float span = s.z_max - s.z_min;
        volatile float four_span = 4.0f * span;
        volatile float ratio = four_span / s.voxel_size;
        d.max_iter = (int)ratio + 64;
        volatile float tB_m = 8.0f * s.voxel_size;
        d.tB_m = tB_m;
        d.inv_sv = (float)(1.0 / (double)s.voxel_size);
        d.zc = s.z_min - 1e-3f;
        d.cta_tiles_x = (x.intr.width + 31) / 32;
        d.cta_begin = cta_total;
        cta_total += d.cta_tiles_x * ((x.intr.height + 7) / 8);
        d.rtiles_x = (x.intr.width + 7) / 8;
        d.rtiles_y = (x.intr.height + 3) / 4;
    }
    h->n = n;
    h->cta_total = cta_total;
    h->scatter_p = scatter_multiplier(cta_total);
    h->pad = 0;
    cudaError_t e = cudaMemcpyAsync(b->d_head, h, sizeof(BatchHead) + sizeof(ItemDev) * (size_t)n,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[slot], st);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    if (b->use_graph && st != nullptr) {
        if (!b->have_graph) {
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = launch_stages(b, st);
                e = cudaStreamEndCapture(st, &b->graph);
                if (e == cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e != cudaSuccess) return ITM_ERR_CUDA;
            b->have_graph = 1;
        }
        e = cudaGraphLaunch(b->exec, st);
    } else {
        e = launch_stages(b, st);
    }
    for (int i = 0; i < n; ++i) {
        items[i].scene->last_stream = st;
        items[i].scene->alloc_epoch++;  // the batch rewrote the scene's range tiles
        items[i].scene->vis_ok = false;  // and its visible list
    }
    return check_cuda(e);
}

}  // extern "C"
