// Sec. 5 swapping: the active part of the map in device memory, the rest in
// a host block store with one slot per hash entry.
//
// Design (Sec. 5 objectives O1-O3, in this library's terms):
//   - the host store is pinned host memory mapped into the device address
//     space: the swap kernels read and write a block's host slot directly
//     (over NVLink-C2C on a Grace host), so the host does no per-block work
//     at all (O2) and no staging copies are needed;
//   - a swapped-out block keeps its hash entry with ptr -1; its device block
//     returns to the free list;
//   - the allocation meets swapped-out keys like missing ones; the commit
//     then gives the existing entry a fresh device block (live depth is
//     integrated there at once) and marks its host data as waiting (kSwMerge);
//   - itm_swap_in fuses up to K waiting blocks into their device blocks, the
//     secondary integration (O3): per voxel (W_d F_d + W_h F_h) / (W_d + W_h),
//     weight min(W_d + W_h, max_w), a side with weight 0 contributing nothing;
//   - itm_swap_out moves up to K blocks to the host: blocks in device memory
//     with no host data waiting that no allocation segment has met for `idle`
//     allocations;
//   - both move at most K blocks per call (O1), chosen bucket by bucket and,
//     within a chain, in ascending key order: an order fixed by the set of
//     keys alone, independent of which thread won which atomic.
//
// Selection (both directions): candidates are blocks in device memory, so
// swap_scan_kernel visits the allocated blocks (the prefix of the free list),
// finds each one's entry and lists the candidates.  When there are at most K,
// all of them move and their order does not matter: that list is the
// selection.  Only when there are more do the ordered kernels run:
// swap_count_kernel counts the candidates of each chunk of 1024 buckets;
// swap_select_kernel gives each chunk its offset (the counts of the chunks
// before it), ranks its buckets with block scans in bucket order and the
// candidates of a chain by key, and writes the entry indices of ranks < K.  Eviction then frees the blocks, and a two-kernel
// compaction swaps the freed blocks of the allocated prefix of the free list
// with blocks still in use from its end, so the prefix stays "the allocated
// blocks".
#include <string.h>

#include <algorithm>
#include <vector>

#include "itm_ops.cuh"

namespace itm {

namespace {

constexpr int kSelThreads = 256;
constexpr int kRounds = 4;
constexpr int kChunk = kSelThreads * kRounds;  // buckets per selection CTA
constexpr int kMoveThreads = 128;              // one block (512 voxels) per CTA iteration
constexpr int kHdrInts = 8;

struct SwapDev {
    float *host_sdf;     // device address of the host store: slot e at e * 512
    uint8_t *host_w8;    // weight mode 0
    float *host_w32;     // weight mode 1
    int32_t *chunk;      // per bucket chunk: candidates
    int32_t *sel;        // [k] selected entry indices, in order
    int32_t *hdr;        // [0] selected, [1] holes, [2] movers, [3] allocated prefix length, [4] freed,
                         // [5] candidates found by the scan of the allocated blocks
    int32_t *holes;      // [k] free-list positions
    int32_t *movers;     // [k]
    unsigned long long *moved;  // [0] fused in, [1] moved out (cumulative)
    int k, idle;
};

// Scratch layout (int32 units after the two cumulative counters).
size_t scratch_bytes(int nb, int k)
{
    const size_t chunks = (size_t)(nb + kChunk - 1) / kChunk;
    return 2 * sizeof(unsigned long long) + sizeof(int32_t) * (chunks + 3 * (size_t)k + kHdrInts);
}

SwapDev swap_dev(const itm_scene *sc)
{
    SwapDev w;
    const size_t chunks = (size_t)(sc->d.nb + kChunk - 1) / kChunk;
    unsigned char *p = static_cast<unsigned char *>(sc->swap_scratch);
    w.moved = reinterpret_cast<unsigned long long *>(p);
    int32_t *q = reinterpret_cast<int32_t *>(p + 2 * sizeof(unsigned long long));
    w.hdr = q;
    w.chunk = q + kHdrInts;
    w.sel = w.chunk + chunks;
    w.holes = w.sel + sc->swap_k;
    w.movers = w.holes + sc->swap_k;
    void *dev_sdf = nullptr, *dev_w = nullptr;
    cudaHostGetDevicePointer(&dev_sdf, sc->host_sdf, 0);
    cudaHostGetDevicePointer(&dev_w, sc->host_w, 0);
    w.host_sdf = static_cast<float *>(dev_sdf);
    w.host_w8 = sc->d.weight_mode == 0 ? static_cast<uint8_t *>(dev_w) : nullptr;
    w.host_w32 = sc->d.weight_mode == 1 ? static_cast<float *>(dev_w) : nullptr;
    w.k = sc->swap_k;
    w.idle = sc->swap_idle;
    return w;
}

__device__ __forceinline__ int block_sum(int v, int *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// inclusive scan over the CTA (thread order); total of all threads
__device__ __forceinline__ int block_scan(int v, int *red, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) red[warp] = x;
    __syncthreads();
    int before = 0;
    total = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        if (i < warp) before += red[i];
        total += red[i];
    }
    return before + x;
}

template <bool OUT>
__device__ __forceinline__ bool candidate(const SceneDev &s, const SwapDev &w, const int4 &e, int idx)
{
    const uint8_t st = s.swap_state[idx];
    if (OUT) return e.w >= 0 && st == kSwDevice && s.swap_frame - __ldcg(&s.touch[e.w]) >= w.idle;
    return st == kSwMerge;
}

// candidates in bucket h's chain
template <bool OUT>
__device__ int bucket_count(const SceneDev &s, const SwapDev &w, int h)
{
    const int4 *E = reinterpret_cast<const int4 *>(s.entries);
    int idx = h, c = 0;
    for (int guard = 0; guard <= s.ne; ++guard) {
        const int4 e = __ldcg(&E[idx]);
        if ((e.y >> 16) == 0) break;  // a bucket that was never used starts no chain
        c += candidate<OUT>(s, w, e, idx);
        if (e.z < 1 || !ITM_IN_BOUNDS(s, e.z - 1 < s.ne)) break;
        idx = s.nb + e.z - 1;
    }
    return c;
}

// Writes the candidates of bucket h's chain at ranks first + (rank by key).
template <bool OUT>
__device__ void emit_bucket(const SceneDev &s, const SwapDev &w, int h, int first)
{
    const int4 *E = reinterpret_cast<const int4 *>(s.entries);
    int idx = h;
    for (int guard = 0; guard <= s.ne; ++guard) {
        const int4 e = __ldcg(&E[idx]);
        if (candidate<OUT>(s, w, e, idx)) {
            const unsigned long long key = entry_key(e);
            int rank = 0, j = h;
            for (int g2 = 0; g2 <= s.ne; ++g2) {
                const int4 f = __ldcg(&E[j]);
                if (j != idx && entry_key(f) < key && candidate<OUT>(s, w, f, j)) ++rank;
                if (f.z < 1 || !ITM_IN_BOUNDS(s, f.z - 1 < s.ne)) break;
                j = s.nb + f.z - 1;
            }
            if (first + rank < w.k) w.sel[first + rank] = idx;
        }
        if (e.z < 1 || !ITM_IN_BOUNDS(s, e.z - 1 < s.ne)) break;
        idx = s.nb + e.z - 1;
    }
}

// The entry holding block ptr (coordinates b): the chain element with b's key
// and that ptr, or -1.
__device__ __forceinline__ int entry_of(const SceneDev &s, short4 b, int ptr)
{
    const unsigned long long key = pack_key(b.x, b.y, b.z);
    const int4 *E = reinterpret_cast<const int4 *>(s.entries);
    int idx = (int)hash_bucket(b.x, b.y, b.z, (uint32_t)(s.nb - 1));
    for (int guard = 0; guard <= s.ne; ++guard) {
        const int4 e = __ldcg(&E[idx]);
        if (entry_key(e) == key) return e.w == ptr ? idx : -1;
        if (e.z < 1 || !ITM_IN_BOUNDS(s, e.z - 1 < s.ne)) return -1;
        idx = s.nb + e.z - 1;
    }
    return -1;
}

// Candidates among the allocated blocks: hdr[5] counts them, the first K
// found are listed.
template <bool OUT>
__global__ void __launch_bounds__(256) swap_scan_kernel(SceneDev s, SwapDev w)
{
    const int head = min(__ldcg(&s.ctr->block_head), s.nv);
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x; p0 < head; p0 += stride) {
        const int p = p0 + threadIdx.x;
        bool cand = false;
        int idx = -1;
        if (p < head) {
            const int ptr = __ldcg(&s.block_free[p]);
            if (ptr >= 0 && ptr < s.nv) {
                const short4 b = __ldcg(&s.block_pos[ptr]);
                if (b.w) {
                    idx = entry_of(s, b, ptr);
                    cand = idx >= 0 && candidate<OUT>(s, w, __ldcg(reinterpret_cast<const int4 *>(s.entries) + idx), idx);
                }
            }
        }
        if (cand) {
            const int q = warp_append(&w.hdr[5]);
            if (q < w.k) w.sel[q] = idx;
        }
    }
}

// The ordered selection runs only when the scan found more than K.
__device__ __forceinline__ bool scan_was_enough(const SwapDev &w)
{
    const int found = __ldcg(&w.hdr[5]);
    if (found > w.k) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) w.hdr[0] = found;
    return true;
}

template <bool OUT>
__global__ void __launch_bounds__(kSelThreads) swap_count_kernel(SceneDev s, SwapDev w)
{
    if (scan_was_enough(w)) return;  // uniform
    __shared__ int red[kSelThreads / 32];
    int c = 0;
    for (int r = 0; r < kRounds; ++r) {
        const int h = blockIdx.x * kChunk + r * kSelThreads + threadIdx.x;
        if (h < s.nb) c += bucket_count<OUT>(s, w, h);
    }
    c = block_sum(c, red);
    if (threadIdx.x == 0) w.chunk[blockIdx.x] = c;
}

template <bool OUT>
__global__ void __launch_bounds__(kSelThreads) swap_select_kernel(SceneDev s, SwapDev w, int n_chunks)
{
    if (__ldcg(&w.hdr[5]) <= w.k) return;  // the scan's list is the selection
    __shared__ int red[kSelThreads / 32];
    int before = 0, all = 0;
    for (int c = threadIdx.x; c < n_chunks; c += kSelThreads) {
        const int v = __ldcg(&w.chunk[c]);
        if (c < (int)blockIdx.x) before += v;
        all += v;
    }
    before = block_sum(before, red);
    if (blockIdx.x == 0) {
        all = block_sum(all, red);
        if (threadIdx.x == 0) w.hdr[0] = min(all, w.k);
    }
    if (before >= w.k) return;  // uniform over the CTA
    int base = before;
    for (int r = 0; r < kRounds; ++r) {
        const int h = blockIdx.x * kChunk + r * kSelThreads + threadIdx.x;
        const int c = h < s.nb ? bucket_count<OUT>(s, w, h) : 0;
        int total = 0;
        const int incl = block_scan(c, red, total);
        const int first = base + incl - c;
        if (c > 0 && first < w.k) emit_bucket<OUT>(s, w, h, first);
        base += total;
        if (base >= w.k) break;  // uniform
    }
}

// Each selected block to its host slot; the device block is reset (sdf 1,
// weight 0), leaves the allocated set and is marked freed (touch -1).  One
// thread claims the entry (its ptr exchanged for -1), so an entry is moved
// once even if it were listed twice; an entry that is not a block in device
// memory is skipped and reported (ITM_ST_BOUNDS).  hdr[4] counts the blocks
// actually freed.
template <int MODE>
__global__ void __launch_bounds__(kMoveThreads) swap_out_kernel(SceneDev s, SwapDev w)
{
    __shared__ int s_idx, s_ptr;
    const int n = __ldcg(&w.hdr[0]);
    const int t = threadIdx.x;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        if (t == 0) {
            const int idx = __ldcg(&w.sel[j]);
            int ptr = -1;
            if (idx >= 0 && idx < s.nb + s.ne && s.swap_state[idx] == kSwDevice) {
                ptr = atomicExch(&s.entries[idx].ptr, -1);
                if (ptr >= s.nv || ptr < -1) ptr = -1;  // not a block index: nothing to move
            }
            if (ptr < 0) set_status(s, ITM_ST_BOUNDS);
            s_idx = idx;
            s_ptr = ptr;
        }
        __syncthreads();
        const int idx = s_idx, ptr = s_ptr;
        __syncthreads();
        if (ptr < 0) continue;  // uniform over the CTA
        float4 *F = reinterpret_cast<float4 *>(s.sdf + (size_t)ptr * kBlockVoxels);
        float4 *HF = reinterpret_cast<float4 *>(w.host_sdf + (size_t)idx * kBlockVoxels);
        HF[t] = __ldcg(&F[t]);
        F[t] = make_float4(1.f, 1.f, 1.f, 1.f);
        if (MODE == 0) {
            if (t < kBlockVoxels / 16) {
                uint4 *Wd = reinterpret_cast<uint4 *>(s.w8 + (size_t)ptr * kBlockVoxels);
                reinterpret_cast<uint4 *>(w.host_w8 + (size_t)idx * kBlockVoxels)[t] = __ldcg(&Wd[t]);
                Wd[t] = make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
            float4 *Wd = reinterpret_cast<float4 *>(s.w32 + (size_t)ptr * kBlockVoxels);
            reinterpret_cast<float4 *>(w.host_w32 + (size_t)idx * kBlockVoxels)[t] = __ldcg(&Wd[t]);
            Wd[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (t == 0) {
            s.swap_state[idx] = kSwHost;
            s.block_pos[ptr].w = 0;
            s.touch[ptr] = -1;
            atomicAdd(&w.hdr[4], 1);
        }
    }
}

// Free-list positions below the new prefix end that hold freed blocks
// (holes) and positions at or above it that hold blocks in use (movers);
// there are as many of each.
__global__ void __launch_bounds__(256) swap_compact_find_kernel(SceneDev s, SwapDev w)
{
    const int head = min(__ldcg(&s.ctr->block_head), s.nv);
    const int n = __ldcg(&w.hdr[4]);
    const int new_head = head - n;
    if (blockIdx.x == 0 && threadIdx.x == 0) w.hdr[3] = head;
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x; p0 < head; p0 += stride) {
        const int p = p0 + threadIdx.x;
        bool hole = false, mover = false;
        if (p < head) {
            const int ptr = __ldcg(&s.block_free[p]);
            const bool freed = ptr >= 0 && ptr < s.nv && __ldcg(&s.touch[ptr]) == -1;
            hole = p < new_head && freed;
            mover = p >= new_head && !freed;
        }
        // at most n <= k of each while every freed block is marked once;
        // the checks keep the lists in bounds regardless
        if (hole) {
            const int q = warp_append(&w.hdr[1]);
            if (q < w.k) w.holes[q] = p;
            else set_status(s, ITM_ST_BOUNDS);
        }
        if (mover) {
            const int q = warp_append(&w.hdr[2]);
            if (q < w.k) w.movers[q] = p;
            else set_status(s, ITM_ST_BOUNDS);
        }
    }
}

__global__ void __launch_bounds__(256) swap_compact_pair_kernel(SceneDev s, SwapDev w)
{
    const int n = min(min(__ldcg(&w.hdr[1]), __ldcg(&w.hdr[2])), w.k);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int a = w.holes[j], b = w.movers[j];
        const int pa = s.block_free[a];
        s.block_free[a] = s.block_free[b];
        s.block_free[b] = pa;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.ctr->block_head = __ldcg(&w.hdr[3]) - __ldcg(&w.hdr[4]);
        w.moved[1] += (unsigned long long)__ldcg(&w.hdr[4]);
    }
}

// Secondary fusion of one voxel: device (F, W) with host (Fh, Wh).
__device__ __forceinline__ void fuse_voxel(float &F, float &W, float Fh, float Wh, float max_w)
{
    if (!(Wh > 0.0f)) return;
    if (!(W > 0.0f)) {
        F = Fh;
        W = Wh;
        return;
    }
    const float den = fadd(W, Wh);
    F = fdiv(fadd(fmul(W, F), fmul(Wh, Fh)), den);
    W = den < max_w ? den : max_w;
}

// Each selected waiting block fused with its host slot.  Thread 0 reads the
// entry once and shares it (the state it then updates is read by no other
// thread); an entry that is not a block waiting for its host data is skipped
// and reported (ITM_ST_BOUNDS).
template <int MODE>
__global__ void __launch_bounds__(kMoveThreads) swap_in_kernel(SceneDev s, SwapDev w)
{
    __shared__ int s_idx, s_ptr;
    const int n = __ldcg(&w.hdr[0]);
    const int t = threadIdx.x;
    const float max_w = (float)s.max_w;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        if (t == 0) {
            const int idx = __ldcg(&w.sel[j]);
            int ptr = -1;
            if (idx >= 0 && idx < s.nb + s.ne && s.swap_state[idx] == kSwMerge) {
                ptr = __ldcg(&s.entries[idx].ptr);
                if (ptr >= s.nv) ptr = -1;
                if (ptr >= 0) s.swap_state[idx] = kSwDevice;  // claimed: fused once
            }
            if (ptr < 0) set_status(s, ITM_ST_BOUNDS);
            s_idx = idx;
            s_ptr = ptr;
        }
        __syncthreads();
        const int idx = s_idx, ptr = s_ptr;
        __syncthreads();
        if (ptr < 0) continue;  // uniform over the CTA
        float4 *F4 = reinterpret_cast<float4 *>(s.sdf + (size_t)ptr * kBlockVoxels);
        const float4 h4 = reinterpret_cast<const float4 *>(w.host_sdf + (size_t)idx * kBlockVoxels)[t];
        const float4 d4 = __ldcg(&F4[t]);
        float F[4] = {d4.x, d4.y, d4.z, d4.w}, Fh[4] = {h4.x, h4.y, h4.z, h4.w}, W[4], Wh[4];
        if (MODE == 0) {
            const uint32_t wd = __ldcg(reinterpret_cast<const uint32_t *>(s.w8 + (size_t)ptr * kBlockVoxels) + t);
            const uint32_t wh = reinterpret_cast<const uint32_t *>(w.host_w8 + (size_t)idx * kBlockVoxels)[t];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                W[q] = (float)((wd >> (8 * q)) & 0xffu);
                Wh[q] = (float)((wh >> (8 * q)) & 0xffu);
            }
        } else {
            const float4 wd = __ldcg(reinterpret_cast<const float4 *>(s.w32 + (size_t)ptr * kBlockVoxels) + t);
            const float4 wh = reinterpret_cast<const float4 *>(w.host_w32 + (size_t)idx * kBlockVoxels)[t];
            W[0] = wd.x; W[1] = wd.y; W[2] = wd.z; W[3] = wd.w;
            Wh[0] = wh.x; Wh[1] = wh.y; Wh[2] = wh.z; Wh[3] = wh.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) fuse_voxel(F[q], W[q], Fh[q], Wh[q], max_w);
        F4[t] = make_float4(F[0], F[1], F[2], F[3]);
        if (MODE == 0) {
            uint32_t packed = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) packed |= (uint32_t)W[q] << (8 * q);  // integers <= max_w <= 255
            reinterpret_cast<uint32_t *>(s.w8 + (size_t)ptr * kBlockVoxels)[t] = packed;
        } else {
            reinterpret_cast<float4 *>(s.w32 + (size_t)ptr * kBlockVoxels)[t] = make_float4(W[0], W[1], W[2], W[3]);
        }
    }
    if (blockIdx.x == 0 && t == 0) w.moved[0] += (unsigned long long)n;
}

int move_grid(int k)
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = 8 * (sms > 0 ? sms : 1);
    }
    return k < g ? k : g;
}

template <bool OUT>
cudaError_t launch_select(const SceneDev &s, const SwapDev &w, cudaStream_t st)
{
    const int n_chunks = (s.nb + kChunk - 1) / kChunk;
    cudaError_t e = cudaMemsetAsync(w.hdr, 0, kHdrInts * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = std::max(1, std::min(4 * sms, (s.nv + 255) / 256));
    swap_scan_kernel<OUT><<<g, 256, 0, st>>>(s, w);
    swap_count_kernel<OUT><<<n_chunks, kSelThreads, 0, st>>>(s, w);
    swap_select_kernel<OUT><<<n_chunks, kSelThreads, 0, st>>>(s, w, n_chunks);
    return cudaGetLastError();
}

}  // namespace

}  // namespace itm

using namespace itm;

extern "C" {

int itm_swap_enable(itm_scene *sc, int transfer_blocks, int idle_frames)
{
    if (!sc || transfer_blocks < 1 || transfer_blocks > (1 << 24) || idle_frames < 0) return ITM_ERR_ARG;
    if (sc->d.swap_state) return ITM_ERR_ARG;  // already on
    if (sc->d.rgbw) return ITM_ERR_ARG;        // colour voxels are not swapped
    SceneDev &d = sc->d;
    const size_t slots = (size_t)d.nb + (size_t)d.ne;
    const size_t wbytes = d.weight_mode == 0 ? 1 : 4;
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    uint8_t *state = nullptr;
    int32_t *touch = nullptr;
    void *scratch = nullptr, *hs = nullptr, *hw = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&state, slots);
    if (e == cudaSuccess) e = cudaMalloc((void **)&touch, sizeof(int32_t) * (size_t)(d.nv > 0 ? d.nv : 1));
    if (e == cudaSuccess) e = cudaMalloc(&scratch, scratch_bytes(d.nb, transfer_blocks));
    if (e == cudaSuccess) e = cudaHostAlloc(&hs, slots * kBlockVoxels * sizeof(float), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&hw, slots * kBlockVoxels * wbytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMemset(state, 0, slots);
    if (e == cudaSuccess) e = cudaMemset(touch, 0, sizeof(int32_t) * (size_t)(d.nv > 0 ? d.nv : 1));
    if (e == cudaSuccess) e = cudaMemset(scratch, 0, scratch_bytes(d.nb, transfer_blocks));
    if (e != cudaSuccess) {
        if (state) cudaFree(state);
        if (touch) cudaFree(touch);
        if (scratch) cudaFree(scratch);
        if (hs) cudaFreeHost(hs);
        if (hw) cudaFreeHost(hw);
        cudaGetLastError();
        return ITM_ERR_CUDA;
    }
    d.swap_state = state;
    d.touch = touch;
    d.swap_frame = 0;
    sc->host_sdf = hs;
    sc->host_w = hw;
    sc->swap_scratch = scratch;
    sc->swap_k = transfer_blocks;
    sc->swap_idle = idle_frames;
    return ITM_OK;
}

int itm_swap_in(itm_scene *sc, itm_stream stream)
{
    Range range_("itm_swap_in");
    if (!sc || !sc->d.swap_state) return ITM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    const SwapDev w = swap_dev(sc);
    cudaError_t e = launch_select<false>(sc->d, w, st);
    if (e != cudaSuccess) return check_cuda(e);
    if (sc->d.weight_mode == 0)
        swap_in_kernel<0><<<move_grid(w.k), kMoveThreads, 0, st>>>(sc->d, w);
    else
        swap_in_kernel<1><<<move_grid(w.k), kMoveThreads, 0, st>>>(sc->d, w);
    return check_cuda(cudaGetLastError());
}

int itm_swap_out(itm_scene *sc, itm_stream stream)
{
    Range range_("itm_swap_out");
    if (!sc || !sc->d.swap_state) return ITM_ERR_ARG;
    sc->vis_ok = false;  // blocks are freed: the visible list's interior flags lapse
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    const SwapDev w = swap_dev(sc);
    cudaError_t e = launch_select<true>(sc->d, w, st);
    if (e != cudaSuccess) return check_cuda(e);
    if (sc->d.weight_mode == 0)
        swap_out_kernel<0><<<move_grid(w.k), kMoveThreads, 0, st>>>(sc->d, w);
    else
        swap_out_kernel<1><<<move_grid(w.k), kMoveThreads, 0, st>>>(sc->d, w);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = std::max(1, std::min(2 * sms, (sc->d.nv + 255) / 256));
    swap_compact_find_kernel<<<g, 256, 0, st>>>(sc->d, w);
    swap_compact_pair_kernel<<<std::max(1, std::min(g, (w.k + 255) / 256)), 256, 0, st>>>(sc->d, w);
    return check_cuda(cudaGetLastError());
}

int itm_swap_get_counters(itm_scene *sc, itm_swap_counters *out)
{
    if (!sc || !out || !sc->d.swap_state) return ITM_ERR_ARG;
    const size_t slots = (size_t)sc->d.nb + (size_t)sc->d.ne;
    std::vector<uint8_t> st(slots);
    unsigned long long moved[2] = {0, 0};
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), sc->d.swap_state, slots, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(moved, sc->swap_scratch, sizeof(moved), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    int64_t host = 0, waiting = 0;
    for (uint8_t v : st) {
        host += v == kSwHost;
        waiting += v == kSwMerge;
    }
    out->host_data = host + waiting;
    out->swapped_out = host;
    out->waiting = waiting;
    out->moved_in = (int64_t)moved[0];
    out->moved_out = (int64_t)moved[1];
    return ITM_OK;
}

int itm_swap_export_host(itm_scene *sc, int16_t *coords_host, float *sdf_host, void *w_host, int32_t *state_host,
                         int cap, int *n)
{
    if (!sc || !n || cap < 0 || !sc->d.swap_state) return ITM_ERR_ARG;
    if (cap > 0 && (!coords_host || !sdf_host || !w_host || !state_host)) return ITM_ERR_ARG;
    const size_t slots = (size_t)sc->d.nb + (size_t)sc->d.ne;
    std::vector<uint8_t> st(slots);
    std::vector<Entry> E(slots);
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), sc->d.swap_state, slots, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(E.data(), sc->d.entries, slots * sizeof(Entry), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    const size_t wbytes = sc->d.weight_mode == 0 ? 1 : 4;
    const float *hs = static_cast<const float *>(sc->host_sdf);
    const unsigned char *hw = static_cast<const unsigned char *>(sc->host_w);
    int count = 0;
    for (size_t i = 0; i < slots; ++i) {
        if (st[i] == kSwDevice) continue;
        if (count < cap) {
            coords_host[3 * count] = E[i].x;
            coords_host[3 * count + 1] = E[i].y;
            coords_host[3 * count + 2] = E[i].z;
            memcpy(sdf_host + (size_t)count * kBlockVoxels, hs + i * kBlockVoxels, kBlockVoxels * sizeof(float));
            memcpy(static_cast<unsigned char *>(w_host) + (size_t)count * kBlockVoxels * wbytes,
                   hw + i * kBlockVoxels * wbytes, kBlockVoxels * wbytes);
            state_host[count] = st[i];
        }
        ++count;
    }
    *n = count;
    if (cap == 0 && !coords_host) return ITM_OK;  // count query
    return count > cap ? ITM_ERR_TOO_LARGE : ITM_OK;
}

}  // extern "C"

namespace itm {

// Frees the swap state of a scene (itm_scene_destroy) and clears it for a
// reset (itm_scene_reset: every entry back to kSwDevice, counters 0).
void swap_free(itm_scene *sc)
{
    if (sc->d.swap_state) cudaFree(sc->d.swap_state);
    if (sc->d.touch) cudaFree(sc->d.touch);
    if (sc->swap_scratch) cudaFree(sc->swap_scratch);
    if (sc->host_sdf) cudaFreeHost(sc->host_sdf);
    if (sc->host_w) cudaFreeHost(sc->host_w);
    sc->d.swap_state = nullptr;
    sc->d.touch = nullptr;
    sc->swap_scratch = sc->host_sdf = sc->host_w = nullptr;
}

cudaError_t swap_reset(itm_scene *sc, cudaStream_t st)
{
    if (!sc->d.swap_state) return cudaSuccess;
    sc->d.swap_frame = 0;
    cudaError_t e = cudaMemsetAsync(sc->d.swap_state, 0, (size_t)sc->d.nb + (size_t)sc->d.ne, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(sc->d.touch, 0, sizeof(int32_t) * (size_t)(sc->d.nv > 0 ? sc->d.nv : 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->swap_scratch, 0, scratch_bytes(sc->d.nb, sc->swap_k), st);
    return e;
}

}  // namespace itm
