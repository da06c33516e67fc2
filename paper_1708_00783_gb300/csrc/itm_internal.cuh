// Internal definitions shared by the CUDA translation units of libitm.
//
// Device layout of one scene (all arrays allocated once by itm_scene_create):
//   entries     Entry[nb + ne]      16 B each; buckets then excess entries (Sec. 3.2)
//   req         uint64[nb]          per-bucket allocation request (packed key, 0 = none)
//   req_list    int32[nb]           buckets that received a request this frame
//   overflow    uint64[ovf_cap]     requests that lost their bucket to another key
//   visible     int32[nv]           visible block indices of the current frame
//   block_pos   short4[nv]          coordinates of the block held at each index (w = 1 in use)
//   sdf         float[nv][512]      TSDF, voxel index x + 8y + 64z (Sec. 3.1)
//   w8 / w32    uint8 / float [nv][512]  weights (constant / learned observation weight)
//   block_free  int32[nv]           free block list, handed out front to back
//   excess_free int32[ne]           free excess slots, handed out front to back
//   ctr         Counters            device counters and the sticky status word
//   swap_state  uint8[nb + ne]      Sec. 5 swapping (itm_swap_enable): kSw* per entry
//   touch       int32[nv]           last allocation whose segments met the block (-1: freed
//                                   by the running swap-out)
//   rgbw        uint32[nv][512]     colour voxels (itm_colour_enable): bytes r, g, b, colour weight
//   host store  pinned host memory mapped into the device, one slot per entry:
//               float[nb + ne][512] sdf and uint8 / float [nb + ne][512] weights
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "itm.h"

namespace itm {

constexpr int kBlockVoxels = 512;
// largest image whose raycast uses the search-range tiles (8x4 pixels each)
constexpr int kRangeMaxW = 4096, kRangeMaxH = 4096;
constexpr int kRangeMaxTiles = (kRangeMaxW / 8) * (kRangeMaxH / 4);
// Raycast tiles are handed out by cost class (march iterations / 8, heaviest
// first) as measured by the previous raycast, for images of at most
// kOrderMaxTiles tiles.
constexpr int kOrderMaxTiles = 1 << 16;
constexpr int kTileClasses = 16;
constexpr int kTileHdrInts = 32;  // per side: next, counts[kTileClasses], padding
constexpr int kCombinedMax = ITM_COMBINED_MAX;
constexpr int kIcpSums = ITM_ICP_SUMS;
constexpr int kIcpWorkDoubles = ITM_ICP_WORK_DOUBLES;
constexpr int kIcpMaxPartials = ITM_ICP_WORK_DOUBLES / ITM_ICP_SUMS - 1;
constexpr int kTrackMaxLevels = ITM_TRACK_MAX_LEVELS;
constexpr unsigned kFull = 0xffffffffu;

// Sec. 5 swap state of a hash entry
constexpr uint8_t kSwDevice = 0;  // current data in the device block (or none)
constexpr uint8_t kSwHost = 1;    // swapped out: data in the host slot only, entry ptr -1
constexpr uint8_t kSwMerge = 2;   // host data waiting to be fused into the device block

// Sec. 3.2 hash entry.  Bytes 0..7 (x, y, z, flag) form the packed block key
// compared and claimed as one 64-bit word; flag = 1 marks an entry that holds
// a block, so the all-zero word means "never used".
struct __align__(16) Entry {
    int16_t x, y, z, flag;
    int32_t offset;  // 0: end of chain; k >= 1: next entry at nb + k - 1 (Sec. 3.3)
    int32_t ptr;     // >= 0 block index; -1 swapped out; < -1 unallocated (Sec. 3.2)
};

struct Counters {
    uint32_t status;
    int32_t block_head;     // blocks handed out (may run past nv when the array is full)
    int32_t excess_head;    // excess slots handed out
    int32_t n_req;          // per-frame: buckets requested
    int32_t n_overflow;     // per-frame: requests that lost their bucket
    int32_t n_visible;      // per-frame: visible blocks
    int32_t depth_max_bits; // per-frame: largest valid depth (float bits, >= 0)
    int32_t commit_done;    // per-frame: CTAs of the commit kernel that finished
    unsigned long long updated;  // cumulative voxel updates
    unsigned long long visited;  // cumulative voxels visited by integration
    unsigned long long frames;   // cumulative integrated frames
    unsigned long long mesh_tris;  // per-mesh: triangles found
};

// Offset and size of the per-frame counters cleared at the start of allocation.
constexpr size_t kFrameCountersOffset = 12;  // n_req
constexpr size_t kFrameCountersBytes = 20;   // n_req .. commit_done


struct SceneDev {
    Entry *entries;
    unsigned long long *req;
    int32_t *req_list;
    unsigned long long *overflow;
    int32_t *visible;
    short4 *block_pos;
    float *sdf;
    uint8_t *w8;
    float *w32;
    int32_t *block_free;
    int32_t *excess_free;
    Counters *ctr;
    uint32_t *range_min;  // per 8x4 tile: nearest / farthest depth (float bits) of covering blocks
    uint32_t *range_max;
    // raycast tile queues, two sides (one written by a raycast, the other
    // read): per side a header {next tile, count of each cost class} and per
    // class a list of up to kOrderMaxTiles tiles
    int32_t *tile_q_hdr;
    int32_t *tile_q_list;
    // Sec. 5 swapping: null while swapping is off
    uint8_t *swap_state;
    int32_t *touch;
    int swap_frame;  // allocations since swapping was enabled
    uint32_t *rgbw;  // colour voxels (Sec. 3.1): null while colour is off
    int nb, ne, nv;
    int ovf_cap;
    float voxel_size, mu, z_min, z_max;
    float inv_mu;  // RN(1 / mu)
    int max_w, weight_mode;
    // one part of a scene split by slabs of block columns (itm_scene_set_shard);
    // shard_n <= 1: the whole scene
    int shard_n, shard_i, shard_w;
};

struct Intr {
    int W, H;
    float fx, fy, cx, cy;
};

// Rows 0..2 of a 4x4 rigid transform, row-major.
struct Mat34 {
    float m[12];
};

// ---------------------------------------------------------------- hashing

// Sec. 3.2 hashIndex: unsigned coordinates times three primes, xor, mask.
__host__ __device__ __forceinline__ uint32_t hash_bucket(int x, int y, int z, uint32_t mask)
{
    return (((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349669u) ^ ((uint32_t)z * 83492791u)) & mask;
}

__host__ __device__ __forceinline__ unsigned long long pack_key(int x, int y, int z)
{
    return (unsigned long long)(uint16_t)x | ((unsigned long long)(uint16_t)y << 16) |
           ((unsigned long long)(uint16_t)z << 32) | (1ull << 48);
}

__device__ __forceinline__ void unpack_key(unsigned long long k, int &x, int &y, int &z)
{
    x = (int)(int16_t)(k & 0xffff);
    y = (int)(int16_t)((k >> 16) & 0xffff);
    z = (int)(int16_t)((k >> 32) & 0xffff);
}

__device__ __forceinline__ unsigned long long entry_key(const int4 &e)
{
    return (unsigned long long)(uint32_t)e.x | ((unsigned long long)(uint32_t)e.y << 32);
}

// Sec. 3.3 retrieval through the read-only path (tables not modified by the
// running kernel).  Returns the block index or -1.
__device__ __forceinline__ void set_status(const SceneDev &s, uint32_t bits)
{
    atomicOr(&s.ctr->status, bits);
}

// Builds with -DITM_CHECK_BOUNDS check the indices into the hash table, the
// voxel block array, the depth image and the per-frame lists before the
// access; a failed check sets ITM_ST_BOUNDS and the access is skipped.  In
// normal builds the checks compile to nothing.
#ifdef ITM_CHECK_BOUNDS
#define ITM_IN_BOUNDS(s, cond) ((cond) ? true : (set_status((s), ITM_ST_BOUNDS), false))
#else
#define ITM_IN_BOUNDS(s, cond) true
#endif

__device__ __forceinline__ int lookup_ro(const SceneDev &s, int bx, int by, int bz)
{
    const unsigned long long key = pack_key(bx, by, bz);
    int idx = (int)hash_bucket(bx, by, bz, (uint32_t)(s.nb - 1));
    const int4 *E = reinterpret_cast<const int4 *>(s.entries);
    for (int guard = 0; guard <= s.ne; ++guard) {
        int4 e = __ldg(&E[idx]);
        if (entry_key(e) == key && e.w >= 0) return ITM_IN_BOUNDS(s, e.w < s.nv) ? e.w : -1;
        if (e.z < 1) return -1;
        if (!ITM_IN_BOUNDS(s, e.z - 1 < s.ne)) return -1;
        idx = s.nb + e.z - 1;
    }
    return -1;
}

// Same, through L2 (coherent with writes made earlier by the same kernel).
__device__ __forceinline__ int lookup_cg(const SceneDev &s, int bx, int by, int bz)
{
    const unsigned long long key = pack_key(bx, by, bz);
    int idx = (int)hash_bucket(bx, by, bz, (uint32_t)(s.nb - 1));
    const int4 *E = reinterpret_cast<const int4 *>(s.entries);
    for (int guard = 0; guard <= s.ne; ++guard) {
        int4 e = __ldcg(&E[idx]);
        if (entry_key(e) == key && e.w >= 0) return ITM_IN_BOUNDS(s, e.w < s.nv) ? e.w : -1;
        if (e.z < 1) return -1;
        if (!ITM_IN_BOUNDS(s, e.z - 1 < s.ne)) return -1;
        idx = s.nb + e.z - 1;
    }
    return -1;
}

// ------------------------------------------------------ slab partition
// Block column x belongs to part floor(x / w) mod n; a part keeps its own
// columns and kShardGhost columns on either side (whose voxels every sample
// around a point of its own columns reads), and reports only raycast hits in
// its own columns.
constexpr int kShardGhost = 1;

__host__ __device__ __forceinline__ int slab_owner(int bx, int n, int w)
{
    const int q = bx >= 0 ? bx / w : -((-bx + w - 1) / w);  // floor(bx / w)
    const int r = q % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ bool shard_keeps(const SceneDev &s, int bx)
{
    if (s.shard_n <= 1) return true;
    bool keep = false;
#pragma unroll
    for (int d = -kShardGhost; d <= kShardGhost; ++d) keep = keep || slab_owner(bx + d, s.shard_n, s.shard_w) == s.shard_i;
    return keep;
}

__device__ __forceinline__ bool shard_owns(const SceneDev &s, int bx)
{
    return s.shard_n <= 1 || slab_owner(bx, s.shard_n, s.shard_w) == s.shard_i;
}

// ------------------------------------------ programmatic dependent launch
// The per-frame kernels are launched with programmatic stream serialization
// (launch_pdl): a kernel may be scheduled while the kernel before it on the
// stream drains, runs only what touches no memory until grid_dep_wait()
// (which returns once the previous kernel has completed and its writes are
// visible), and calls grid_dep_launch() when its own main work is done so
// that the next kernel can be scheduled early.  Both are no-ops for a kernel
// launched the ordinary way.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

namespace {
// Zeroes n 32-bit words at p after the previous kernel (a launch_pdl stand-in
// for cudaMemsetAsync, which would break the chain of dependent launches).
__global__ void __launch_bounds__(32) zero_words_kernel(int32_t *p, int n)
{
    grid_dep_wait();
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
    grid_dep_launch();
}
}  // namespace

// ------------------------------------------------ IEEE round-to-nearest ops
// Every operation that decides an integer (which block, which pixel, whether
// a voxel is updated) is written with these so that no multiply-add is fused.
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// ((m0 x + m1 y) + m2 z) + m3, each operation rounded on its own.
__device__ __forceinline__ float row_apply(const float *m, float x, float y, float z)
{
    return fadd(fadd(fadd(fmul(m[0], x), fmul(m[1], y)), fmul(m[2], z)), m[3]);
}

// --------------------------------------------------------------- atomics


// Warp-aggregated append: the lanes active at the call each get a distinct
// slot of their counter; lanes naming the same counter share one atomic
// (lanes of one warp may work for different scenes in a batch).
__device__ __forceinline__ int warp_append(int32_t *counter)
{
    const unsigned active = __activemask();
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(active, (unsigned long long)counter);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(peers));
    base = __shfl_sync(active, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

}  // namespace itm

// Opaque handle behind the C ABI.
struct itm_scene {
    itm_scene_params params;
    itm::SceneDev d;
    cudaStream_t last_stream;
    int device;
    // the search-range tiles hold the range of a raycast from range_pose /
    // range_intr over the blocks allocated at epoch range_epoch
    long long alloc_epoch;
    long long range_epoch;
    float range_pose[16];
    itm_intrinsics range_intr;
    // the tile queues of side 1 - (order_side & 1) hold every tile of a
    // tiles_x x tiles_y image ({0, 0}: none yet); the next raycast writes side
    // order_side & 1, whose header is already clear when bit 1 is set
    int order_dims[2];
    int order_side;
    // the visible list's interior flags were computed for vis_pose /
    // vis_intr (vis_ok: by the last allocation, with no block moved or freed
    // since)
    bool vis_ok;
    float vis_pose[16];
    itm_intrinsics vis_intr;
    // Sec. 5 swapping (itm_swap_enable): the host store (pinned, mapped) and
    // the device scratch of the selection
    void *host_sdf, *host_w;
    void *swap_scratch;
    int swap_k, swap_idle;
    // weight mode 1: a second stream and fork / join events, so that
    // itm_process_frame_weighted runs the per-pixel weights beside the
    // allocation (made by itm_scene_create)
    cudaStream_t aux;
    cudaEvent_t ev_fork, ev_join;
};

// An NVTX range named after a C-ABI call for the duration of the call, so
// profiler timelines group each call's kernels (no cost without a profiler).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Host helpers implemented in itm_scene.cu.
namespace itm {
int check_cuda(cudaError_t e);
void pose_rows(const float T[16], Mat34 &out);        // rows 0..2 of T
void rigid_inverse_rows(const float T[16], Mat34 &out); // rows 0..2 of T^-1 (fp64, rounded once)
int valid_intr(const itm_intrinsics *in);
Intr to_intr(const itm_intrinsics *in);
// the visible list's interior flags hold for an integration with this pose
// and these intrinsics (launch_integrate's interior_ok)
bool interior_flags_hold(const itm_scene *sc, const float T_wc[16], const itm_intrinsics *intr);
}  // namespace itm

// Launchers implemented in the kernel translation units.
namespace itm {
cudaError_t launch_allocate(const SceneDev &s, const float *depth, const Intr &in, const Mat34 &T_wc,
                            const Mat34 &M_d, bool with_range, cudaStream_t st, const uint16_t *raw = nullptr);
// interior_ok: the visible list was built by an allocation with this pose and
// these intrinsics, and no block changed since, so its interior flags hold
cudaError_t launch_integrate(const SceneDev &s, const float *depth, const float *wpx, const Intr &in,
                             const Mat34 &M_d, bool interior_ok, cudaStream_t st);
cudaError_t launch_raycast(const SceneDev &s, const Intr &in, const Mat34 &T_wc, const Mat34 &M_d, float4 *vtx,
                           float4 *nrm, bool range_ready, int order_dims[2], int &order_side, cudaStream_t st);
cudaError_t launch_raycast_range(const SceneDev &s, const Intr &in, const Mat34 &M_d, uint32_t *rmin, uint32_t *rmax,
                                 cudaStream_t st);
bool range_fits(const Intr &in);
cudaError_t launch_mesh(const SceneDev &s, float *out, long long cap, unsigned long long *counter, cudaStream_t st);
// Sec. 5 swapping state of a scene: freed by itm_scene_destroy, cleared by
// itm_scene_reset (itm_swap.cu)
void swap_free(itm_scene *sc);
cudaError_t swap_reset(itm_scene *sc, cudaStream_t st);
cudaError_t launch_depth_halve(const float *in, int W, int H, float *out, cudaStream_t st);
cudaError_t launch_icp_reduce(const float *depth, const Intr &in, const Mat34 &T_g, const float4 *V, const float4 *N,
                              const Intr &ref, const Mat34 &M_ref, float dist_thresh, double *work, cudaStream_t st);
size_t track_scratch_bytes(int W, int H, int levels);
cudaError_t launch_track(const float *depth, const Intr &in0, int levels, const int *iters, const float *thresh,
                         const float4 *V, const float4 *N, const Intr &ref, const Mat34 &M_ref, float T[16],
                         int *steps, void *scratch, cudaStream_t st);
cudaError_t launch_raycast_combined(const SceneDev *subs, const Mat34 *P, int n, const Intr &in, const Mat34 &T_wc,
                                    float4 *vtx, float4 *nrm, cudaStream_t st);
cudaError_t launch_depth_u16(const uint16_t *raw, float *out, int64_t n, cudaStream_t st);
cudaError_t launch_raycast_merge(const float4 *vtx, const float4 *nrm, int parts, long long npix, const Mat34 &M_d,
                                 float4 *vo, float4 *no, cudaStream_t st);
cudaError_t launch_reset(const SceneDev &s, cudaStream_t st);
}  // namespace itm
