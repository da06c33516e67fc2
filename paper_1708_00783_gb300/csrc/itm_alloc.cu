// Sec. 4.2 allocation on the GPU, in three launches per frame:
//
//  1. alloc_enumerate  one thread per pixel walks the blocks crossed by its
//     segment d-mu .. d+mu (3D DDA).  The 32 lanes of a warp cover an 8x4
//     pixel tile, so neighbouring rays emit mostly the same blocks: each step,
//     __match_any_sync groups equal block keys and only one lane per group
//     probes the hash.  A missing block claims its bucket's request word with
//     one 64-bit CAS (the paper's per-entry allocation array, Sec. 4.2); the
//     winner of a bucket appends the bucket to the request list, a block that
//     finds its bucket claimed by another key goes to the overflow list
//     (warp-aggregated appends, one atomic per warp).
//  2. alloc_commit     one thread per requested bucket inserts its key
//     (Sec. 3.3 insertion).  Each bucket's chain has exactly one writer, so
//     chains are extended without locks; blocks and excess slots come from
//     prepopulated free lists through warp-aggregated atomic counters (the
//     paper's "atomic subtraction on a stack").  The CTA that finishes last
//     then resolves the overflow list in rounds: look up, claim the bucket,
//     let winners insert, repeat with the losers.  The paper leaves such
//     intra-frame collisions for the next frame; resolving them makes the
//     allocated set the complete union over all pixels.
//  3. build_visible    every allocated block whose voxels can project into the
//     image with z > 0 and lie within the frame's depth range + mu is
//     appended to the visible list (Sec. 4.2, third part); eight lanes per
//     block, one per corner.  When the raycast will use the allocation pose,
//     the same pass also rasterises each block's search range.
//
// Counts produced on the device are read by the next kernel from device
// memory (persistent grid-stride loops), so no host synchronisation and no
// allocation happen per frame.
#include "itm_ops.cuh"

namespace itm {

namespace {

// Also clears the search-range tiles of this frame (n_range_tiles of them;
// nothing reads them before the visible-list pass).
__global__ void __launch_bounds__(256) alloc_enumerate_kernel(SceneDev s, const float *__restrict__ depth,
                                                              Intr in, Mat34 T, float inv_b, int n_range_tiles,
                                                              const uint16_t *__restrict__ raw,
                                                              float *__restrict__ depth_out)
{
    const int cta = blockIdx.y * gridDim.x + blockIdx.x, ctas = gridDim.x * gridDim.y;
    grid_dep_wait();  // the previous raycast may still read the range tiles
    for (int i = cta * blockDim.x + threadIdx.x; i < n_range_tiles; i += ctas * blockDim.x) {
        s.range_min[i] = 0xffffffffu;
        s.range_max[i] = 0u;
    }
    enumerate_tile(s, depth, in, T, inv_b, blockIdx.x, blockIdx.y, raw, depth_out);
    grid_dep_launch();
}

// The last CTA to finish its requests then resolves the overflow list (its
// inserts are visible through the fences before the completion count).
__global__ void __launch_bounds__(256) alloc_commit_kernel(SceneDev s)
{
    __shared__ int is_last, remaining;
    grid_dep_wait();
    const int n = min(__ldcg(&s.ctr->n_req), s.nb);
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int i = i0 + threadIdx.x;
        if (i < n) commit_request(s, i);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&s.ctr->commit_done, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (is_last) {
        __threadfence();
        overflow_scene(s, remaining);
    }
    grid_dep_launch();
}

__global__ void __launch_bounds__(256) build_visible_kernel(SceneDev s, Mat34 M, Intr in)
{
    grid_dep_wait();
    const int n = min(__ldcg(&s.ctr->block_head), s.nv);
    const float zfar = visible_zfar(s);
    const int groups = gridDim.x * (blockDim.x >> 3);
    for (int g0 = blockIdx.x * (blockDim.x >> 3); g0 < n; g0 += groups) {
        const int i = g0 + (threadIdx.x >> 3);
        visible_8<false>(s, M, in, zfar, i < n, i, 0.0f, 1, 1);
    }
    grid_dep_launch();
}

// The same, also filling the search range of a raycast from this pose (the
// loop is uniform per CTA so every warp reaches the rasterisation together).
__global__ void __launch_bounds__(256) build_visible_range_kernel(SceneDev s, Mat34 M, Intr in, float zc,
                                                                  int tiles_x, int tiles_y)
{
    grid_dep_wait();
    const int n = min(__ldcg(&s.ctr->block_head), s.nv);
    const float zfar = visible_zfar(s);
    const int groups = gridDim.x * (blockDim.x >> 3);
    for (int g0 = blockIdx.x * (blockDim.x >> 3); g0 < n; g0 += groups) {
        const int i = g0 + (threadIdx.x >> 3);
        visible_8<true>(s, M, in, zfar, i < n, i, zc, tiles_x, tiles_y);
    }
    grid_dep_launch();
}

int sm_count()
{
    static int cached_sm = 0;
    if (!cached_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached_sm, cudaDevAttrMultiProcessorCount, dev);
        if (cached_sm <= 0) cached_sm = 1;
    }
    return cached_sm;
}

int persistent_grid(int threads, const void *kernel)
{
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm < 1) per_sm = 1;
    return sm_count() * per_sm;
}

}  // namespace

cudaError_t launch_allocate(const SceneDev &s, const float *depth, const Intr &in, const Mat34 &T_wc,
                            const Mat34 &M_d, bool with_range, cudaStream_t st, const uint16_t *raw)
{
    static_assert(kFrameCountersOffset % 4 == 0 && kFrameCountersBytes % 4 == 0, "word-aligned frame counters");
    cudaError_t e = launch_pdl(zero_words_kernel, dim3(1), dim3(32), 0, st,
                               reinterpret_cast<int32_t *>(reinterpret_cast<char *>(s.ctr) + kFrameCountersOffset),
                               (int)(kFrameCountersBytes / 4));
    if (e != cudaSuccess) return e;
    const float inv_b = (float)(1.0 / (8.0 * (double)s.voxel_size));
    dim3 grid((in.W + 31) / 32, (in.H + 7) / 8);
    const int n_range_tiles = with_range ? ((in.W + 7) / 8) * ((in.H + 3) / 4) : 0;
    // with raw, depth is the output of the frame's conversion
    e = launch_pdl(alloc_enumerate_kernel, grid, dim3(256), 0, st, s, raw ? nullptr : depth, in, T_wc, inv_b,
                   n_range_tiles, raw, raw ? const_cast<float *>(depth) : nullptr);
    if (e != cudaSuccess) return e;
    static int g_commit = 0, g_visible = 0, g_visrange = 0;
    // one CTA per SM: a frame's requests (usually a few thousand) fit in one
    // pass, and fewer CTAs pay the completion count's fences
    if (!g_commit) g_commit = sm_count();
    if (!g_visible) g_visible = persistent_grid(256, (const void *)build_visible_kernel);
    if (!g_visrange) g_visrange = persistent_grid(256, (const void *)build_visible_range_kernel);
    e = launch_pdl(alloc_commit_kernel, dim3(g_commit), dim3(256), 0, st, s);
    if (e != cudaSuccess) return e;
    if (with_range) {
        const int tx = (in.W + 7) / 8, ty = (in.H + 3) / 4;
        e = launch_pdl(build_visible_range_kernel, dim3(g_visrange), dim3(256), 0, st, s, M_d, in, s.z_min - 1e-3f,
                       tx, ty);
    } else {
        e = launch_pdl(build_visible_kernel, dim3(g_visible), dim3(256), 0, st, s, M_d, in);
    }
    return e;
}

int overflow_capacity() { return kOvfCapacity; }

}  // namespace itm
