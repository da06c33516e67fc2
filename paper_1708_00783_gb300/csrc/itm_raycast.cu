// Sec. 4.4 raycast: one thread per pixel, a warp covering an 8x4 pixel tile.
//
// The march is the state machine of Sec. 4.4 (SEARCH_BLOCK_COARSE ->
// SEARCH_BLOCK_FINE -> SEARCH_SURFACE -> BEHIND_SURFACE, or WRONG_SIDE), with
// these step rules (the paper names the states, not the constants):
//   ray o + t dir, dir = R ((u-cx)/fx, (v-cy)/fy, 1): t is z-depth;
//   len = |((u-cx)/fx, (v-cy)/fy, 1)|, tB = 8s/len, tmu = mu/len, ts = s/len;
//   t starts at z_min; the ray misses when t > z_max or after
//   4 (z_max - z_min)/s + 64 iterations;
//   "the block at p" is the block of the nearest voxel floor(p/s + 1/2);
//   COARSE : unallocated -> t += tB; allocated -> t -= tB, FINE;
//   FINE   : unallocated -> t += tmu; allocated -> F (trilinear) <= 0 ->
//            WRONG_SIDE, else SURFACE at the same t;
//   SURFACE: unallocated -> COARSE; F <= 0 -> BEHIND; else
//            t += max(F tmu, ts);
//   BEHIND : twice t += F(t) tmu (trilinear), hit = o + t dir.
// The TSDF field outside allocated blocks is the default voxel value 1
// (Sec. 3.3 retrieval of a missing block).  Normals: central differences of
// the trilinear field at +-1 voxel per axis, emitted only when all 48 voxels
// read are allocated and observed (weight > 0).
//
// Search range (Sec. 4.4, second half): before the march, every allocated
// block is projected into the image and each 8x4-pixel tile (the pixels of
// one warp) records the nearest and farthest camera depth of the blocks that
// cover it.  A block's extent here is its query region -- the points whose
// nearest voxel lies in it, [8b - 1/2, 8b + 15/2] voxels per axis -- clipped
// to z >= z_min, grown by a small margin.  The march uses the range without
// changing its result: coarse steps in front of the tile's nearest depth are
// replayed as additions (no hash probes, the same t sequence and iteration
// count), and a ray in COARSE or FINE beyond the tile's farthest depth can
// only miss.  The paper renders 16x16-pixel fragments with per-pixel atomic
// min/max; here the fragment is the warp's tile and the atomics go to one
// word per tile.
//
// The per-iteration "is the block at p allocated" query goes through a
// one-entry cache per lane (the last block the lane looked up); on a miss the
// lane walks the hash chain itself (Sec. 3.3), lanes that read the same entry
// sharing the load.  (A warp-cooperative query -- lanes grouped by block with
// __match_any_sync, one walk per group, answers by shuffle -- measured slower:
// few warp iterations have every lane on its cached block.)  Every arithmetic
// step of the march uses IEEE round-to-nearest operations in a fixed order.
#include "itm_ops.cuh"

namespace itm {

namespace {

// One warp takes 32 allocated blocks and rasterises their tile rectangles.
__global__ void __launch_bounds__(256) range_kernel(SceneDev s, Mat34 M, Intr in, float zc, int tiles_x,
                                                    int tiles_y, uint32_t *__restrict__ rmin,
                                                    uint32_t *__restrict__ rmax)
{
    const int n = min(__ldcg(&s.ctr->block_head), s.nv);
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n; base += warps * 32) {
        const int i = base + lane;
        TileRange r{0, -1, 0, -1, 0.f, 0.f};
        bool ok = false;
        if (i < n) {
            const int ptr = __ldg(&s.block_free[i]);
            const short4 b = __ldg(&s.block_pos[ptr]);
            if (b.w) ok = block_tile_range(b, M, in, s.voxel_size, zc, tiles_x, tiles_y, r);
        }
        range_rasterize(ok, r, tiles_x, rmin, rmax);
    }
}

// Persistent raycast, first phase (the march): each warp takes the next 8x4
// tile from a device counter until none is left, so warps that finish early
// pick up more work instead of idling behind the slowest tiles of a fixed
// grid.  raycast_finish_kernel then refines the hits and takes their normals
// (two kernels with smaller code each measured faster than the one that did
// both).  With use_order the tiles
// are handed out from the queues of the previous raycast, heaviest cost class
// first (longest processing time first), so the expensive tiles do not start
// last.  With write_order each finished tile is appended to the queue of its
// cost class for the next raycast.  hdr_w[0] is this raycast's tile counter.
template <int MODE>
__global__ void __launch_bounds__(256, 4) raycast_dynamic_kernel(SceneDev s, Intr in, Mat34 T, float4 *__restrict__ vtx,
                                                              float4 *__restrict__ nrm, int max_iter, float tB_m,
                                                              float inv_sv, const uint32_t *__restrict__ rmin,
                                                              const uint32_t *__restrict__ rmax, int tiles_x,
                                                              int n_tiles, int32_t *__restrict__ hdr_w,
                                                              int32_t *__restrict__ list_w,
                                                              const int32_t *__restrict__ hdr_r,
                                                              const int32_t *__restrict__ list_r, bool use_order,
                                                              bool write_order)
{
    // first position of each class slot k (class kTileClasses - 1 - k)
    __shared__ int first[kTileClasses + 1];
    const int lane = threadIdx.x & 31;
    grid_dep_wait();
    if (use_order) {
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int k = 0; k < kTileClasses; ++k) {
                first[k] = acc;
                acc += __ldg(&hdr_r[1 + kTileClasses - 1 - k]);
            }
            first[kTileClasses] = acc;
        }
        __syncthreads();
        // queues that do not hold every tile once (cannot happen when the
        // previous raycast covered the same tiles) fall back to raster order
        use_order = first[kTileClasses] == n_tiles;
    }
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&hdr_w[0], 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_tiles) {
            grid_dep_launch();
            return;
        }
        int tile = t;
        if (use_order) {
            int k = 0;
            while (k < kTileClasses - 1 && first[k + 1] <= t) ++k;
            tile = __ldg(&list_r[(size_t)(kTileClasses - 1 - k) * kOrderMaxTiles + (t - first[k])]);
            if ((unsigned)tile >= (unsigned)n_tiles) tile = t;
        }
        const int cost = raycast_warp_tile<MODE, true, 1>(s, in, T, vtx, nrm, max_iter, tB_m, inv_sv, rmin, rmax,
                                                          tiles_x, tile % tiles_x, tile / tiles_x);
        if (write_order && lane == 0) {
            const int c = min(cost >> 3, kTileClasses - 1);
            const int p = atomicAdd(&hdr_w[1 + c], 1);
            list_w[(size_t)c * kOrderMaxTiles + p] = tile;
        }
    }
}

// second phase of the split raycast: refinement, hit point and normal of the
// pixels whose march (raycast_dynamic_kernel) ended behind the surface.
// hdr_clear (or null): the tile-queue header the march read, cleared for the
// next raycast, which writes that side (so it needs no clearing launch).
template <int MODE>
__global__ void __launch_bounds__(256, 4) raycast_finish_kernel(SceneDev s, Intr in, Mat34 T, float4 *__restrict__ vtx,
                                                             float4 *__restrict__ nrm, int max_iter, float tB_m,
                                                             float inv_sv, int32_t *__restrict__ hdr_clear)
{
    grid_dep_wait();
    if (hdr_clear && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < kTileHdrInts) hdr_clear[threadIdx.x] = 0;
    const int warp = threadIdx.x >> 5;
    const int tix = blockIdx.x * 4 + (warp & 3), tiy = blockIdx.y * 2 + (warp >> 2);
    if (tix >= (in.W + 7) / 8 || tiy >= (in.H + 3) / 4) return;
    raycast_warp_tile<MODE, false, 2>(s, in, T, vtx, nrm, max_iter, tB_m, inv_sv, nullptr, nullptr, 0, tix, tiy);
}

template <int MODE, bool RANGE>
__global__ void __launch_bounds__(256) raycast_kernel(SceneDev s, Intr in, Mat34 T, float4 *__restrict__ vtx,
                                                      float4 *__restrict__ nrm, int max_iter, float tB_m,
                                                      float inv_sv, const uint32_t *__restrict__ rmin,
                                                      const uint32_t *__restrict__ rmax, int tiles_x, int tiles_y)
{
    raycast_tile<MODE, RANGE>(s, in, T, vtx, nrm, max_iter, tB_m, inv_sv, rmin, rmax, tiles_x, tiles_y, blockIdx.x,
                              blockIdx.y);
}

int range_grid()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = sms * 4;
    }
    return g;
}

}  // namespace

bool range_fits(const Intr &in) { return in.W <= kRangeMaxW && in.H <= kRangeMaxH; }

cudaError_t launch_raycast_range(const SceneDev &s, const Intr &in, const Mat34 &M_d, uint32_t *rmin, uint32_t *rmax,
                                 cudaStream_t st)
{
    const int tx = (in.W + 7) / 8, ty = (in.H + 3) / 4;
    cudaError_t e = cudaMemsetAsync(rmin, 0xff, sizeof(uint32_t) * (size_t)tx * ty, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rmax, 0, sizeof(uint32_t) * (size_t)tx * ty, st);
    if (e != cudaSuccess) return e;
    const float zc = s.z_min - 1e-3f;
    range_kernel<<<range_grid(), 256, 0, st>>>(s, M_d, in, zc, tx, ty, rmin, rmax);
    return cudaGetLastError();
}

cudaError_t launch_raycast(const SceneDev &s, const Intr &in, const Mat34 &T_wc, const Mat34 &M_d, float4 *vtx,
                           float4 *nrm, bool range_ready, int order_dims[2], int &order_side, cudaStream_t st)
{
    // host-side constants with the same float operations as the oracle
    volatile float span = s.z_max - s.z_min;
    volatile float four_span = 4.0f * span;
    volatile float ratio = four_span / s.voxel_size;
    const int max_iter = (int)ratio + 64;
    volatile float tB_m = 8.0f * s.voxel_size;
    const float inv_sv = (float)(1.0 / (double)s.voxel_size);  // voxel coordinates: p * (1/s), 1/s rounded once
    dim3 grid((in.W + 31) / 32, (in.H + 7) / 8);
    const int tx = (in.W + 7) / 8, ty = (in.H + 3) / 4;
    if (range_fits(in)) {
        // the allocation of this frame may have filled the range already
        cudaError_t e = range_ready ? cudaSuccess : launch_raycast_range(s, in, M_d, s.range_min, s.range_max, st);
        // bit 1 of order_side: the header of side order_side & 1 is already
        // clear (the previous raycast's finish kernel cleared it); it is
        // dropped first, so that a launch error below leaves it unset
        const int w = order_side & 1;
        const bool pre_cleared = (order_side & 2) != 0;
        order_side = w;
        int32_t *hdr_w = s.tile_q_hdr + w * kTileHdrInts, *list_w = s.tile_q_list + (size_t)w * kTileClasses * kOrderMaxTiles;
        const int32_t *hdr_r = s.tile_q_hdr + (1 - w) * kTileHdrInts;
        const int32_t *list_r = s.tile_q_list + (size_t)(1 - w) * kTileClasses * kOrderMaxTiles;
        if (e == cudaSuccess && !pre_cleared) e = launch_pdl(zero_words_kernel, dim3(1), dim3(32), 0, st, hdr_w, kTileHdrInts);
        if (e != cudaSuccess) return e;
        static int g_dyn[2] = {0, 0};
        const int mode = s.weight_mode ? 1 : 0;
        if (!g_dyn[mode]) {
            int dev = 0, sms = 1, per = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per, mode ? (const void *)raycast_dynamic_kernel<1> : (const void *)raycast_dynamic_kernel<0>, 256, 0);
            g_dyn[mode] = sms * (per > 0 ? per : 1);
        }
        const int n_tiles = tx * ty;
        const int g = g_dyn[mode] < (n_tiles + 7) / 8 ? g_dyn[mode] : (n_tiles + 7) / 8;
        const bool write_order = n_tiles <= kOrderMaxTiles;
        const bool use_order = write_order && order_dims[0] == tx && order_dims[1] == ty;
        const float tBm = tB_m;
        if (mode == 0)
            e = launch_pdl(raycast_dynamic_kernel<0>, dim3(g), dim3(256), 0, st, s, in, T_wc, vtx, nrm, max_iter, tBm,
                           inv_sv, (const uint32_t *)s.range_min, (const uint32_t *)s.range_max, tx, n_tiles, hdr_w,
                           list_w, hdr_r, list_r, use_order, write_order);
        else
            e = launch_pdl(raycast_dynamic_kernel<1>, dim3(g), dim3(256), 0, st, s, in, T_wc, vtx, nrm, max_iter, tBm,
                           inv_sv, (const uint32_t *)s.range_min, (const uint32_t *)s.range_max, tx, n_tiles, hdr_w,
                           list_w, hdr_r, list_r, use_order, write_order);
        if (e != cudaSuccess) return e;
        // with write_order the next raycast writes side 1 - w, which this
        // one only read: the finish kernel clears its header
        int32_t *hdr_clear = write_order ? s.tile_q_hdr + (1 - w) * kTileHdrInts : nullptr;
        if (mode == 0)
            e = launch_pdl(raycast_finish_kernel<0>, grid, dim3(256), 0, st, s, in, T_wc, vtx, nrm, max_iter, tBm, inv_sv,
                           hdr_clear);
        else
            e = launch_pdl(raycast_finish_kernel<1>, grid, dim3(256), 0, st, s, in, T_wc, vtx, nrm, max_iter, tBm, inv_sv,
                           hdr_clear);
        if (e != cudaSuccess) return e;
        if (write_order) {
            order_dims[0] = tx;
            order_dims[1] = ty;
            order_side = (1 - w) | 2;
        }
        return cudaSuccess;
    } else {
        if (s.weight_mode == 0)
            raycast_kernel<0, false><<<grid, 256, 0, st>>>(s, in, T_wc, vtx, nrm, max_iter, tB_m, inv_sv, nullptr,
                                                           nullptr, tx, ty);
        else
            raycast_kernel<1, false><<<grid, 256, 0, st>>>(s, in, T_wc, vtx, nrm, max_iter, tB_m, inv_sv, nullptr,
                                                           nullptr, tx, ty);
    }
    return cudaGetLastError();
}

// Parts' raycasts of a split scene merged per pixel: the hit nearest to the
// camera (camera depth = row 2 of M_d applied to the vertex, each operation
// rounded on its own), equal depths to the lower part; no hit: zeros.
__global__ void __launch_bounds__(256) merge_kernel(const float4 *__restrict__ vtx, const float4 *__restrict__ nrm,
                                                    int parts, long long npix, Mat34 M, float4 *__restrict__ vo,
                                                    float4 *__restrict__ no)
{
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < npix;
         o += (long long)gridDim.x * blockDim.x) {
        int best = -1;
        float best_z = 0.0f;
        for (int k = 0; k < parts; ++k) {
            const float4 V = __ldg(&vtx[(size_t)k * npix + o]);
            if (!(V.w > 0.0f)) continue;
            const float z = row_apply(&M.m[8], V.x, V.y, V.z);
            if (best < 0 || z < best_z) {
                best = k;
                best_z = z;
            }
        }
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        vo[o] = best < 0 ? zero : __ldg(&vtx[(size_t)best * npix + o]);
        no[o] = best < 0 ? zero : __ldg(&nrm[(size_t)best * npix + o]);
    }
}

cudaError_t launch_raycast_merge(const float4 *vtx, const float4 *nrm, int parts, long long npix, const Mat34 &M_d,
                                 float4 *vo, float4 *no, cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    const long long blocks = (npix + 255) / 256;
    merge_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(vtx, nrm, parts, npix, M_d, vo, no);
    return cudaGetLastError();
}

}  // namespace itm
