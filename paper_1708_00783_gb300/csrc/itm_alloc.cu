// Sec. 4.2 allocation on the GPU, in four launches per frame:
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
//     paper's "atomic subtraction on a stack").
//  3. alloc_overflow   one CTA resolves the overflow list in rounds: look up,
//     claim the bucket, let winners insert, repeat with the losers.  The
//     paper leaves such intra-frame collisions for the next frame; resolving
//     them makes the allocated set the complete union over all pixels.
//  4. build_visible    every allocated block whose voxels can project into the
//     image with z > 0 and lie within the frame's depth range + mu is
//     appended to the visible list (Sec. 4.2, third part).
//
// Counts produced on the device are read by the next kernel from device
// memory (persistent grid-stride loops), so no host synchronisation and no
// allocation happen per frame.
#include "itm_internal.cuh"

namespace itm {

namespace {

// ------------------------------------------------------------ 1. enumerate

__global__ void __launch_bounds__(256) alloc_enumerate_kernel(SceneDev s, const float *__restrict__ depth,
                                                              Intr in, Mat34 T, float inv_b)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int u = blockIdx.x * 32 + (warp & 3) * 8 + (lane & 7);
    const int v = blockIdx.y * 8 + (warp >> 2) * 4 + (lane >> 3);
    float d = 0.0f;
    if (u < in.W && v < in.H) d = __ldg(&depth[(size_t)v * in.W + u]);

    // frame's largest valid depth, for the visible-list depth cull
    {
        float dm = (d > 0.0f) ? d : 0.0f;
        for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(kFull, dm, o));
        if (lane == 0 && dm > 0.0f) atomicMax(&s.ctr->depth_max_bits, __float_as_int(dm));
    }

    bool more = (d > 0.0f) && !(d < s.z_min) && !(d > s.z_max);
    int cur[3] = {0, 0, 0}, step[3] = {0, 0, 0}, left[3] = {0, 0, 0};
    float tmax[3] = {0.f, 0.f, 0.f}, tdelta[3] = {0.f, 0.f, 0.f};
    if (more) {
        const float rx = fdiv(fsub((float)u, in.cx), in.fx);
        const float ry = fdiv(fsub((float)v, in.cy), in.fy);
        float z0 = fsub(d, s.mu);
        const float z1 = fadd(d, s.mu);
        if (z0 < 1e-3f) z0 = 1e-3f;
        const float ax = fmul(rx, z0), ay = fmul(ry, z0);
        const float bx = fmul(rx, z1), by = fmul(ry, z1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float q0 = fmul(row_apply(&T.m[4 * i], ax, ay, z0), inv_b);
            const float q1 = fmul(row_apply(&T.m[4 * i], bx, by, z1), inv_b);
            const float f0 = floorf(q0), f1 = floorf(q1);
            if (!(f0 >= -32768.0f && f0 <= 32767.0f && f1 >= -32768.0f && f1 <= 32767.0f)) {
                more = false;
                continue;
            }
            cur[i] = (int)f0;
            const int end = (int)f1;
            const float dir = fsub(q1, q0);
            if (end > cur[i]) {
                step[i] = 1;
                left[i] = end - cur[i];
                tdelta[i] = fdiv(1.0f, dir);
                tmax[i] = fdiv(fsub((float)(cur[i] + 1), q0), dir);
            } else if (end < cur[i]) {
                step[i] = -1;
                left[i] = cur[i] - end;
                tdelta[i] = fdiv(-1.0f, dir);
                tmax[i] = fdiv(fsub((float)cur[i], q0), dir);
            }
        }
        if (!more) set_status(s, ITM_ST_RANGE);
    }

    const uint32_t mask = (uint32_t)(s.nb - 1);
    while (__any_sync(kFull, more)) {
        const unsigned long long key = more ? pack_key(cur[0], cur[1], cur[2]) : 0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        if (more && lane == __ffs(peers) - 1) {
            if (lookup_ro(s, cur[0], cur[1], cur[2]) < 0) {
                const uint32_t h = hash_bucket(cur[0], cur[1], cur[2], mask);
                const unsigned long long old = atomicCAS(&s.req[h], 0ull, key);
                if (old == 0ull) {
                    const int p = warp_append(&s.ctr->n_req);
                    s.req_list[p] = (int32_t)h;  // at most one request per bucket: p < nb
                } else if (old != key) {
                    const int p = warp_append(&s.ctr->n_overflow);
                    if (p < s.ovf_cap) s.overflow[p] = key;
                    else set_status(s, ITM_ST_OVERFLOW);
                }
            }
        }
        if (more) {
            if (left[0] + left[1] + left[2] == 0) {
                more = false;
            } else {
                int a = -1;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    if (left[i] > 0 && (a < 0 || tmax[i] < tmax[a])) a = i;
                cur[a] += step[a];
                tmax[a] = fadd(tmax[a], tdelta[a]);
                left[a] -= 1;
            }
        }
    }
}

// Insert `key` into the chain of bucket h.  The caller is the only thread
// touching this chain in the running kernel.  blk is a block index already
// handed to the caller (or >= nv when the array is exhausted).
__device__ void insert_into_chain(const SceneDev &s, int h, unsigned long long key, int blk, bool need_excess_slot,
                                  int excess_slot)
{
    int bx, by, bz;
    unpack_key(key, bx, by, bz);
    int4 *E = reinterpret_cast<int4 *>(s.entries);
    if (blk >= s.nv) {
        set_status(s, ITM_ST_VBA_FULL);
        return;
    }
    const int ptr = __ldcg(&s.block_free[blk]);
    s.block_pos[ptr] = make_short4((short)bx, (short)by, (short)bz, 1);
    if (!need_excess_slot) {
        // the bucket itself was never used
        E[h] = make_int4((int)(uint32_t)(key & 0xffffffffull), (int)(uint32_t)(key >> 32), 0, ptr);
        return;
    }
    if (excess_slot >= s.ne) {
        set_status(s, ITM_ST_HASH_FULL);
        s.block_pos[ptr].w = 0;  // block handed out but unused
        return;
    }
    const int slot = __ldcg(&s.excess_free[excess_slot]);
    int idx = h;
    for (int guard = 0; guard <= s.ne; ++guard) {
        const int off = __ldcg(&E[idx].z);
        if (off < 1) break;
        idx = s.nb + off - 1;
    }
    E[s.nb + slot] = make_int4((int)(uint32_t)(key & 0xffffffffull), (int)(uint32_t)(key >> 32), 0, ptr);
    s.entries[idx].offset = slot + 1;
}

// ---------------------------------------------------------------- 2. commit

__global__ void __launch_bounds__(256) alloc_commit_kernel(SceneDev s)
{
    const int n = min(__ldcg(&s.ctr->n_req), s.nb);
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int i = i0 + threadIdx.x;
        if (i >= n) continue;
        const int h = s.req_list[i];
        const unsigned long long key = s.req[h];
        s.req[h] = 0ull;
        const bool bucket_used = __ldcg(&s.entries[h].flag) != 0;
        const int blk = warp_append(&s.ctr->block_head);
        int slot = 0;
        if (bucket_used) slot = warp_append(&s.ctr->excess_head);
        insert_into_chain(s, h, key, blk, bucket_used, slot);
    }
}

// -------------------------------------------------------------- 3. overflow

constexpr int kOvfThreads = 1024;
constexpr int kOvfCapacity = 1 << 20;
// bit 62 of a queued key marks "won its bucket this round" (keys use bits 0..48)
constexpr unsigned long long kWon = 1ull << 62;

__global__ void __launch_bounds__(kOvfThreads) alloc_overflow_kernel(SceneDev s)
{
    __shared__ int remaining;
    const int n = min(__ldcg(&s.ctr->n_overflow), s.ovf_cap);
    if (n == 0) return;
    const uint32_t mask = (uint32_t)(s.nb - 1);
    // every round inserts at least one key of each contended bucket
    for (int round = 0; round <= n; ++round) {
        if (threadIdx.x == 0) remaining = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kOvfThreads) {
            const unsigned long long key = __ldcg(&s.overflow[i]);
            if (key == 0ull) continue;
            int bx, by, bz;
            unpack_key(key, bx, by, bz);
            if (lookup_cg(s, bx, by, bz) >= 0) {
                s.overflow[i] = 0ull;
                continue;
            }
            const uint32_t h = hash_bucket(bx, by, bz, mask);
            const unsigned long long old = atomicCAS(&s.req[h], 0ull, key);
            if (old == 0ull) s.overflow[i] = key | kWon;
            else if (old == key) s.overflow[i] = 0ull;  // a twin won: it inserts the block
            else remaining = 1;
        }
        __threadfence();
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kOvfThreads) {
            const unsigned long long q = __ldcg(&s.overflow[i]);
            if (!(q & kWon)) continue;
            const unsigned long long key = q & ~kWon;
            int bx, by, bz;
            unpack_key(key, bx, by, bz);
            const uint32_t h = hash_bucket(bx, by, bz, mask);
            const bool bucket_used = __ldcg(&s.entries[h].flag) != 0;
            const int blk = atomicAdd(&s.ctr->block_head, 1);
            const int slot = bucket_used ? atomicAdd(&s.ctr->excess_head, 1) : 0;
            insert_into_chain(s, (int)h, key, blk, bucket_used, slot);
            s.req[h] = 0ull;
            s.overflow[i] = 0ull;
        }
        __threadfence();
        __syncthreads();
        const int rem = remaining;  // read by every thread before thread 0 clears it
        __syncthreads();
        if (rem == 0) return;
    }
    if (threadIdx.x == 0) set_status(s, ITM_ST_TIMEOUT);
}

// --------------------------------------------------------------- 4. visible

// Conservative test: can any voxel of block b be updated by this frame?
// Voxel sample positions span [8b, 8b+7] * s per axis; the projection of that
// box is bounded by the projections of its corners when all lie in front of
// the camera.  Margins absorb rounding differences to the exact per-voxel
// arithmetic of the integration.
__device__ __forceinline__ bool block_visible(const short4 b, const Mat34 &M, const Intr &in, float vs, float zfar)
{
    float zmin = 3.0e38f, zmax = -3.0e38f, umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
    bool all_front = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float px = (float)(b.x * 8 + ((c & 1) ? 7 : 0)) * vs;
        const float py = (float)(b.y * 8 + ((c & 2) ? 7 : 0)) * vs;
        const float pz = (float)(b.z * 8 + ((c & 4) ? 7 : 0)) * vs;
        const float X = M.m[0] * px + M.m[1] * py + M.m[2] * pz + M.m[3];
        const float Y = M.m[4] * px + M.m[5] * py + M.m[6] * pz + M.m[7];
        const float Z = M.m[8] * px + M.m[9] * py + M.m[10] * pz + M.m[11];
        zmin = fminf(zmin, Z);
        zmax = fmaxf(zmax, Z);
        if (Z < 1e-3f) {
            all_front = false;
        } else {
            const float u = in.fx * X / Z + in.cx, v = in.fy * Y / Z + in.cy;
            umin = fminf(umin, u);
            umax = fmaxf(umax, u);
            vmin = fminf(vmin, v);
            vmax = fmaxf(vmax, v);
        }
    }
    if (zmax < -1e-3f) return false;                 // entirely behind the camera
    if (zmin > zfar) return false;                   // every voxel is > mu behind any depth
    if (!all_front) return true;                     // straddles the image plane
    return umax >= 0.0f && umin <= (float)(in.W - 1) && vmax >= 0.0f && vmin <= (float)(in.H - 1);
}

__global__ void __launch_bounds__(256) build_visible_kernel(SceneDev s, Mat34 M, Intr in)
{
    const int n = min(__ldcg(&s.ctr->block_head), s.nv);
    const float dmax = __int_as_float(__ldcg(&s.ctr->depth_max_bits));
    const float zfar = (dmax + s.mu) * 1.001f + 1e-3f;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int i = i0 + threadIdx.x;
        if (i >= n) continue;
        const int ptr = __ldg(&s.block_free[i]);
        const short4 b = s.block_pos[ptr];
        if (b.w == 0) continue;
        if (block_visible(b, M, in, s.voxel_size, zfar)) {
            const int p = warp_append(&s.ctr->n_visible);
            s.visible[p] = ptr;
        }
    }
}

int persistent_grid(int threads, const void *kernel)
{
    static int cached_sm = 0;
    if (!cached_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached_sm, cudaDevAttrMultiProcessorCount, dev);
        if (cached_sm <= 0) cached_sm = 1;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm < 1) per_sm = 1;
    return cached_sm * per_sm;
}

}  // namespace

cudaError_t launch_allocate(const SceneDev &s, const float *depth, const Intr &in, const Mat34 &T_wc,
                            const Mat34 &M_d, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(reinterpret_cast<char *>(s.ctr) + kFrameCountersOffset, 0,
                                    kFrameCountersBytes, st);
    if (e != cudaSuccess) return e;
    const float inv_b = (float)(1.0 / (8.0 * (double)s.voxel_size));
    dim3 grid((in.W + 31) / 32, (in.H + 7) / 8);
    alloc_enumerate_kernel<<<grid, 256, 0, st>>>(s, depth, in, T_wc, inv_b);
    static int g_commit = 0, g_visible = 0;
    if (!g_commit) g_commit = persistent_grid(256, (const void *)alloc_commit_kernel);
    if (!g_visible) g_visible = persistent_grid(256, (const void *)build_visible_kernel);
    alloc_commit_kernel<<<g_commit, 256, 0, st>>>(s);
    alloc_overflow_kernel<<<1, kOvfThreads, 0, st>>>(s);
    build_visible_kernel<<<g_visible, 256, 0, st>>>(s, M_d, in);
    return cudaGetLastError();
}

int overflow_capacity() { return kOvfCapacity; }

}  // namespace itm
