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
// The per-iteration "is the block at p allocated" query runs with the whole
// warp converged: lanes asking for the same block are grouped with
// __match_any_sync and one lane per group walks the hash chain (Sec. 3.3),
// the others take its answer by shuffle.  Every arithmetic step uses IEEE
// round-to-nearest operations in a fixed order.
#include "itm_internal.cuh"

namespace itm {

namespace {

enum { COARSE = 0, FINE = 1, SURFACE = 2, BEHIND = 3, WRONG = 4, MISS = 5 };

__device__ __forceinline__ bool coord_ok(float q) { return q > -262000.0f && q < 262000.0f; }
__device__ __forceinline__ bool in_i16(int v) { return v >= -32768 && v <= 32767; }

__device__ __forceinline__ float lerp_rn(float a, float b, float t) { return fadd(a, fmul(t, fsub(b, a))); }

// Block index of block (bx, by, bz) or -1; a per-thread one-entry cache
// holds the last answer.
struct BlockCache {
    unsigned long long key;
    int ptr;
};

__device__ __forceinline__ int cached_lookup(const SceneDev &s, BlockCache &c, int bx, int by, int bz)
{
    if (!(in_i16(bx) && in_i16(by) && in_i16(bz))) return -1;
    const unsigned long long k = pack_key(bx, by, bz);
    if (k == c.key) return c.ptr;
    c.key = k;
    c.ptr = lookup_ro(s, bx, by, bz);
    return c.ptr;
}

// Voxel value and "observed" flag (allocated with weight > 0).
template <int MODE>
__device__ __forceinline__ float voxel_at(const SceneDev &s, int ptr, int gx, int gy, int gz, bool &obs)
{
    if (ptr < 0) {
        obs = false;
        return 1.0f;
    }
    const size_t i = (size_t)ptr * kBlockVoxels + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
    if (MODE == 0) obs = __ldg(&s.w8[i]) != 0;
    else obs = __ldg(&s.w32[i]) > 0.0f;
    return __ldg(&s.sdf[i]);
}

// Trilinear interpolation at voxel coordinates q; clears all_obs when one of
// the eight voxels is unallocated or unobserved.
template <int MODE>
__device__ float trilinear(const SceneDev &s, BlockCache &c, const float q[3], bool &all_obs)
{
    const float g0x = floorf(q[0]), g0y = floorf(q[1]), g0z = floorf(q[2]);
    const float fx = fsub(q[0], g0x), fy = fsub(q[1], g0y), fz = fsub(q[2], g0z);
    const int x = (int)g0x, y = (int)g0y, z = (int)g0z;
    float cv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int gx = x + (k & 1), gy = y + ((k >> 1) & 1), gz = z + ((k >> 2) & 1);
        const int ptr = cached_lookup(s, c, gx >> 3, gy >> 3, gz >> 3);
        bool o;
        cv[k] = voxel_at<MODE>(s, ptr, gx, gy, gz, o);
        all_obs = all_obs && o;
    }
    const float c00 = lerp_rn(cv[0], cv[1], fx);
    const float c10 = lerp_rn(cv[2], cv[3], fx);
    const float c01 = lerp_rn(cv[4], cv[5], fx);
    const float c11 = lerp_rn(cv[6], cv[7], fx);
    const float c0 = lerp_rn(c00, c10, fy);
    const float c1 = lerp_rn(c01, c11, fy);
    return lerp_rn(c0, c1, fz);
}

template <int MODE>
__global__ void __launch_bounds__(256) raycast_kernel(SceneDev s, Intr in, Mat34 T, float4 *__restrict__ vtx,
                                                      float4 *__restrict__ nrm, int max_iter, float tB_m,
                                                      float inv_sv)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int u = blockIdx.x * 32 + (warp & 3) * 8 + (lane & 7);
    const int v = blockIdx.y * 8 + (warp >> 2) * 4 + (lane >> 3);
    const bool inside = u < in.W && v < in.H;

    const float vs = s.voxel_size;
    float org[3], dir[3];
    const float dc0 = fdiv(fsub((float)u, in.cx), in.fx);
    const float dc1 = fdiv(fsub((float)v, in.cy), in.fy);
    const float len = __fsqrt_rn(fadd(fadd(fmul(dc0, dc0), fmul(dc1, dc1)), 1.0f));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dir[i] = fadd(fadd(fmul(T.m[4 * i], dc0), fmul(T.m[4 * i + 1], dc1)), T.m[4 * i + 2]);
        org[i] = T.m[4 * i + 3];
    }
    const float tB = fdiv(tB_m, len), tmu = fdiv(s.mu, len), ts = fdiv(vs, len);

    BlockCache cache{0ull, -1};
    float t = s.z_min;
    int state = inside ? COARSE : MISS;
    int it = 0;
    float q[3];

    while (__any_sync(kFull, state <= SURFACE)) {
        bool marching = state <= SURFACE;
        if (marching && !(it < max_iter && t <= s.z_max)) {
            state = MISS;
            marching = false;
        }
        bool ok = marching;
        int bx = 0, by = 0, bz = 0;
        if (marching) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                q[i] = fmul(fadd(org[i], fmul(t, dir[i])), inv_sv);
                ok = ok && coord_ok(q[i]);
            }
            if (ok) {
                bx = ((int)floorf(fadd(q[0], 0.5f))) >> 3;
                by = ((int)floorf(fadd(q[1], 0.5f))) >> 3;
                bz = ((int)floorf(fadd(q[2], 0.5f))) >> 3;
                ok = in_i16(bx) && in_i16(by) && in_i16(bz);
            }
        }
        // warp-cooperative block query
        const unsigned long long key = ok ? pack_key(bx, by, bz) : 0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        const int leader = __ffs(peers) - 1;
        int ptr = -1;
        if (ok && lane == leader) ptr = (key == cache.key) ? cache.ptr : lookup_ro(s, bx, by, bz);
        ptr = __shfl_sync(kFull, ptr, leader);
        if (ok) {
            cache.key = key;
            cache.ptr = ptr;
        }
        if (!marching) continue;
        ++it;
        const bool alloc = ok && ptr >= 0;
        if (state == COARSE) {
            if (!alloc) {
                t = fadd(t, tB);
            } else {
                t = fsub(t, tB);
                state = FINE;
            }
            continue;
        }
        if (!alloc) {
            if (state == FINE) t = fadd(t, tmu);
            else state = COARSE;
            continue;
        }
        bool obs = true;
        const float F = trilinear<MODE>(s, cache, q, obs);
        if (state == FINE) {
            if (F <= 0.0f) {
                state = WRONG;
                continue;
            }
            state = SURFACE;
        }
        if (F <= 0.0f) {
            state = BEHIND;
            continue;
        }
        float step = fmul(F, tmu);
        if (step < ts) step = ts;
        t = fadd(t, step);
    }
    if (!inside) return;
    const size_t o = (size_t)v * in.W + u;
    float4 V = make_float4(0.f, 0.f, 0.f, 0.f), N = make_float4(0.f, 0.f, 0.f, 0.f);
    if (state == BEHIND) {
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int i = 0; i < 3; ++i) q[i] = fmul(fadd(org[i], fmul(t, dir[i])), inv_sv);
            bool obs = true;
            const float F = trilinear<MODE>(s, cache, q, obs);
            t = fadd(t, fmul(F, tmu));
        }
        float p[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            p[i] = fadd(org[i], fmul(t, dir[i]));
            q[i] = fmul(p[i], inv_sv);
        }
        if (coord_ok(q[0]) && coord_ok(q[1]) && coord_ok(q[2])) {
            V = make_float4(p[0], p[1], p[2], 1.0f);
            float g[3];
            bool obs = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
                qp[a] = fadd(q[a], 1.0f);
                qm[a] = fsub(q[a], 1.0f);
                const float fp = trilinear<MODE>(s, cache, qp, obs);
                const float fm = trilinear<MODE>(s, cache, qm, obs);
                g[a] = fsub(fp, fm);
            }
            const float gl = __fsqrt_rn(fadd(fadd(fmul(g[0], g[0]), fmul(g[1], g[1])), fmul(g[2], g[2])));
            if (obs && gl > 0.0f) N = make_float4(fdiv(g[0], gl), fdiv(g[1], gl), fdiv(g[2], gl), 1.0f);
        }
    }
    vtx[o] = V;
    nrm[o] = N;
}

}  // namespace

cudaError_t launch_raycast(const SceneDev &s, const Intr &in, const Mat34 &T_wc, float4 *vtx, float4 *nrm,
                           cudaStream_t st)
{
    // host-side constants with the same float operations as the oracle
    volatile float span = s.z_max - s.z_min;
    volatile float four_span = 4.0f * span;
    volatile float ratio = four_span / s.voxel_size;
    const int max_iter = (int)ratio + 64;
    volatile float tB_m = 8.0f * s.voxel_size;
    const float inv_sv = (float)(1.0 / (double)s.voxel_size);  // voxel coordinates: p * (1/s), 1/s rounded once
    dim3 grid((in.W + 31) / 32, (in.H + 7) / 8);
    if (s.weight_mode == 0)
        raycast_kernel<0><<<grid, 256, 0, st>>>(s, in, T_wc, vtx, nrm, max_iter, tB_m, inv_sv);
    else
        raycast_kernel<1><<<grid, 256, 0, st>>>(s, in, T_wc, vtx, nrm, max_iter, tB_m, inv_sv);
    return cudaGetLastError();
}

}  // namespace itm
