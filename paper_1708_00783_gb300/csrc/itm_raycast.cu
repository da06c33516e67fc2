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
// The per-iteration "is the block at p allocated" query runs with the whole
// warp converged: lanes asking for the same block are grouped with
// __match_any_sync and one lane per group walks the hash chain (Sec. 3.3),
// the others take its answer by shuffle.  Every arithmetic step of the march
// uses IEEE round-to-nearest operations in a fixed order.
#include "itm_internal.cuh"

namespace itm {

namespace {

enum { COARSE = 0, FINE = 1, SURFACE = 2, BEHIND = 3, WRONG = 4, MISS = 5 };

constexpr float kRangeMarginZ = 1e-4f;  // metres, covers rounding of p(t) vs t
constexpr float kRangeMarginPx = 1.0f;  // pixels

__device__ __forceinline__ bool coord_ok(float q) { return q > -262000.0f && q < 262000.0f; }
__device__ __forceinline__ bool in_i16(int v) { return v >= -32768 && v <= 32767; }

__device__ __forceinline__ float lerp_rn(float a, float b, float t) { return fadd(a, fmul(t, fsub(b, a))); }

// One-entry cache of the last block looked up by this thread.
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

template <int MODE, bool OBS>
__device__ __forceinline__ float voxel_at(const SceneDev &s, int ptr, int gx, int gy, int gz, bool &all_obs)
{
    if (ptr < 0) {
        if (OBS) all_obs = false;
        return 1.0f;
    }
    const size_t i = (size_t)ptr * kBlockVoxels + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
    if (OBS) {
        if (MODE == 0) all_obs = all_obs && (__ldg(&s.w8[i]) != 0);
        else all_obs = all_obs && (__ldg(&s.w32[i]) > 0.0f);
    }
    return __ldg(&s.sdf[i]);
}

// Trilinear interpolation at voxel coordinates (q0, q1, q2).  Each distinct
// block under the 2x2x2 stencil is looked up once.  With OBS, all_obs is
// cleared when one of the eight voxels is unallocated or unobserved.
template <int MODE, bool OBS>
__device__ __forceinline__ float trilinear(const SceneDev &s, BlockCache &c, float q0, float q1, float q2,
                                           bool &all_obs)
{
    const float g0x = floorf(q0), g0y = floorf(q1), g0z = floorf(q2);
    const float fx = fsub(q0, g0x), fy = fsub(q1, g0y), fz = fsub(q2, g0z);
    const int x = (int)g0x, y = (int)g0y, z = (int)g0z;
    const int bx = x >> 3, by = y >> 3, bz = z >> 3;
    const bool cx = (x & 7) == 7, cy = (y & 7) == 7, cz = (z & 7) == 7;
    int P[8];
    P[0] = cached_lookup(s, c, bx, by, bz);
    P[1] = cx ? cached_lookup(s, c, bx + 1, by, bz) : P[0];
    P[2] = cy ? cached_lookup(s, c, bx, by + 1, bz) : P[0];
    P[3] = cy ? (cx ? cached_lookup(s, c, bx + 1, by + 1, bz) : P[2]) : P[1];
    P[4] = cz ? cached_lookup(s, c, bx, by, bz + 1) : P[0];
    P[5] = cz ? (cx ? cached_lookup(s, c, bx + 1, by, bz + 1) : P[4]) : P[1];
    P[6] = cz ? (cy ? cached_lookup(s, c, bx, by + 1, bz + 1) : P[4]) : P[2];
    P[7] = cz ? (cy ? (cx ? cached_lookup(s, c, bx + 1, by + 1, bz + 1) : P[6]) : P[5]) : P[3];
    float cv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        cv[k] = voxel_at<MODE, OBS>(s, P[k], x + (k & 1), y + ((k >> 1) & 1), z + ((k >> 2) & 1), all_obs);
    const float c00 = lerp_rn(cv[0], cv[1], fx);
    const float c10 = lerp_rn(cv[2], cv[3], fx);
    const float c01 = lerp_rn(cv[4], cv[5], fx);
    const float c11 = lerp_rn(cv[6], cv[7], fx);
    const float c0 = lerp_rn(c00, c10, fy);
    const float c1 = lerp_rn(c01, c11, fy);
    return lerp_rn(c0, c1, fz);
}

// ------------------------------------------------------------ search range

struct TileRange {
    int tx0, tx1, ty0, ty1;
    float zlo, zhi;
};

// Conservative tile rectangle and depth range of block b's query region
// clipped to z >= zc.  Returns false when the region cannot be met by a ray.
__device__ bool block_tile_range(short4 b, const Mat34 &M, const Intr &in, float vs, float zc, int tiles_x,
                                 int tiles_y, TileRange &r)
{
    const float eps = 1e-5f;
    const float lo[3] = {((float)(b.x * 8) - 0.51f) * vs - eps, ((float)(b.y * 8) - 0.51f) * vs - eps,
                         ((float)(b.z * 8) - 0.51f) * vs - eps};
    const float hi[3] = {((float)(b.x * 8) + 7.51f) * vs + eps, ((float)(b.y * 8) + 7.51f) * vs + eps,
                         ((float)(b.z * 8) + 7.51f) * vs + eps};
    float X[8], Y[8], Z[8];
    float zmax = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float px = (c & 1) ? hi[0] : lo[0], py = (c & 2) ? hi[1] : lo[1], pz = (c & 4) ? hi[2] : lo[2];
        X[c] = M.m[0] * px + M.m[1] * py + M.m[2] * pz + M.m[3];
        Y[c] = M.m[4] * px + M.m[5] * py + M.m[6] * pz + M.m[7];
        Z[c] = M.m[8] * px + M.m[9] * py + M.m[10] * pz + M.m[11];
        zmax = fmaxf(zmax, Z[c]);
    }
    if (zmax < zc) return false;
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f, zmin = 3.0e38f;
    auto add_point = [&](float x, float y, float z) {
        const float u = in.fx * x / z + in.cx, v = in.fy * y / z + in.cy;
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
        zmin = fminf(zmin, z);
    };
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (Z[c] >= zc) add_point(X[c], Y[c], Z[c]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int d = c | (1 << a);
            if (d == c) continue;
            // edge c-d crosses the plane z = zc
            if ((Z[c] < zc) != (Z[d] < zc)) {
                const float w = (zc - Z[c]) / (Z[d] - Z[c]);
                add_point(X[c] + w * (X[d] - X[c]), Y[c] + w * (Y[d] - Y[c]), zc);
            }
        }
    }
    if (!(umax >= -kRangeMarginPx && vmax >= -kRangeMarginPx && umin <= (float)in.W - 1.0f + kRangeMarginPx &&
          vmin <= (float)in.H - 1.0f + kRangeMarginPx))
        return false;
    const float u0 = fmaxf(umin - kRangeMarginPx, 0.0f), u1 = fminf(umax + kRangeMarginPx, (float)(in.W - 1));
    const float v0 = fmaxf(vmin - kRangeMarginPx, 0.0f), v1 = fminf(vmax + kRangeMarginPx, (float)(in.H - 1));
    r.tx0 = min((int)u0 >> 3, tiles_x - 1);
    r.tx1 = min((int)u1 >> 3, tiles_x - 1);
    r.ty0 = min((int)v0 >> 2, tiles_y - 1);
    r.ty1 = min((int)v1 >> 2, tiles_y - 1);
    r.zlo = fmaxf(zmin - kRangeMarginZ, 0.0f);
    r.zhi = zmax + kRangeMarginZ;
    return r.tx0 <= r.tx1 && r.ty0 <= r.ty1;
}

// One warp takes 32 allocated blocks; their tile rectangles are then
// rasterised by the whole warp, block after block, with atomic min/max on the
// float bits (non-negative floats order like their bit patterns).
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
        unsigned todo = __ballot_sync(kFull, ok);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const int tx0 = __shfl_sync(kFull, r.tx0, j), tx1 = __shfl_sync(kFull, r.tx1, j);
            const int ty0 = __shfl_sync(kFull, r.ty0, j), ty1 = __shfl_sync(kFull, r.ty1, j);
            const uint32_t zlo = __float_as_uint(__shfl_sync(kFull, r.zlo, j));
            const uint32_t zhi = __float_as_uint(__shfl_sync(kFull, r.zhi, j));
            const int w = tx1 - tx0 + 1, cnt = w * (ty1 - ty0 + 1);
            for (int k = lane; k < cnt; k += 32) {
                const int t = (ty0 + k / w) * tiles_x + tx0 + k % w;
                atomicMin(&rmin[t], zlo);
                atomicMax(&rmax[t], zhi);
            }
        }
    }
}

// ---------------------------------------------------------------- march

template <int MODE, bool RANGE>
__global__ void __launch_bounds__(256) raycast_kernel(SceneDev s, Intr in, Mat34 T, float4 *__restrict__ vtx,
                                                      float4 *__restrict__ nrm, int max_iter, float tB_m,
                                                      float inv_sv, const uint32_t *__restrict__ rmin,
                                                      const uint32_t *__restrict__ rmax, int tiles_x, int tiles_y)
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
    float tlo = 0.0f, thi = 3.0e38f;
    const int tix = blockIdx.x * 4 + (warp & 3), tiy = blockIdx.y * 2 + (warp >> 2);
    if (RANGE && tix < tiles_x && tiy < tiles_y) {
        // the warp's pixels form one tile (a tile outside the image has no pixel inside)
        const int tile = tiy * tiles_x + tix;
        const uint32_t lo = __ldg(&rmin[tile]), hi = __ldg(&rmax[tile]);
        if (lo == 0xffffffffu) {
            tlo = thi = -1.0f;  // no block covers the tile
        } else {
            tlo = __uint_as_float(lo);
            thi = __uint_as_float(hi);
        }
        if (state == COARSE) {
            if (thi < 0.0f) {
                state = MISS;
            } else {
                // the oracle's coarse steps in front of every block: t += tB each
                while (t < tlo && it < max_iter && t <= s.z_max) {
                    t = fadd(t, tB);
                    ++it;
                }
            }
        }
    }
    float q[3] = {0.f, 0.f, 0.f};

    while (__any_sync(kFull, state <= SURFACE)) {
        bool marching = state <= SURFACE;
        if (marching && !(it < max_iter && t <= s.z_max)) {
            state = MISS;
            marching = false;
        }
        if (RANGE && marching && state != SURFACE && t > thi) {
            state = MISS;  // only unallocated space ahead: the march can only miss
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
        bool unused = true;
        const float F = trilinear<MODE, false>(s, cache, q[0], q[1], q[2], unused);
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
            bool unused = true;
            const float F = trilinear<MODE, false>(s, cache, q[0], q[1], q[2], unused);
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
            bool obs = true;
            const float gx = fsub(trilinear<MODE, true>(s, cache, fadd(q[0], 1.0f), q[1], q[2], obs),
                                  trilinear<MODE, true>(s, cache, fsub(q[0], 1.0f), q[1], q[2], obs));
            const float gy = fsub(trilinear<MODE, true>(s, cache, q[0], fadd(q[1], 1.0f), q[2], obs),
                                  trilinear<MODE, true>(s, cache, q[0], fsub(q[1], 1.0f), q[2], obs));
            const float gz = fsub(trilinear<MODE, true>(s, cache, q[0], q[1], fadd(q[2], 1.0f), obs),
                                  trilinear<MODE, true>(s, cache, q[0], q[1], fsub(q[2], 1.0f), obs));
            const float gl = __fsqrt_rn(fadd(fadd(fmul(gx, gx), fmul(gy, gy)), fmul(gz, gz)));
            if (obs && gl > 0.0f) N = make_float4(fdiv(gx, gl), fdiv(gy, gl), fdiv(gz, gl), 1.0f);
        }
    }
    vtx[o] = V;
    nrm[o] = N;
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
                           float4 *nrm, cudaStream_t st)
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
        cudaError_t e = launch_raycast_range(s, in, M_d, s.range_min, s.range_max, st);
        if (e != cudaSuccess) return e;
        if (s.weight_mode == 0)
            raycast_kernel<0, true><<<grid, 256, 0, st>>>(s, in, T_wc, vtx, nrm, max_iter, tB_m, inv_sv, s.range_min,
                                                          s.range_max, tx, ty);
        else
            raycast_kernel<1, true><<<grid, 256, 0, st>>>(s, in, T_wc, vtx, nrm, max_iter, tB_m, inv_sv, s.range_min,
                                                          s.range_max, tx, ty);
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

}  // namespace itm
