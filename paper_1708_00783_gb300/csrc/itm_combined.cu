// Sec. 7.2 combined-map raycast: the global map of posed submaps rendered
// without building it.  At a world point X the combined TSDF is the sum over
// submaps of weight times TSDF at P_i X, divided by the weight sum (the
// printed sum is not normalised; dividing by the positive weight sum keeps
// its zero set and gives the Sec. 4.4 step rule a TSDF in [-1, 1]); where no
// submap has weight the value is the unobserved default 1.  In each submap
// the TSDF and the weight are interpolated trilinearly over the same eight
// voxels, an unallocated voxel counting as value 1, weight 0.  The march is
// the Sec. 4.4 state machine of itm_raycast in world coordinates, with "the
// block at X" allocated when the block of the nearest voxel of P_i X is
// allocated in some submap; refinement, hit point and iteration limit are
// those of itm_raycast; the normal is the normalised central difference of
// the combined value at X +- s along each world axis, absent when one of the
// six samples has no weight in any submap.
//
// Launch shape: one warp per 8x4-pixel tile, 32x8-pixel CTAs.  Every float
// operation that reaches a decision is an explicit round-to-nearest
// intrinsic in the order above (built with -fmad=false), so the result is
// that of the same arithmetic on any IEEE machine.  The submaps' tables and
// poses travel in the kernels' parameter block, so a call allocates nothing.
//
// Search ranges (Sec. 4.4, per submap): first every submap's allocated
// blocks are projected into the image, each block taken as the region of
// points whose trilinear stencil reads one of its voxels ([8b - 1.01,
// 8b + 8.01] voxels), giving per 8x4 tile and submap the nearest and
// farthest camera depth (written into the submap's own range scratch).  A
// submap whose range misses the sample's depth has no allocated voxel in
// the sample's stencil, so its term is an exact zero and is skipped; the
// coarse steps in front of every range are replayed without probes, and a
// ray beyond every range in the coarse or fine state can only miss.  The
// result is therefore the same with or without ranges.
#include "itm_ops.cuh"

namespace itm {

namespace {

struct CombinedArgs {
    SceneDev sub[kCombinedMax];
    Mat34 P[kCombinedMax];   // rows 0..2 of each submap-from-world pose
    Mat34 Mc[kCombinedMax];  // rows 0..2 of each camera-from-submap pose
    int n;
    int use_range;           // tile ranges in sub[i].range_min / range_max
    int tiles_x, tiles_y;
    float zc;                // the ranges cover points of camera depth >= zc
};

// The submap's term may be nonzero at ray depth t (always with no ranges).
__device__ __forceinline__ bool in_range(const CombinedArgs &A, const float *lo, const float *hi, int i, float t)
{
    return !A.use_range || t < A.zc || (t >= lo[i] && t <= hi[i]);
}

__global__ void __launch_bounds__(256) combined_range_clear_kernel(const CombinedArgs A, int n_tiles)
{
    const SceneDev &s = A.sub[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tiles; i += gridDim.x * blockDim.x) {
        s.range_min[i] = 0xffffffffu;
        s.range_max[i] = 0u;
    }
}

// Stencil-region ranges of the allocated blocks of submap blockIdx.y.
__global__ void __launch_bounds__(256) combined_range_kernel(const CombinedArgs A, Intr in)
{
    const SceneDev &s = A.sub[blockIdx.y];
    const Mat34 M = A.Mc[blockIdx.y];
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
            if (b.w) ok = block_tile_range(b, M, in, s.voxel_size, A.zc, A.tiles_x, A.tiles_y, r, 1.01f, 8.01f);
        }
        range_rasterize(ok, r, A.tiles_x, s.range_min, s.range_max);
    }
}

// Trilinear interpolation of the sdf and of the weight of submap s at its
// voxel coordinates q (|q| < 262000); unallocated voxels: sdf 1, weight 0.
template <int MODE>
__device__ __forceinline__ void trilinear_fw(const SceneDev &s, const float (&q)[3], float &F, float &Wt)
{
    const float g0x = floorf(q[0]), g0y = floorf(q[1]), g0z = floorf(q[2]);
    const float fx = fsub(q[0], g0x), fy = fsub(q[1], g0y), fz = fsub(q[2], g0z);
    const int x = (int)g0x, y = (int)g0y, z = (int)g0z;
    const int bx = x >> 3, by = y >> 3, bz = z >> 3;
    const bool cx = (x & 7) == 7, cy = (y & 7) == 7, cz = (z & 7) == 7;
    int P[8];
    P[0] = lookup_ro(s, bx, by, bz);
    P[1] = cx ? lookup_ro(s, bx + 1, by, bz) : P[0];
    P[2] = cy ? lookup_ro(s, bx, by + 1, bz) : P[0];
    P[3] = cy ? (cx ? lookup_ro(s, bx + 1, by + 1, bz) : P[2]) : P[1];
    P[4] = cz ? lookup_ro(s, bx, by, bz + 1) : P[0];
    P[5] = cz ? (cx ? lookup_ro(s, bx + 1, by, bz + 1) : P[4]) : P[1];
    P[6] = cz ? (cy ? lookup_ro(s, bx, by + 1, bz + 1) : P[4]) : P[2];
    P[7] = cz ? (cy ? (cx ? lookup_ro(s, bx + 1, by + 1, bz + 1) : P[6]) : P[5]) : P[3];
    const int lx[2] = {x & 7, (x + 1) & 7};
    const int ly[2] = {8 * (y & 7), 8 * ((y + 1) & 7)};
    const int lz[2] = {64 * (z & 7), 64 * ((z + 1) & 7)};
    float cv[8], wv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int ptr = P[k];
        if (ptr < 0) {
            cv[k] = 1.0f;
            wv[k] = 0.0f;
            continue;
        }
        const size_t i = (size_t)ptr * kBlockVoxels + (lx[k & 1] + ly[(k >> 1) & 1] + lz[(k >> 2) & 1]);
        cv[k] = __ldg(&s.sdf[i]);
        wv[k] = MODE == 0 ? u8_to_f(__ldg(&s.w8[i])) : __ldg(&s.w32[i]);
    }
    float out[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const float *v = m == 0 ? cv : wv;
        const float c00 = lerp_rn(v[0], v[1], fx);
        const float c10 = lerp_rn(v[2], v[3], fx);
        const float c01 = lerp_rn(v[4], v[5], fx);
        const float c11 = lerp_rn(v[6], v[7], fx);
        const float c0 = lerp_rn(c00, c10, fy);
        const float c1 = lerp_rn(c01, c11, fy);
        out[m] = lerp_rn(c0, c1, fz);
    }
    F = out[0];
    Wt = out[1];
}

// Voxel coordinates of world point X in submap i; false when out of range.
__device__ __forceinline__ bool submap_coords(const CombinedArgs &A, int i, const float (&X)[3], float inv_s,
                                              float (&q)[3])
{
    bool ok = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        q[r] = fmul(row_apply(A.P[i].m + 4 * r, X[0], X[1], X[2]), inv_s);
        ok = ok && coord_ok(q[r]);
    }
    return ok;
}

// Is the block of the voxel nearest to X (ray depth t) allocated in some submap?
__device__ __forceinline__ bool combined_alloc(const CombinedArgs &A, const float (&X)[3], float inv_s, float t,
                                               const float *lo, const float *hi)
{
    for (int i = 0; i < A.n; ++i) {
        if (!in_range(A, lo, hi, i, t)) continue;
        float q[3];
        if (!submap_coords(A, i, X, inv_s, q)) continue;
        const int bx = ((int)floorf(fadd(q[0], 0.5f))) >> 3;
        const int by = ((int)floorf(fadd(q[1], 0.5f))) >> 3;
        const int bz = ((int)floorf(fadd(q[2], 0.5f))) >> 3;
        if (in_i16(bx) && in_i16(by) && in_i16(bz) && lookup_ro(A.sub[i], bx, by, bz) >= 0) return true;
    }
    return false;
}

// The combined value at X; den receives the weight sum.  With ray depth t
// (on_ray) submaps whose range misses t are skipped (their term is 0).
template <int MODE>
__device__ __forceinline__ float combined_value(const CombinedArgs &A, const float (&X)[3], float inv_s, float &den,
                                                bool on_ray = false, float t = 0.0f, const float *lo = nullptr,
                                                const float *hi = nullptr)
{
    float num = 0.0f, dsum = 0.0f;
    for (int i = 0; i < A.n; ++i) {
        if (on_ray && !in_range(A, lo, hi, i, t)) continue;
        float q[3];
        if (!submap_coords(A, i, X, inv_s, q)) continue;
        float F, Wt;
        trilinear_fw<MODE>(A.sub[i], q, F, Wt);
        num = fadd(num, fmul(Wt, F));
        dsum = fadd(dsum, Wt);
    }
    den = dsum;
    return dsum > 0.0f ? fdiv(num, dsum) : 1.0f;
}

template <int MODE>
__global__ void __launch_bounds__(256) raycast_combined_kernel(const CombinedArgs A, Intr in, Mat34 T,
                                                               float4 *__restrict__ vtx, float4 *__restrict__ nrm,
                                                               int max_iter, float tB_m, float inv_s, float vs,
                                                               float mu, float z_min, float z_max)
{
    __shared__ float s_lo[8][kCombinedMax], s_hi[8][kCombinedMax];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tix = blockIdx.x * 4 + (warp & 3), tiy = blockIdx.y * 2 + (warp >> 2);
    if (tix * 8 >= in.W || tiy * 4 >= in.H) return;  // the whole warp's tile is outside
    const float *lo = s_lo[warp], *hi = s_hi[warp];
    float T0 = 0.0f, T1 = 3.0e38f;  // nearest and farthest range over the submaps
    if (A.use_range) {
        if (lane < A.n) {
            const int tile = tiy * A.tiles_x + tix;
            const uint32_t a = __ldg(&A.sub[lane].range_min[tile]), b = __ldg(&A.sub[lane].range_max[tile]);
            s_lo[warp][lane] = a == 0xffffffffu ? 3.0e38f : __uint_as_float(a);
            s_hi[warp][lane] = a == 0xffffffffu ? -3.0e38f : __uint_as_float(b);
        }
        __syncwarp();
        T0 = 3.0e38f;
        T1 = -3.0e38f;
        for (int i = 0; i < A.n; ++i) {
            T0 = fminf(T0, lo[i]);
            T1 = fmaxf(T1, hi[i]);
        }
    }
    const int u = tix * 8 + (lane & 7), v = tiy * 4 + (lane >> 3);
    if (u >= in.W || v >= in.H) return;
    const size_t o = (size_t)v * in.W + u;
    const float dc0 = fdiv(fsub((float)u, in.cx), in.fx);
    const float dc1 = fdiv(fsub((float)v, in.cy), in.fy);
    const float len = __fsqrt_rn(fadd(fadd(fmul(dc0, dc0), fmul(dc1, dc1)), 1.0f));
    float org[3], dir[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dir[i] = fadd(fadd(fmul(T.m[4 * i], dc0), fmul(T.m[4 * i + 1], dc1)), T.m[4 * i + 2]);
        org[i] = T.m[4 * i + 3];
    }
    const float tB = fdiv(tB_m, len), tmu = fdiv(mu, len), ts = fdiv(vs, len);
    float t = z_min;
    int state = COARSE;
    int it = 0;
    if (A.use_range) {
        if (T1 < T0) {
            state = MISS;  // no submap has a block near this tile
        } else {
            // the oracle's coarse steps in front of every range: t += tB each
            while (t < T0 && it < max_iter && t <= z_max) {
                t = fadd(t, tB);
                ++it;
            }
        }
    }
    float X[3];
    for (; state <= SURFACE && it < max_iter && t <= z_max; ++it) {
        if (A.use_range && state != SURFACE && t > T1) break;  // only unallocated space ahead: a miss
#pragma unroll
        for (int i = 0; i < 3; ++i) X[i] = fadd(org[i], fmul(t, dir[i]));
        const bool alloc = combined_alloc(A, X, inv_s, t, lo, hi);
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
        float den;
        const float F = combined_value<MODE>(A, X, inv_s, den, true, t, lo, hi);
        if (state == FINE) {
            if (F <= 0.0f) {
                state = WRONG;
                break;
            }
            state = SURFACE;
        }
        if (F <= 0.0f) {
            state = BEHIND;
            break;
        }
        float step = fmul(F, tmu);
        if (step < ts) step = ts;
        t = fadd(t, step);
    }
    float4 V = make_float4(0.f, 0.f, 0.f, 0.f), N = make_float4(0.f, 0.f, 0.f, 0.f);
    if (state == BEHIND) {
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int i = 0; i < 3; ++i) X[i] = fadd(org[i], fmul(t, dir[i]));
            float den;
            const float F = combined_value<MODE>(A, X, inv_s, den, true, t, lo, hi);
            t = fadd(t, fmul(F, tmu));
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) X[i] = fadd(org[i], fmul(t, dir[i]));
        V = make_float4(X[0], X[1], X[2], 1.0f);
        float g[3];
        bool obs = true;
#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            float Xp[3] = {X[0], X[1], X[2]}, Xm[3] = {X[0], X[1], X[2]};
            Xp[a] = fadd(X[a], vs);
            Xm[a] = fsub(X[a], vs);
            float dp, dm;
            const float fp = combined_value<MODE>(A, Xp, inv_s, dp);
            const float fm = combined_value<MODE>(A, Xm, inv_s, dm);
            obs = obs && dp > 0.0f && dm > 0.0f;
            g[a] = fsub(fp, fm);
        }
        const float gl = __fsqrt_rn(fadd(fadd(fmul(g[0], g[0]), fmul(g[1], g[1])), fmul(g[2], g[2])));
        if (obs && gl > 0.0f) N = make_float4(fdiv(g[0], gl), fdiv(g[1], gl), fdiv(g[2], gl), 1.0f);
    }
    vtx[o] = V;
    nrm[o] = N;
}

}  // namespace

cudaError_t launch_raycast_combined(const SceneDev *subs, const Mat34 *P, int n, const Intr &in, const Mat34 &T_wc,
                                    float4 *vtx, float4 *nrm, cudaStream_t st)
{
    CombinedArgs A;
    memset(&A, 0, sizeof(A));
    for (int i = 0; i < n; ++i) {
        A.sub[i] = subs[i];
        A.P[i] = P[i];
        // camera-from-submap = (P_i T_wc)^-1, composed and inverted in fp64
        double R[3][3], t[3];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) {
                R[r][c] = 0.0;
                for (int k = 0; k < 3; ++k) R[r][c] += (double)P[i].m[4 * r + k] * (double)T_wc.m[4 * k + c];
            }
            t[r] = (double)P[i].m[4 * r + 3];
            for (int k = 0; k < 3; ++k) t[r] += (double)P[i].m[4 * r + k] * (double)T_wc.m[4 * k + 3];
        }
        for (int r = 0; r < 3; ++r) {
            double tr = 0.0;
            for (int k = 0; k < 3; ++k) {
                A.Mc[i].m[4 * r + k] = (float)R[k][r];
                tr -= R[k][r] * t[k];
            }
            A.Mc[i].m[4 * r + 3] = (float)tr;
        }
    }
    A.n = n;
    const SceneDev &s0 = subs[0];
    A.use_range = range_fits(in) ? 1 : 0;
    A.tiles_x = (in.W + 7) / 8;
    A.tiles_y = (in.H + 3) / 4;
    A.zc = s0.z_min - 1e-3f;
    // host-side constants with the same float operations as the oracle
    volatile float span = s0.z_max - s0.z_min;
    volatile float four_span = 4.0f * span;
    volatile float ratio = four_span / s0.voxel_size;
    const int max_iter = (int)ratio + 64;
    volatile float tB_m = 8.0f * s0.voxel_size;
    const float inv_s = (float)(1.0 / (double)s0.voxel_size);
    if (A.use_range) {
        const int n_tiles = A.tiles_x * A.tiles_y;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int gx = (n_tiles + 255) / 256 < sms ? (n_tiles + 255) / 256 : sms;
        combined_range_clear_kernel<<<dim3(gx, n), 256, 0, st>>>(A, n_tiles);
        const int gr = (4 * sms + n - 1) / n;
        combined_range_kernel<<<dim3(gr, n), 256, 0, st>>>(A, in);
    }
    dim3 grid((in.W + 31) / 32, (in.H + 7) / 8);
    if (s0.weight_mode == 0)
        raycast_combined_kernel<0><<<grid, 256, 0, st>>>(A, in, T_wc, vtx, nrm, max_iter, tB_m, inv_s, s0.voxel_size,
                                                         s0.mu, s0.z_min, s0.z_max);
    else
        raycast_combined_kernel<1><<<grid, 256, 0, st>>>(A, in, T_wc, vtx, nrm, max_iter, tB_m, inv_s, s0.voxel_size,
                                                         s0.mu, s0.z_min, s0.z_max);
    return cudaGetLastError();
}

}  // namespace itm
