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
// poses travel in the kernel's parameter block, so a call allocates nothing.
#include "itm_ops.cuh"

namespace itm {

namespace {

struct CombinedArgs {
    SceneDev sub[kCombinedMax];
    Mat34 P[kCombinedMax];  // rows 0..2 of each submap-from-world pose
    int n;
};

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

// Is the block of the voxel nearest to X allocated in some submap?
__device__ __forceinline__ bool combined_alloc(const CombinedArgs &A, const float (&X)[3], float inv_s)
{
    for (int i = 0; i < A.n; ++i) {
        float q[3];
        if (!submap_coords(A, i, X, inv_s, q)) continue;
        const int bx = ((int)floorf(fadd(q[0], 0.5f))) >> 3;
        const int by = ((int)floorf(fadd(q[1], 0.5f))) >> 3;
        const int bz = ((int)floorf(fadd(q[2], 0.5f))) >> 3;
        if (in_i16(bx) && in_i16(by) && in_i16(bz) && lookup_ro(A.sub[i], bx, by, bz) >= 0) return true;
    }
    return false;
}

// The combined value at X; den receives the weight sum.
template <int MODE>
__device__ __forceinline__ float combined_value(const CombinedArgs &A, const float (&X)[3], float inv_s, float &den)
{
    float num = 0.0f, dsum = 0.0f;
    for (int i = 0; i < A.n; ++i) {
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
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = (blockIdx.x * 4 + (warp & 3)) * 8 + (lane & 7);
    const int v = (blockIdx.y * 2 + (warp >> 2)) * 4 + (lane >> 3);
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
    float X[3];
    for (int it = 0; it < max_iter && t <= z_max; ++it) {
#pragma unroll
        for (int i = 0; i < 3; ++i) X[i] = fadd(org[i], fmul(t, dir[i]));
        const bool alloc = combined_alloc(A, X, inv_s);
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
        const float F = combined_value<MODE>(A, X, inv_s, den);
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
            const float F = combined_value<MODE>(A, X, inv_s, den);
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
    }
    A.n = n;
    const SceneDev &s0 = subs[0];
    // host-side constants with the same float operations as the oracle
    volatile float span = s0.z_max - s0.z_min;
    volatile float four_span = 4.0f * span;
    volatile float ratio = four_span / s0.voxel_size;
    const int max_iter = (int)ratio + 64;
    volatile float tB_m = 8.0f * s0.voxel_size;
    const float inv_s = (float)(1.0 / (double)s0.voxel_size);
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
