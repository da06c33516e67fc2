// Sec. 4.3 integration over the visible blocks.
//
// Launch shape: a persistent grid of 128-thread CTAs walks the visible list
// (its length is read from device memory).  A CTA takes one 8^3 block per
// iteration; thread t owns voxels 4t .. 4t+3 (x = 4(t&1) .. +3, y = (t>>1)&7,
// z = t>>4), so a warp covers two z-slices: 512 contiguous bytes of sdf and
// 128 of weights, fully coalesced 16-byte and 4-byte accesses.
//
// Each voxel runs the listing computeUpdatedVoxelDepthInfo with IEEE
// round-to-nearest operations in the listing's order (no fused multiply-add),
// so the skip decisions, the pixel read and the integer weights are
// reproducible bit for bit.  The decision needs no voxel data: a thread loads
// its 16 bytes of sdf and 4 bytes of weight only when one of its four voxels
// is updated, and stores them back after the update.  Skipped voxels cost no
// HBM traffic.
#include "itm_internal.cuh"

namespace itm {

namespace {

constexpr int kThreads = 128;

template <int MODE>  // 0: constant weight 1, uint8 weights; 1: per-pixel weight, float weights
__global__ void __launch_bounds__(kThreads) integrate_kernel(SceneDev s, const float *__restrict__ depth,
                                                             const float *__restrict__ wpx, Intr in, Mat34 M)
{
    const int n = min(__ldcg(&s.ctr->n_visible), s.nv);
    const int t = threadIdx.x;
    const int lx = (t & 1) * 4, ly = (t >> 1) & 7, lz = t >> 4;
    const float vs = s.voxel_size, mu = s.mu, neg_mu = -s.mu;
    const float umax = (float)(in.W - 2), vmax = (float)(in.H - 2);
    const float max_w = (float)s.max_w;
    unsigned updated = 0;

    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int ptr = __ldg(&s.visible[i]);
        const short4 b = __ldg(&s.block_pos[ptr]);
        const float py = fmul((float)(b.y * 8 + ly), vs);
        const float pz = fmul((float)(b.z * 8 + lz), vs);
        // products that do not depend on x are shared by the thread's four voxels
        const float xy = fmul(M.m[1], py), xz = fmul(M.m[2], pz);
        const float yy = fmul(M.m[5], py), yz = fmul(M.m[6], pz);
        const float zy = fmul(M.m[9], py), zz = fmul(M.m[10], pz);

        float f[4], obs[4];
        unsigned upd = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float px = fmul((float)(b.x * 8 + lx + k), vs);
            const float Z = fadd(fadd(fadd(fmul(M.m[8], px), zy), zz), M.m[11]);
            f[k] = 0.0f;
            obs[k] = 1.0f;
            if (Z <= 0.0f) continue;
            const float X = fadd(fadd(fadd(fmul(M.m[0], px), xy), xz), M.m[3]);
            const float Y = fadd(fadd(fadd(fmul(M.m[4], px), yy), yz), M.m[7]);
            const float u = fadd(fdiv(fmul(in.fx, X), Z), in.cx);
            const float v = fadd(fdiv(fmul(in.fy, Y), Z), in.cy);
            if (u < 1.0f || u > umax || v < 1.0f || v > vmax) continue;
            const int pix = (int)fadd(u, 0.5f) + (int)fadd(v, 0.5f) * in.W;
            const float d = __ldg(&depth[pix]);
            if (!(d > 0.0f)) continue;
            const float eta = fsub(d, Z);
            if (eta < neg_mu) continue;
            if (MODE == 1) {
                obs[k] = __ldg(&wpx[pix]);
                if (!(obs[k] > 0.0f)) continue;
            }
            float fk = fdiv(eta, mu);
            f[k] = fk > 1.0f ? 1.0f : fk;
            upd |= 1u << k;
        }
        if (!upd) continue;
        updated += __popc(upd);

        const size_t base = (size_t)ptr * kBlockVoxels + 4 * t;
        float4 F = __ldcs(reinterpret_cast<const float4 *>(s.sdf + base));
        float Fv[4] = {F.x, F.y, F.z, F.w};
        if (MODE == 0) {
            uint32_t Wp = __ldcs(reinterpret_cast<const uint32_t *>(s.w8 + base));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!(upd & (1u << k))) continue;
                const float oldW = (float)((Wp >> (8 * k)) & 0xffu);
                const float den = fadd(oldW, 1.0f);
                Fv[k] = fdiv(fadd(fmul(oldW, Fv[k]), f[k]), den);
                const float nw = den < max_w ? den : max_w;
                Wp = (Wp & ~(0xffu << (8 * k))) | ((uint32_t)nw << (8 * k));
            }
            __stcs(reinterpret_cast<uint32_t *>(s.w8 + base), Wp);
        } else {
            float4 Wq = __ldcs(reinterpret_cast<const float4 *>(s.w32 + base));
            float Wv[4] = {Wq.x, Wq.y, Wq.z, Wq.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!(upd & (1u << k))) continue;
                const float den = fadd(Wv[k], obs[k]);
                Fv[k] = fdiv(fadd(fmul(Wv[k], Fv[k]), fmul(obs[k], f[k])), den);
                Wv[k] = den < max_w ? den : max_w;
            }
            __stcs(reinterpret_cast<float4 *>(s.w32 + base), make_float4(Wv[0], Wv[1], Wv[2], Wv[3]));
        }
        __stcs(reinterpret_cast<float4 *>(s.sdf + base), make_float4(Fv[0], Fv[1], Fv[2], Fv[3]));
    }

    // counters: one atomic per warp
    for (int o = 16; o > 0; o >>= 1) updated += __shfl_xor_sync(kFull, updated, o);
    if ((t & 31) == 0 && updated) atomicAdd(&s.ctr->updated, (unsigned long long)updated);
    if (blockIdx.x == 0 && t == 0) {
        atomicAdd(&s.ctr->visited, (unsigned long long)n * kBlockVoxels);
        atomicAdd(&s.ctr->frames, 1ull);
    }
}

template <int MODE>
int integrate_grid()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 1, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, integrate_kernel<MODE>, kThreads, 0);
        g = sms * (per > 0 ? per : 1);
    }
    return g;
}

}  // namespace

cudaError_t launch_integrate(const SceneDev &s, const float *depth, const float *wpx, const Intr &in,
                             const Mat34 &M_d, cudaStream_t st)
{
    if (wpx) integrate_kernel<1><<<integrate_grid<1>(), kThreads, 0, st>>>(s, depth, wpx, in, M_d);
    else integrate_kernel<0><<<integrate_grid<0>(), kThreads, 0, st>>>(s, depth, nullptr, in, M_d);
    return cudaGetLastError();
}

}  // namespace itm
