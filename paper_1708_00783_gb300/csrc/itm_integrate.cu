// Sec. 4.3 integration over the visible blocks.
//
// Launch shape: a persistent grid of 64-thread CTAs walks the visible list
// (its length is read from device memory).  A CTA takes one 8^3 block per
// iteration; thread t owns the x-row of voxels 8t .. 8t+7 (y = t & 7,
// z = t >> 3): 32 contiguous bytes of sdf and 8 of weights, so each warp
// covers four z-slices with fully coalesced 16-byte accesses.  The next
// block's index and coordinates are fetched while the current one is
// processed.
//
// Each voxel runs the listing computeUpdatedVoxelDepthInfo with IEEE
// round-to-nearest operations in the listing's order (no fused multiply-add,
// correctly rounded divisions), so the skip decisions, the pixel read, the
// weights and the sdf values are reproducible bit for bit.  The thread first
// projects its eight voxels (no memory access), then issues their eight depth
// reads together, then takes the update decisions: the reads overlap instead
// of waiting on each other.  (Evaluating the projection with an approximate
// reciprocal plus an exact fallback near decision boundaries measured no
// faster: the kernel is bound by instruction issue across the whole voxel
// update, not by the divisions.  The packed f32x2 add/multiply of sm_100+ was
// also tried: in this broadcast-operand chain it did not reproduce the
// separately rounded scalar results.)  Small integers move between int and
// float through the 2^23 mantissa trick (exact for 0 <= n < 2^23) instead of
// conversion instructions.
//
// The decision needs no voxel data: a thread loads a 16-byte quad of sdf
// only when one of its four voxels is updated (and its 8 bytes of weights
// when any of its eight is), and stores it back after the update.  Skipped
// voxels cost no HBM traffic.
#include "itm_internal.cuh"

namespace itm {

namespace {

constexpr int kThreads = 64;

// exact small-integer <-> float through the float whose mantissa holds n
constexpr float kMagic = 8388608.0f;  // 2^23
__device__ __forceinline__ float u8_to_f(uint32_t n) { return __fsub_rn(__uint_as_float(0x4B000000u | n), kMagic); }
__device__ __forceinline__ uint32_t f_to_u8(float w) { return __float_as_uint(__fadd_rn(w, kMagic)) & 0xffu; }

template <int MODE>  // 0: constant weight 1, uint8 weights; 1: per-pixel weight, float weights
__global__ void __launch_bounds__(kThreads) integrate_kernel(SceneDev s, const float *__restrict__ depth,
                                                             const float *__restrict__ wpx, Intr in, Mat34 M)
{
    const int n = min(__ldcg(&s.ctr->n_visible), s.nv);
    const int t = threadIdx.x;
    const int ly = t & 7, lz = t >> 3;
    const float vs = s.voxel_size, neg_mu = -s.mu;
    const float umax = (float)(in.W - 2), vmax = (float)(in.H - 2);
    const float max_w = (float)s.max_w;
    unsigned updated = 0;

    int i = blockIdx.x;
    int ptr = 0;
    short4 b = make_short4(0, 0, 0, 0);
    if (i < n) {
        ptr = __ldg(&s.visible[i]);
        b = __ldg(&s.block_pos[ptr]);
    }
    while (i < n) {
        // prefetch the next block's index and coordinates
        const int i_next = i + gridDim.x;
        int ptr_next = 0;
        if (i_next < n) ptr_next = __ldg(&s.visible[i_next]);

        const float py = fmul((float)(b.y * 8 + ly), vs);
        const float pz = fmul((float)(b.z * 8 + lz), vs);
        const float xy = fmul(M.m[1], py), xz = fmul(M.m[2], pz);
        const float yy = fmul(M.m[5], py), yz = fmul(M.m[6], pz);
        const float zy = fmul(M.m[9], py), zz = fmul(M.m[10], pz);
        const float gx0 = (float)(b.x * 8);

        // phase 1: projection and pixel of each voxel (no memory access)
        float Zk[8];
        int pix[8];
        unsigned valid = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            pix[k] = 0;
            // (float)(8 b.x + k) is exact, so is gx0 + k
            const float px = fmul(fadd(gx0, (float)k), vs);
            const float Z = fadd(fadd(fadd(fmul(M.m[8], px), zy), zz), M.m[11]);
            Zk[k] = Z;
            if (Z <= 0.0f) continue;
            const float X = fadd(fadd(fadd(fmul(M.m[0], px), xy), xz), M.m[3]);
            const float Y = fadd(fadd(fadd(fmul(M.m[4], px), yy), yz), M.m[7]);
            const float ax = fmul(in.fx, X), ay = fmul(in.fy, Y);
            const float u = fadd(fdiv(ax, Z), in.cx);
            const float v = fadd(fdiv(ay, Z), in.cy);
            if (u < 1.0f || u > umax || v < 1.0f || v > vmax) continue;
            pix[k] = (int)fadd(u, 0.5f) + (int)fadd(v, 0.5f) * in.W;
            valid |= 1u << k;
        }
        // phase 2: the thread's depth reads, issued together
        float dk[8], ok_obs[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            dk[k] = (valid & (1u << k)) ? __ldg(&depth[pix[k]]) : 0.0f;
            if (MODE == 1) ok_obs[k] = (valid & (1u << k)) ? __ldg(&wpx[pix[k]]) : 0.0f;
        }
        // phase 3: the update decision and the new observation
        float f[8], obs[8];
        unsigned upd = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            f[k] = 0.0f;
            obs[k] = 1.0f;
            if (!(valid & (1u << k))) continue;
            if (!(dk[k] > 0.0f)) continue;
            const float eta = fsub(dk[k], Zk[k]);
            if (eta < neg_mu) continue;
            if (MODE == 1) {
                obs[k] = ok_obs[k];
                if (!(obs[k] > 0.0f)) continue;
            }
            const float fk = fdiv(eta, s.mu);
            f[k] = fk > 1.0f ? 1.0f : fk;
            upd |= 1u << k;
        }
        if (i_next < n) b = __ldg(&s.block_pos[ptr_next]);

        if (upd) {
            updated += __popc(upd);
            const size_t base = (size_t)ptr * kBlockVoxels + 8 * t;
            float4 *F4 = reinterpret_cast<float4 *>(s.sdf + base);
            float Fv[8];
            if (upd & 0x0fu) {
                const float4 a = __ldcs(F4);
                Fv[0] = a.x; Fv[1] = a.y; Fv[2] = a.z; Fv[3] = a.w;
            }
            if (upd & 0xf0u) {
                const float4 a = __ldcs(F4 + 1);
                Fv[4] = a.x; Fv[5] = a.y; Fv[6] = a.z; Fv[7] = a.w;
            }
            if (MODE == 0) {
                uint2 Wp = __ldcs(reinterpret_cast<const uint2 *>(s.w8 + base));
                uint32_t wlo = Wp.x, whi = Wp.y;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (!(upd & (1u << k))) continue;
                    uint32_t &wr = (k < 4) ? wlo : whi;
                    const int sh = 8 * (k & 3);
                    const float oldW = u8_to_f((wr >> sh) & 0xffu);
                    const float den = fadd(oldW, 1.0f);
                    Fv[k] = fdiv(fadd(fmul(oldW, Fv[k]), f[k]), den);
                    const float nw = den < max_w ? den : max_w;
                    wr = (wr & ~(0xffu << sh)) | (f_to_u8(nw) << sh);
                }
                __stcs(reinterpret_cast<uint2 *>(s.w8 + base), make_uint2(wlo, whi));
            } else {
                float4 *W4 = reinterpret_cast<float4 *>(s.w32 + base);
                float Wv[8];
                if (upd & 0x0fu) {
                    const float4 a = __ldcs(W4);
                    Wv[0] = a.x; Wv[1] = a.y; Wv[2] = a.z; Wv[3] = a.w;
                }
                if (upd & 0xf0u) {
                    const float4 a = __ldcs(W4 + 1);
                    Wv[4] = a.x; Wv[5] = a.y; Wv[6] = a.z; Wv[7] = a.w;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (!(upd & (1u << k))) continue;
                    const float den = fadd(Wv[k], obs[k]);
                    Fv[k] = fdiv(fadd(fmul(Wv[k], Fv[k]), fmul(obs[k], f[k])), den);
                    Wv[k] = den < max_w ? den : max_w;
                }
                if (upd & 0x0fu) __stcs(W4, make_float4(Wv[0], Wv[1], Wv[2], Wv[3]));
                if (upd & 0xf0u) __stcs(W4 + 1, make_float4(Wv[4], Wv[5], Wv[6], Wv[7]));
            }
            if (upd & 0x0fu) __stcs(F4, make_float4(Fv[0], Fv[1], Fv[2], Fv[3]));
            if (upd & 0xf0u) __stcs(F4 + 1, make_float4(Fv[4], Fv[5], Fv[6], Fv[7]));
        }
        i = i_next;
        ptr = ptr_next;
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
