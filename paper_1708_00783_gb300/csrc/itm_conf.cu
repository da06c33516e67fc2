// Learned per-pixel confidence weight (not in the paper; it replaces the
// constant observation weight 1 of the Sec. 4.3 listing, see
// itm_integrate_weighted).
//
// Definitions (the repository's):
//   features x (52): the 7x7 depth patch around the pixel, entry (i, j) for row
//     offset i and column offset j in -3..3 at index (i+3)*7 + (j+3), equal to
//     clamp((D(u+j, v+i) - D(u, v)) / mu, -4, 4) where that pixel is inside the
//     image with depth > 0, else 0; then the unit normal of the back-projected
//     depth, P(u, v) = D(u, v) ((u-cx)/fx, (v-cy)/fy, 1),
//     n = normalise((P(u,v+1) - P(u,v-1)) x (P(u+1,v) - P(u-1,v))), or 0 when a
//     neighbour is outside or has no depth;
//   network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2) (64 each),
//     w_px = sigmoid(w3 . h2 + b3); pixels without depth get w_px = 0;
//   parameters (fp32 master copy, 7617): W1[64][52], b1, W2[64][64], b2, w3, b3.
//
// Inference (conf_weights_kernel): 128-thread CTAs over 16x8-pixel tiles.
// The depth tile and its 3-pixel halo are staged in shared memory and each
// thread writes its pixel's 52 features, rounded to bfloat16 and zero padded
// to 64, as one row of the tile's 128 x 64 A operand.  Both hidden layers are
// 5th-generation tensor-core products (tcgen05.mma, M=128, N=64, K=64, bf16
// operands from shared memory, fp32 accumulators in 64 TMEM columns) issued
// by one thread and completed through an mbarrier.  Each thread reads its
// pixel's accumulator row back from TMEM (its warp's lane quarter), adds the
// bias and applies the ReLU; after layer 1 the rounded row overwrites the
// pixel's A row as layer 2's input, after layer 2 the 64-term output dot
// product and the sigmoid run in fp32 in the same thread.  The packed weights
// sit in shared memory, in the tensor core's canonical layout, for the CTA's
// whole persistent loop.
//
// Training: features of sampled pixels (conf_features_kernel), a per-sample
// forward/backward in fp32 with the same bfloat16-rounded weights and inputs
// as inference (the rounding is taken as the identity for the gradient),
// a gradient reduction over the batch, and Adam on the fp32 master copy.
#include <cuda_bf16.h>

#include <algorithm>

#include "itm_internal.cuh"

namespace itm {

namespace {

constexpr int NF = ITM_MLP_FEATURES, NH = ITM_MLP_HIDDEN, NP = ITM_MLP_PARAMS;
constexpr int P_W1 = 0, P_B1 = NH * NF, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH, P_B3 = P_W3 + NH;
// packed inference layout (bytes)
constexpr size_t kOffW1 = 0, kOffW2 = NH * 64 * 2, kOffB1 = 2 * NH * 64 * 2;
constexpr size_t kOffB2 = kOffB1 + NH * 4, kOffW3 = kOffB2 + NH * 4, kOffB3 = kOffW3 + NH * 4;
static_assert(kOffB3 + 16 == ITM_MLP_PACKED_BYTES, "packed layout");

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- features

struct GlobalDepth {
    const float *D;
    int W, H;
    __device__ float operator()(int u, int v) const
    {
        if (u < 0 || v < 0 || u >= W || v >= H) return 0.0f;
        const float d = __ldg(&D[(size_t)v * W + u]);
        return d > 0.0f ? d : 0.0f;
    }
};

// depth tile with a 3-pixel halo in shared memory; out-of-image entries are 0
struct TileDepth {
    const float *S;
    int u0, v0, stride;
    __device__ float operator()(int u, int v) const { return S[(v - v0 + 3) * stride + (u - u0 + 3)]; }
};

// patch entry k < 49: row offset i = k / 7 - 3, column offset j = k % 7 - 3
template <class Depth>
__device__ __forceinline__ float patch_feature(const Depth &D, int u, int v, float dc, float inv_mu, int k)
{
    const float d = D(u + k % 7 - 3, v + k / 7 - 3);
    return d > 0.0f ? fminf(fmaxf((d - dc) * inv_mu, -4.0f), 4.0f) : 0.0f;
}

// entries 49..51: the unit normal from central differences, or 0; rfx and
// rfy are 1 / fx and 1 / fy
template <class Depth>
__device__ __forceinline__ void normal_feature(const Depth &D, const Intr &in, float rfx, float rfy, int u, int v,
                                               float (&n)[3])
{
    n[0] = n[1] = n[2] = 0.0f;
    const float dl = D(u - 1, v), dr = D(u + 1, v), du = D(u, v - 1), dd = D(u, v + 1);
    if (dl > 0.0f && dr > 0.0f && du > 0.0f && dd > 0.0f) {
        const float xl = ((float)(u - 1) - in.cx) * rfx, xc = ((float)u - in.cx) * rfx;
        const float xr = ((float)(u + 1) - in.cx) * rfx;
        const float yu = ((float)(v - 1) - in.cy) * rfy, yc = ((float)v - in.cy) * rfy;
        const float yd = ((float)(v + 1) - in.cy) * rfy;
        const float ax = dd * xc - du * xc, ay = dd * yd - du * yu, az = dd - du;  // along +v
        const float bx = dr * xr - dl * xl, by = dr * yc - dl * yc, bz = dr - dl;  // along +u
        const float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
        const float l = sqrtf(nx * nx + ny * ny + nz * nz);
        if (l > 0.0f) {
            const float r = 1.0f / l;
            n[0] = nx * r;
            n[1] = ny * r;
            n[2] = nz * r;
        }
    }
}

template <class Depth>
__device__ __forceinline__ bool conf_features(const Depth &D, const Intr &in, float mu, int u, int v, float *x)
{
    const float dc = D(u, v);
#pragma unroll
    for (int k = 0; k < NF; ++k) x[k] = 0.0f;
    if (!(dc > 0.0f)) return false;
    const float inv_mu = 1.0f / mu;
#pragma unroll
    for (int k = 0; k < 49; ++k) x[k] = patch_feature(D, u, v, dc, inv_mu, k);
    float n[3];
    normal_feature(D, in, 1.0f / in.fx, 1.0f / in.fy, u, v, n);
    x[49] = n[0];
    x[50] = n[1];
    x[51] = n[2];
    return true;
}

// --------------------------------------------------------------- inference

constexpr int kTW = 16, kTH = 8, kHW = kTW + 6, kHH = kTH + 6;
constexpr int kSW = 48;  // row stride of a staged depth tile (words; 16 mod 32 banks)
constexpr int kRows = kTW * kTH;  // pixels per tile = rows of the A operand = TMEM lanes
static_assert(kRows == 128 && NH == 64, "one M=128, N=64, K=64 product per layer and tile");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// ---- tcgen05 glue (inline PTX).  Operands sit in shared memory in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// the two core matrices of one K=16 step 128 B apart (leading byte offset),
// consecutive 8-row groups 1024 B apart (stride byte offset).

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of row r, elements 8 kc .. 8 kc + 7, in a 64-wide bf16 operand
__device__ __forceinline__ uint32_t canon_off(int r, int kc) { return (r >> 3) * 1024 + kc * 128 + (r & 7) * 16; }

// shared-memory matrix descriptor: start >> 4, leading and stride byte
// offsets >> 4, bit 46 the descriptor version; base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo = 1024)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 D (bit 4), bf16 A (bits 7-9) and
// B (bits 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NH >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void mma_step(uint32_t tmem, uint64_t ad, uint64_t bd, bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate ? 1u : 0u));
}

// D[128 x 64] (TMEM, fp32) = A[128 x 64] B[64 x 64]^T as four K=16 steps,
// plus, with bias_a, the product of the 128 x 16 tile bias_a and the 64 x 16
// tile bias_b (8-row groups 256 B apart) as a fifth step; completion
// (operands read, D written) arrives on the mbarrier
__device__ __forceinline__ void mma_layer(uint32_t tmem, uint32_t a, uint32_t b, uint32_t bar, uint32_t bias_a = 0,
                                          uint32_t bias_b = 0)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) mma_step(tmem, smem_desc(a + 256 * k), smem_desc(b + 256 * k), k > 0);
    if (bias_a) mma_step(tmem, smem_desc(bias_a, 256), smem_desc(bias_b, 256), true);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

constexpr int kWaitSpins = 1 << 20;

constexpr int kStage = (kHH * kHW + 127) / 128;  // depth values a thread stages per tile

// depth of tile's pixels and their 3-pixel halo, entry i = tid + 128 j of the
// row-major (kTH + 6) x (kTW + 6) patch; 0 outside the image and where D <= 0
__device__ __forceinline__ void fetch_depth(const float *__restrict__ depth, const Intr &in, int tiles_x, int tile,
                                            int tid, float (&pre)[kStage])
{
    const int u0 = (tile % tiles_x) * kTW - 3, v0 = (tile / tiles_x) * kTH - 3;
#pragma unroll
    for (int j = 0; j < kStage; ++j) {
        const int i = tid + 128 * j, u = u0 + i % kHW, v = v0 + i / kHW;
        float d = 0.0f;
        if (i < kHH * kHW && u >= 0 && v >= 0 && u < in.W && v < in.H) d = __ldg(&depth[(size_t)v * in.W + u]);
        pre[j] = d > 0.0f ? d : 0.0f;
    }
}  // try_wait rounds before a wait is given up

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < kWaitSpins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
            " selp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// the warp's 32 lanes x 32 fp32 columns of D from column taddr: thread t of
// warp w gets row 32 w + t
__device__ __forceinline__ void tmem_row32(uint32_t taddr, float (&d)[32])
{
    uint32_t r[32];
#pragma unroll
    for (int c = 0; c < 2; ++c)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[16 * c]), "=r"(r[16 * c + 1]), "=r"(r[16 * c + 2]), "=r"(r[16 * c + 3]), "=r"(r[16 * c + 4]),
              "=r"(r[16 * c + 5]), "=r"(r[16 * c + 6]), "=r"(r[16 * c + 7]), "=r"(r[16 * c + 8]),
              "=r"(r[16 * c + 9]), "=r"(r[16 * c + 10]), "=r"(r[16 * c + 11]), "=r"(r[16 * c + 12]),
              "=r"(r[16 * c + 13]), "=r"(r[16 * c + 14]), "=r"(r[16 * c + 15])
            : "r"(taddr + 16 * c));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // the registers are defined again after the wait, so no use moves above it
#pragma unroll
    for (int c = 0; c < 2; ++c)
        asm volatile(""
                     : "+r"(r[16 * c]), "+r"(r[16 * c + 1]), "+r"(r[16 * c + 2]), "+r"(r[16 * c + 3]),
                       "+r"(r[16 * c + 4]), "+r"(r[16 * c + 5]), "+r"(r[16 * c + 6]), "+r"(r[16 * c + 7]),
                       "+r"(r[16 * c + 8]), "+r"(r[16 * c + 9]), "+r"(r[16 * c + 10]), "+r"(r[16 * c + 11]),
                       "+r"(r[16 * c + 12]), "+r"(r[16 * c + 13]), "+r"(r[16 * c + 14]), "+r"(r[16 * c + 15]));
#pragma unroll
    for (int i = 0; i < 32; ++i) d[i] = __uint_as_float(r[i]);
}

// dynamic shared memory: W1, W2 and two A tiles in the canonical layout, the
// layer-2 bias tiles, then w3, b3 (fp32), two depth tiles with their halo and
// two sets of valid flags (one per tile slot)
constexpr size_t kOffSW1 = 0, kOffSW2 = NH * 64 * 2, kOffSA = 2 * NH * 64 * 2;
constexpr size_t kASize = kRows * 64 * 2;
constexpr size_t kOffSBA = kOffSA + 2 * kASize;          // 128 x 16 bf16: rows [1, 1, 1, 0, ...]
constexpr size_t kOffSBB = kOffSBA + kRows * 16 * 2;     // 64 x 16 bf16: rows [b2 split in three, 0, ...]
constexpr size_t kOffSF = kOffSBB + NH * 16 * 2;         // w3 (64), b3
constexpr size_t kOffSD = kOffSF + (NH + 4) * 4;
constexpr size_t kDSize = kHH * kSW * 4;
constexpr size_t kOffSV = kOffSD + 2 * kDSize;
constexpr size_t kConfSmem = kOffSV + 2 * kRows;
constexpr int kTmemCols = 128;  // two tile slots of 64 fp32 accumulator columns
// at most 4 CTAs per SM (228 KB of shared memory, 1 KB reserved per CTA), so
// their TMEM columns fit the SM's 512 and no allocation waits
static_assert(5 * (kConfSmem + 1024) > 228 * 1024 && 4 * kTmemCols <= 512, "TMEM budget");
static_assert(NF + 3 <= 64, "three bias columns after the features");

// byte offset of row r, elements 8 kc .. 8 kc + 7, in a 16-wide bf16 operand
__device__ __forceinline__ uint32_t canon16_off(int r, int kc) { return (r >> 3) * 256 + kc * 128 + (r & 7) * 16; }

// b = hi + mid + lo with three bf16 values (exact for a normal fp32 b: 8
// significant bits each)
__device__ __forceinline__ void split3_bf16(float b, __nv_bfloat16 (&o)[3])
{
    o[0] = __float2bfloat16_rn(b);
    const float r1 = b - __bfloat162float(o[0]);
    o[1] = __float2bfloat16_rn(r1);
    o[2] = __float2bfloat16_rn(r1 - __bfloat162float(o[1]));
}

// Tile tile's depth and its 3-pixel halo into sD (kHH rows of kHW values,
// row stride kSW); 0 outside the image and where D <= 0.
__device__ __forceinline__ void stage_depth(const float *__restrict__ depth, const Intr &in, int tiles_x, int tile,
                                            int tid, float *sD)
{
    float pre[kStage];
    fetch_depth(depth, in, tiles_x, tile, tid, pre);
#pragma unroll
    for (int j = 0; j < kStage; ++j) {
        const int i = tid + 128 * j;
        if (i < kHH * kHW) sD[(i / kHW) * kSW + i % kHW] = pre[j];
    }
}

// The pixel's 52 features rounded to bf16, then 1, 1, 1 (the inputs of the
// three bias columns of W1) and zeros, as row tid of the A tile at sA;
// returns whether the pixel has depth.
__device__ __forceinline__ bool write_features(const float *sD, const Intr &in, float rfx, float rfy, float inv_mu,
                                               int u0, int v0, int tid, unsigned char *sA)
{
    const int u = u0 + (tid & (kTW - 1)), v = v0 + tid / kTW;
    const TileDepth D{sD, u0, v0, kSW};
    const float dc = D(u, v);
    const bool ok = u < in.W && v < in.H && dc > 0.0f;
    float n[3] = {0.0f, 0.0f, 0.0f};
    if (ok) normal_feature(D, in, rfx, rfy, u, v, n);
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
        float f[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = 8 * kc + q;
            f[q] = k < 49 ? patch_feature(D, u, v, dc, inv_mu, k) : (k < NF ? n[k - 49] : 0.0f);
            if (!ok) f[q] = 0.0f;
            if (k >= NF && k < NF + 3) f[q] = 1.0f;
        }
        *reinterpret_cast<uint4 *>(sA + canon_off(tid, kc)) =
            make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
    }
    return ok;
}

// relu of two accumulators, rounded to bf16 (relu of the rounded value: the
// same, as 0 and the rounding are monotone)
__device__ __forceinline__ uint32_t relu_bf16x2(float a, float b)
{
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    p = __hmax2(p, __float2bfloat162_rn(0.0f));
    return *reinterpret_cast<const uint32_t *>(&p);
}

// One CTA (one warpgroup of 128 threads) runs its tiles t_0, t_1, ... as a
// two-slot software pipeline, so that the tensor core and the threads work at
// the same time:
//
//   features(t_0) -> A0; MMA1(t_0)
//   for each i (slot s = i & 1):
//     features(t_i+1) -> A[s^1]            while MMA1(t_i) runs
//     wait MMA1(t_i); h1 = relu(acc) -> A[s]
//     MMA2(t_i) -> TMEM slot s; MMA1(t_i+1) -> TMEM slot s^1
//     wait MMA2(t_i); output of t_i       while MMA1(t_i+1) runs
//
// Both biases are added by the tensor core: b1 through three extra columns
// of W1 (its bf16 split) against inputs of 1, b2 through a fifth K=16 step
// of a constant tile of ones against b2's split.  MMA1 completions arrive on
// bar1, MMA2 completions on bar2 (one phase per tile each).  One thread waits
// on each (a bounded number of polls) while the others sit at a barrier; a
// wait that gives up sends the CTA to its failure path: NaN weights for its
// remaining pixels (weighted integration skips them), one more bounded wait
// for each product in flight, then the TMEM is freed.
__global__ void __launch_bounds__(128) conf_weights_kernel(const float *__restrict__ depth, Intr in, float mu,
                                                           const unsigned char *__restrict__ packed,
                                                           float *__restrict__ wpx, int tiles_x, int n_tiles)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    const float *sW3 = reinterpret_cast<const float *>(smem + kOffSF);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = smem_addr(smem), bar1 = smem_addr(&bar[0]), bar2 = smem_addr(&bar[1]);
    auto sA = [&](int slot) { return smem + kOffSA + slot * kASize; };
    auto sD = [&](int slot) { return reinterpret_cast<float *>(smem + kOffSD + slot * kDSize); };
    auto sValid = [&](int slot) { return smem + kOffSV + slot * kRows; };
    const float rfx = 1.0f / in.fx, rfy = 1.0f / in.fy, inv_mu = 1.0f / mu;
    const int stride = (int)gridDim.x;
    const int t0 = blockIdx.x;

    {
        // weights: 16-byte chunks of the row-major 64 x 64 matrices
        const uint4 *W = reinterpret_cast<const uint4 *>(packed + kOffW1);
        for (int j = tid; j < 2 * NH * 8; j += 128) {
            const int m = j >> 9, n = (j >> 3) & 63, kc = j & 7;
            *reinterpret_cast<uint4 *>(smem + (m ? kOffSW2 : kOffSW1) + canon_off(n, kc)) = __ldg(&W[j]);
        }
        const float *f32 = reinterpret_cast<const float *>(packed + kOffB1);  // b1, b2, w3, b3
        float *dst = reinterpret_cast<float *>(smem + kOffSF);
        for (int i = tid; i < NH + 1; i += 128) dst[i] = f32[2 * NH + i];
        __syncthreads();  // W1's chunks are in place before their bias columns are written
        if (tid < NH) {
            // b1 into W1's columns NF .. NF+2 (bf16 split), b2 into the bias tile
            __nv_bfloat16 h[3];
            split3_bf16(f32[tid], h);
            __nv_bfloat16 *w1row = reinterpret_cast<__nv_bfloat16 *>(smem + kOffSW1 + canon_off(tid, NF / 8));
            for (int q = 0; q < 3; ++q) w1row[NF % 8 + q] = h[q];
            split3_bf16(f32[NH + tid], h);
            __nv_bfloat16 bb[8] = {h[0], h[1], h[2]};
            for (int q = 3; q < 8; ++q) bb[q] = __float2bfloat16_rn(0.0f);
            *reinterpret_cast<uint4 *>(smem + kOffSBB + canon16_off(tid, 0)) = *reinterpret_cast<const uint4 *>(bb);
            *reinterpret_cast<uint4 *>(smem + kOffSBB + canon16_off(tid, 1)) = make_uint4(0u, 0u, 0u, 0u);
        }
        // the constant tile: every row [1, 1, 1, 0, ...]
        const uint32_t one = 0x3F80u;  // bf16 1.0
        *reinterpret_cast<uint4 *>(smem + kOffSBA + canon16_off(tid, 0)) =
            make_uint4(one | (one << 16), one, 0u, 0u);
        *reinterpret_cast<uint4 *>(smem + kOffSBA + canon16_off(tid, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar2) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the first tile's depth and features
    stage_depth(depth, in, tiles_x, t0, tid, sD(0));
    __syncthreads();
    sValid(0)[tid] = write_features(sD(0), in, rfx, rfy, inv_mu, (t0 % tiles_x) * kTW, (t0 / tiles_x) * kTH, tid,
                                    sA(0));
    async_proxy_fence();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;  // this warp's TMEM lane quarter
    if (tid == 0) mma_layer(tmem, sbase + kOffSA, sbase + kOffSW1, bar1);

    // products issued and completions consumed on each barrier (thread 0's
    // counts, for the final wait after a failure)
    int issued1 = 1, issued2 = 0, done1 = 0, done2 = 0;
    int fail_from = -1;  // first tile whose output was not written
    int i = 0;
    for (int t = t0; t < n_tiles; t += stride, ++i) {
        const int s = i & 1, tn = t + stride;
        const bool has_next = tn < n_tiles;
        const int u0 = (t % tiles_x) * kTW, v0 = (t / tiles_x) * kTH;
        // the next tile's features while this tile's first product runs
        if (has_next) {
            stage_depth(depth, in, tiles_x, tn, tid, sD(s ^ 1));
            asm volatile("bar.sync 1, 128;" ::: "memory");
            sValid(s ^ 1)[tid] = write_features(sD(s ^ 1), in, rfx, rfy, inv_mu, (tn % tiles_x) * kTW,
                                                (tn / tiles_x) * kTH, tid, sA(s ^ 1));
        }
        bool ok = true;
        if (tid == 0) {
            ok = mbar_wait(bar1, (uint32_t)(done1 & 1));
            done1 += ok;
        }
        if (__syncthreads_or(!ok)) {
            fail_from = t;
            break;
        }
        tc_after_sync();
        // h1 = bf16(relu(acc)) is layer 2's A tile, in place of x
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float h[32];
            tmem_row32(tmem + lane_off + 64 * s + 32 * half, h);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const int j = 8 * kc;
                *reinterpret_cast<uint4 *>(sA(s) + canon_off(tid, 4 * half + kc)) =
                    make_uint4(relu_bf16x2(h[j], h[j + 1]), relu_bf16x2(h[j + 2], h[j + 3]),
                               relu_bf16x2(h[j + 4], h[j + 5]), relu_bf16x2(h[j + 6], h[j + 7]));
            }
        }
        async_proxy_fence();
        tc_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc_after_sync();
            mma_layer(tmem + 64 * s, sbase + kOffSA + s * kASize, sbase + kOffSW2, bar2, sbase + kOffSBA,
                      sbase + kOffSBB);
            ++issued2;
            if (has_next) {
                mma_layer(tmem + 64 * (s ^ 1), sbase + kOffSA + (s ^ 1) * kASize, sbase + kOffSW1, bar1);
                ++issued1;
            }
            ok = mbar_wait(bar2, (uint32_t)(done2 & 1));
            done2 += ok;
        }
        if (__syncthreads_or(!ok)) {
            fail_from = t;
            break;
        }
        tc_after_sync();
        {
            // w_px = sigmoid(w3 . relu(h2) + b3), h2 = acc (b2 added by the product)
            float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float h[32];
                tmem_row32(tmem + lane_off + 64 * s + 32 * half, h);
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 w = *reinterpret_cast<const float4 *>(sW3 + 32 * half + j);
                    acc = __ffma2_rn(make_float2(w.x, w.y), make_float2(fmaxf(h[j], 0.0f), fmaxf(h[j + 1], 0.0f)), acc);
                    acc = __ffma2_rn(make_float2(w.z, w.w), make_float2(fmaxf(h[j + 2], 0.0f), fmaxf(h[j + 3], 0.0f)),
                                     acc);
                }
            }
            const float o = acc.x + acc.y + sW3[NH];
            const int u = u0 + (tid & (kTW - 1)), v = v0 + tid / kTW;
            if (u < in.W && v < in.H) wpx[(size_t)v * in.W + u] = sValid(s)[tid] ? 1.0f / (1.0f + expf(-o)) : 0.0f;
        }
        tc_before_sync();  // this tile's TMEM reads come before later products into its slot
        __syncthreads();
    }
    if (fail_from >= 0) {
        // NaN weights for the CTA's pixels from the failed tile on; one more
        // bounded wait for each product still in flight
        for (int t = fail_from; t < n_tiles; t += stride) {
            const int u = (t % tiles_x) * kTW + (tid & (kTW - 1)), v = (t / tiles_x) * kTH + tid / kTW;
            if (u < in.W && v < in.H) wpx[(size_t)v * in.W + u] = __int_as_float(0x7fc00000);
        }
        if (tid == 0) {
            for (; done1 < issued1; ++done1)
                if (!mbar_wait(bar1, (uint32_t)(done1 & 1))) break;
            for (; done2 < issued2; ++done2)
                if (!mbar_wait(bar2, (uint32_t)(done2 & 1))) break;
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------- training

__global__ void pack_kernel(const float *__restrict__ P, unsigned char *__restrict__ packed)
{
    __nv_bfloat16 *W1p = reinterpret_cast<__nv_bfloat16 *>(packed + kOffW1);
    __nv_bfloat16 *W2p = reinterpret_cast<__nv_bfloat16 *>(packed + kOffW2);
    float *f32 = reinterpret_cast<float *>(packed + kOffB1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH * 64; i += gridDim.x * blockDim.x) {
        const int n = i >> 6, k = i & 63;
        W1p[i] = __float2bfloat16_rn(k < NF ? P[P_W1 + n * NF + k] : 0.0f);
        W2p[i] = __float2bfloat16_rn(P[P_W2 + i]);
        if (i < NH) {
            f32[i] = P[P_B1 + i];
            f32[NH + i] = P[P_B2 + i];
            f32[2 * NH + i] = P[P_W3 + i];
        }
        if (i == 0) {
            f32[3 * NH] = P[P_B3];
            f32[3 * NH + 1] = f32[3 * NH + 2] = f32[3 * NH + 3] = 0.0f;
        }
    }
}

__global__ void conf_features_kernel(const float *__restrict__ depth, Intr in, float mu, const int32_t *__restrict__ pix,
                                     int n, float *__restrict__ feat)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int p = pix[s];
    float x[NF];
    const GlobalDepth D{depth, in.W, in.H};
    if (p >= 0 && p < in.W * in.H) conf_features(D, in, mu, p % in.W, p / in.W, x);
    else
        for (int k = 0; k < NF; ++k) x[k] = 0.0f;
    for (int k = 0; k < NF; ++k) feat[(size_t)s * NF + k] = x[k];
}

// scratch per sample: h1 (bf16-rounded), h2, d2, d1 (64 each), dout
constexpr int kSH1 = 0, kSH2 = 64, kSD2 = 128, kSD1 = 192, kSDO = 256, kSRow = ITM_MLP_SCRATCH_PER_SAMPLE;

__global__ void __launch_bounds__(128) mlp_fwd_bwd_kernel(const float *__restrict__ P, const float *__restrict__ feat,
                                                          const float *__restrict__ y, int n,
                                                          float *__restrict__ scratch, float *__restrict__ loss)
{
    __shared__ float sW1[NH * NF], sW2[NH * NH], sB1[NH], sB2[NH], sW3[NH], sB3;
    __shared__ float sLoss[4];
    for (int i = threadIdx.x; i < NH * NF; i += blockDim.x) sW1[i] = bf16r(P[P_W1 + i]);
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) sW2[i] = bf16r(P[P_W2 + i]);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        sB1[i] = P[P_B1 + i];
        sB2[i] = P[P_B2 + i];
        sW3[i] = P[P_W3 + i];
    }
    if (threadIdx.x == 0) sB3 = P[P_B3];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (s < n) {
        float *row = scratch + (size_t)s * kSRow;
        float x[NF];
        for (int k = 0; k < NF; ++k) x[k] = bf16r(feat[(size_t)s * NF + k]);
        for (int m = 0; m < NH; ++m) {
            float a = sB1[m];
            for (int k = 0; k < NF; ++k) a = fmaf(sW1[m * NF + k], x[k], a);
            row[kSH1 + m] = bf16r(fmaxf(a, 0.0f));  // as consumed by layer 2; 0 where the ReLU is off
        }
        float o = sB3;
        for (int a = 0; a < NH; ++a) {
            float acc = sB2[a];
            for (int m = 0; m < NH; ++m) acc = fmaf(sW2[a * NH + m], row[kSH1 + m], acc);
            const float h2 = fmaxf(acc, 0.0f);
            row[kSH2 + a] = h2;
            o = fmaf(sW3[a], h2, o);
        }
        const float t = y[s];
        const float p = 1.0f / (1.0f + expf(-o));
        l = fmaxf(o, 0.0f) - o * t + log1pf(expf(-fabsf(o)));
        const float dout = (p - t) / (float)n;
        row[kSDO] = dout;
        for (int a = 0; a < NH; ++a) row[kSD2 + a] = row[kSH2 + a] > 0.0f ? dout * sW3[a] : 0.0f;
        for (int m = 0; m < NH; ++m) {
            float acc = 0.0f;
            for (int a = 0; a < NH; ++a) acc = fmaf(sW2[a * NH + m], row[kSD2 + a], acc);
            row[kSD1 + m] = row[kSH1 + m] > 0.0f ? acc : 0.0f;
        }
    }
    // loss: warp sums, one atomic per CTA
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(kFull, l, o);
    if ((threadIdx.x & 31) == 0) sLoss[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(loss, (sLoss[0] + sLoss[1] + sLoss[2] + sLoss[3]) / (float)n);
}

// one thread per parameter, summing its gradient over the batch
__global__ void mlp_grad_kernel(const float *__restrict__ feat, const float *__restrict__ scratch, int n,
                                float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    float acc = 0.0f;
    if (i < P_B1) {
        const int m = i / NF, k = i % NF;
        for (int s = 0; s < n; ++s) acc = fmaf(scratch[(size_t)s * kSRow + kSD1 + m], bf16r(feat[(size_t)s * NF + k]), acc);
    } else if (i < P_W2) {
        const int m = i - P_B1;
        for (int s = 0; s < n; ++s) acc += scratch[(size_t)s * kSRow + kSD1 + m];
    } else if (i < P_B2) {
        const int a = (i - P_W2) / NH, m = (i - P_W2) % NH;
        for (int s = 0; s < n; ++s)
            acc = fmaf(scratch[(size_t)s * kSRow + kSD2 + a], scratch[(size_t)s * kSRow + kSH1 + m], acc);
    } else if (i < P_W3) {
        const int a = i - P_B2;
        for (int s = 0; s < n; ++s) acc += scratch[(size_t)s * kSRow + kSD2 + a];
    } else if (i < P_B3) {
        const int a = i - P_W3;
        for (int s = 0; s < n; ++s) acc = fmaf(scratch[(size_t)s * kSRow + kSDO], scratch[(size_t)s * kSRow + kSH2 + a], acc);
    } else {
        for (int s = 0; s < n; ++s) acc += scratch[(size_t)s * kSRow + kSDO];
    }
    grad[i] = acc;
}

__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// CTAs of conf_weights_kernel resident per SM, counted from its registers,
// shared memory and TMEM columns (the runtime's occupancy calculator answers
// one CTA per SM for this kernel), times the SM count
int conf_grid()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 1, regs_sm = 65536, smem_sm = 0, reserved = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, conf_weights_kernel);
        const int regs_cta = (fa.numRegs + 7) / 8 * 8 * 128;  // registers are allocated 256 per warp
        int per = 512 / kTmemCols;
        if (regs_cta > 0) per = std::min(per, regs_sm / regs_cta);
        per = std::min(per, (int)(smem_sm / (kConfSmem + fa.sharedSizeBytes + (size_t)reserved)));
        g = sms * std::max(per, 1);
    }
    return g;
}

}  // namespace

}  // namespace itm

using namespace itm;

extern "C" {

int itm_mlp_pack(const float *params_dev, void *packed_dev, itm_stream stream)
{
    if (!params_dev || !packed_dev || (reinterpret_cast<uintptr_t>(packed_dev) & 15)) return ITM_ERR_ARG;
    pack_kernel<<<16, 256, 0, (cudaStream_t)stream>>>(params_dev, static_cast<unsigned char *>(packed_dev));
    return check_cuda(cudaGetLastError());
}

int itm_conf_weights(const float *depth_dev, const itm_intrinsics *intr, float mu, const void *packed_dev,
                     float *wpx_dev, itm_stream stream)
{
    if (!depth_dev || !packed_dev || !wpx_dev || !valid_intr(intr) || !(mu > 0.0f)) return ITM_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed_dev) & 15) return ITM_ERR_ARG;
    const int tx = (intr->width + kTW - 1) / kTW, ty = (intr->height + kTH - 1) / kTH;
    const int n_tiles = tx * ty;
    static const cudaError_t attr =
        cudaFuncSetAttribute(conf_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConfSmem);
    if (attr != cudaSuccess) return check_cuda(attr);
    int grid = conf_grid();
    if (grid > n_tiles) grid = n_tiles;
    conf_weights_kernel<<<grid, 128, kConfSmem, (cudaStream_t)stream>>>(
        depth_dev, to_intr(intr), mu, static_cast<const unsigned char *>(packed_dev), wpx_dev, tx, n_tiles);
    return check_cuda(cudaGetLastError());
}

int itm_conf_features(const float *depth_dev, const itm_intrinsics *intr, float mu, const int32_t *pixels_dev, int n,
                      float *feat_dev, itm_stream stream)
{
    if (n < 0 || (n > 0 && (!depth_dev || !pixels_dev || !feat_dev)) || !valid_intr(intr) || !(mu > 0.0f))
        return ITM_ERR_ARG;
    if (n == 0) return ITM_OK;
    conf_features_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(depth_dev, to_intr(intr), mu, pixels_dev,
                                                                            n, feat_dev);
    return check_cuda(cudaGetLastError());
}

int itm_mlp_loss_grad(const float *params_dev, const float *feat_dev, const float *labels_dev, int n,
                      float *scratch_dev, float *grad_dev, float *loss_dev, itm_stream stream)
{
    if (n <= 0 || !params_dev || !feat_dev || !labels_dev || !scratch_dev || !grad_dev || !loss_dev) return ITM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(float), st);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    mlp_fwd_bwd_kernel<<<(n + 127) / 128, 128, 0, st>>>(params_dev, feat_dev, labels_dev, n, scratch_dev, loss_dev);
    mlp_grad_kernel<<<(NP + 127) / 128, 128, 0, st>>>(feat_dev, scratch_dev, n, grad_dev);
    return check_cuda(cudaGetLastError());
}

int itm_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int step, float lr,
                 itm_stream stream)
{
    if (!params_dev || !grad_dev || !m_dev || !v_dev || step < 1 || !(lr > 0.0f)) return ITM_ERR_ARG;
    const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    adam_kernel<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params_dev, grad_dev, m_dev, v_dev, lr, c1, c2);
    return check_cuda(cudaGetLastError());
}

}  // extern "C"
