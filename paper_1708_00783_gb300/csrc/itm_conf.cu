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
// The depth tile and its 3-pixel halo are staged in shared memory, each
// thread writes its pixel's 52 features as bfloat16 into a 128x64 A tile
// (zero padded), and each warp multiplies its 32 pixels through both layers
// on the tensor cores (mma.sync m16n8k16, bf16 operands, fp32 accumulation).
// The fp32 accumulators of layer 1 are exactly the A fragments of layer 2
// after bias, ReLU and rounding to bfloat16, so h1 never leaves registers.
// The 64-wide dot product of layer 3 runs in fp32 with two shuffles.  The
// packed weights (bf16 W1 padded to 64x64, bf16 W2, fp32 biases and w3) sit
// in shared memory for the CTA's whole persistent loop.
//
// Training: features of sampled pixels (conf_features_kernel), a per-sample
// forward/backward in fp32 with the same bfloat16-rounded weights and inputs
// as inference (the rounding is taken as the identity for the gradient),
// a gradient reduction over the batch, and Adam on the fp32 master copy.
#include <cuda_bf16.h>

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

template <class Depth>
__device__ __forceinline__ bool conf_features(const Depth &D, const Intr &in, float mu, int u, int v, float *x)
{
    const float dc = D(u, v);
#pragma unroll
    for (int k = 0; k < NF; ++k) x[k] = 0.0f;
    if (!(dc > 0.0f)) return false;
    const float inv_mu = 1.0f / mu;
#pragma unroll
    for (int i = -3; i <= 3; ++i)
#pragma unroll
        for (int j = -3; j <= 3; ++j) {
            const float d = D(u + j, v + i);
            float f = 0.0f;
            if (d > 0.0f) f = fminf(fmaxf((d - dc) * inv_mu, -4.0f), 4.0f);
            x[(i + 3) * 7 + (j + 3)] = f;
        }
    const float dl = D(u - 1, v), dr = D(u + 1, v), du = D(u, v - 1), dd = D(u, v + 1);
    if (dl > 0.0f && dr > 0.0f && du > 0.0f && dd > 0.0f) {
        const float Plx = dl * ((float)(u - 1) - in.cx) / in.fx, Ply = dl * ((float)v - in.cy) / in.fy;
        const float Prx = dr * ((float)(u + 1) - in.cx) / in.fx, Pry = dr * ((float)v - in.cy) / in.fy;
        const float Pux = du * ((float)u - in.cx) / in.fx, Puy = du * ((float)(v - 1) - in.cy) / in.fy;
        const float Pdx = dd * ((float)u - in.cx) / in.fx, Pdy = dd * ((float)(v + 1) - in.cy) / in.fy;
        const float ax = Pdx - Pux, ay = Pdy - Puy, az = dd - du;  // along +v
        const float bx = Prx - Plx, by = Pry - Ply, bz = dr - dl;  // along +u
        const float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
        const float l = sqrtf(nx * nx + ny * ny + nz * nz);
        if (l > 0.0f) {
            x[49] = nx / l;
            x[50] = ny / l;
            x[51] = nz / l;
        }
    }
    return true;
}

// --------------------------------------------------------------- inference

constexpr int kTW = 16, kTH = 8, kHW = kTW + 6, kHH = kTH + 6;
constexpr int kStride = 72;  // bf16 per shared-memory row (64 + 8 pad: conflict-free fragment loads)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr size_t kConfSmem = (size_t)(2 * NH + kTW * kTH) * kStride * 2 + (3 * NH + 4) * 4 + kHH * kHW * 4 + 128;

__global__ void __launch_bounds__(128) conf_weights_kernel(const float *__restrict__ depth, Intr in, float mu,
                                                           const unsigned char *__restrict__ packed,
                                                           float *__restrict__ wpx, int tiles_x, int n_tiles)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *sW1 = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sW2 = sW1 + NH * kStride;
    __nv_bfloat16 *sA = sW2 + NH * kStride;
    float *sB1 = reinterpret_cast<float *>(sA + kTW * kTH * kStride);
    float *sB2 = sB1 + NH, *sW3 = sB2 + NH, *sB3 = sW3 + NH;
    float *sD = sB3 + 4;
    unsigned char *sValid = reinterpret_cast<unsigned char *>(sD + kHH * kHW);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    {
        const __nv_bfloat16 *W1p = reinterpret_cast<const __nv_bfloat16 *>(packed + kOffW1);
        const __nv_bfloat16 *W2p = reinterpret_cast<const __nv_bfloat16 *>(packed + kOffW2);
        for (int i = tid; i < NH * 64; i += 128) {
            sW1[(i >> 6) * kStride + (i & 63)] = W1p[i];
            sW2[(i >> 6) * kStride + (i & 63)] = W2p[i];
        }
        const float *f32 = reinterpret_cast<const float *>(packed + kOffB1);
        for (int i = tid; i < 3 * NH + 1; i += 128) sB1[i] = f32[i];  // b1, b2, w3, b3 are contiguous
    }
    __syncthreads();

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int u0 = (tile % tiles_x) * kTW, v0 = (tile / tiles_x) * kTH;
        for (int i = tid; i < kHH * kHW; i += 128) {
            const int u = u0 + (i % kHW) - 3, v = v0 + (i / kHW) - 3;
            float d = 0.0f;
            if (u >= 0 && v >= 0 && u < in.W && v < in.H) {
                d = __ldg(&depth[(size_t)v * in.W + u]);
                if (!(d > 0.0f)) d = 0.0f;
            }
            sD[i] = d;
        }
        __syncthreads();
        {
            const int u = u0 + (tid & (kTW - 1)), v = v0 + tid / kTW;
            float x[NF];
            const TileDepth D{sD, u0, v0, kHW};
            const bool ok = (u < in.W && v < in.H) && conf_features(D, in, mu, u, v, x);
            sValid[tid] = ok;
            uint32_t *row = reinterpret_cast<uint32_t *>(sA + tid * kStride);
#pragma unroll
            for (int k = 0; k < 32; ++k) row[k] = (2 * k + 1 < NF) ? pack_bf16(x[2 * k], x[2 * k + 1]) : 0u;
        }
        __syncthreads();

#pragma unroll 1
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = warp * 32 + mt * 16;
            float acc[8][4];
#pragma unroll
            for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
            const uint32_t *A = reinterpret_cast<const uint32_t *>(sA);
            const uint32_t *B1 = reinterpret_cast<const uint32_t *>(sW1);
            const uint32_t *B2 = reinterpret_cast<const uint32_t *>(sW2);
            constexpr int RW = kStride / 2;  // 32-bit words per row
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t a0 = A[(r0 + g) * RW + kk * 8 + t4], a1 = A[(r0 + g + 8) * RW + kk * 8 + t4];
                const uint32_t a2 = A[(r0 + g) * RW + kk * 8 + 4 + t4], a3 = A[(r0 + g + 8) * RW + kk * 8 + 4 + t4];
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    const uint32_t b0 = B1[(n * 8 + g) * RW + kk * 8 + t4], b1 = B1[(n * 8 + g) * RW + kk * 8 + 4 + t4];
                    mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
                }
            }
            // bias + ReLU + bf16: the accumulators become layer-2 A fragments
            uint32_t h[4][4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int c0 = (2 * kk) * 8 + 2 * t4, c1 = (2 * kk + 1) * 8 + 2 * t4;
                h[kk][0] = pack_bf16(fmaxf(acc[2 * kk][0] + sB1[c0], 0.f), fmaxf(acc[2 * kk][1] + sB1[c0 + 1], 0.f));
                h[kk][1] = pack_bf16(fmaxf(acc[2 * kk][2] + sB1[c0], 0.f), fmaxf(acc[2 * kk][3] + sB1[c0 + 1], 0.f));
                h[kk][2] =
                    pack_bf16(fmaxf(acc[2 * kk + 1][0] + sB1[c1], 0.f), fmaxf(acc[2 * kk + 1][1] + sB1[c1 + 1], 0.f));
                h[kk][3] =
                    pack_bf16(fmaxf(acc[2 * kk + 1][2] + sB1[c1], 0.f), fmaxf(acc[2 * kk + 1][3] + sB1[c1 + 1], 0.f));
            }
#pragma unroll
            for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    const uint32_t b0 = B2[(n * 8 + g) * RW + kk * 8 + t4], b1 = B2[(n * 8 + g) * RW + kk * 8 + 4 + t4];
                    mma_bf16(acc[n], h[kk][0], h[kk][1], h[kk][2], h[kk][3], b0, b1);
                }
            }
            float olo = 0.0f, ohi = 0.0f;
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int c = n * 8 + 2 * t4;
                olo += sW3[c] * fmaxf(acc[n][0] + sB2[c], 0.f) + sW3[c + 1] * fmaxf(acc[n][1] + sB2[c + 1], 0.f);
                ohi += sW3[c] * fmaxf(acc[n][2] + sB2[c], 0.f) + sW3[c + 1] * fmaxf(acc[n][3] + sB2[c + 1], 0.f);
            }
            olo += __shfl_xor_sync(kFull, olo, 1);
            olo += __shfl_xor_sync(kFull, olo, 2);
            ohi += __shfl_xor_sync(kFull, ohi, 1);
            ohi += __shfl_xor_sync(kFull, ohi, 2);
            if (t4 == 0) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int p = r0 + g + 8 * half;
                    const int u = u0 + (p & (kTW - 1)), v = v0 + p / kTW;
                    if (u < in.W && v < in.H) {
                        const float o = (half ? ohi : olo) + sB3[0];
                        wpx[(size_t)v * in.W + u] = sValid[p] ? 1.0f / (1.0f + expf(-o)) : 0.0f;
                    }
                }
            }
        }
        __syncthreads();
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

int conf_grid()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 1, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(conf_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConfSmem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, conf_weights_kernel, 128, kConfSmem);
        g = sms * (per > 0 ? per : 1);
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
