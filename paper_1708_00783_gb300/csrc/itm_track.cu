// Sec. 4.1.1 depth tracker (ITMDepthTracker): point-to-plane alignment of a
// depth frame to the raycast vertex/normal maps, coarse to fine.
//
//  * depth_halve_kernel: one pyramid level, the mean of the valid depths of
//    each 2x2 block (summed in raster order, one rounded division).
//  * icp_partial_kernel: per pixel, the camera point d ((u-cx)/fx,
//    (v-cy)/fy, 1) mapped to the world by the current estimate T, projected
//    into the reference view (nearest pixel); with both maps valid there and
//    |T p - V| within the outlier distance, the residual r = (T p - V) . N and
//    J = (T p x N, N) give J J^T, J r, r^2 and a count.  The per-pixel
//    arithmetic is float with each operation rounded on its own (built with
//    -fmad=false), so the selection of pixels is the same on any IEEE
//    machine; a thread accumulates its pixels (about eight) in float and a
//    warp adds its lanes by a float shuffle tree (FP64 is a small fraction
//    of the FP32 rate here); the CTA adds its warps in double and writes one
//    partial row.  Each float sum is within 13 roundings of 2^-24 of the
//    magnitude of its terms.
//  * icp_solve_kernel (one CTA): sums the partial rows in a fixed order (the
//    result does not depend on scheduling), then, in double, solves
//    H x = -g by Cholesky and applies the motion x = (omega, tau) on the world
//    side, T <- [R(omega) | tau] T with R by Rodrigues' formula.  The pose
//    stays in device memory, so a whole coarse-to-fine track runs without a
//    host round trip per step (the paper solves on the host).
#include "itm_ops.cuh"

namespace itm {

namespace {

constexpr int kIcpThreads = 256;

__global__ void __launch_bounds__(256) depth_halve_kernel(const float *__restrict__ in, int W, int H,
                                                          float *__restrict__ out)
{
    const int w = W / 2, h = H / 2;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < w * h; o += gridDim.x * blockDim.x) {
        const int i = o % w, j = o / w;
        float sum = 0.0f;
        int n = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float d = __ldg(&in[(size_t)(2 * j + (k >> 1)) * W + 2 * i + (k & 1)]);
            if (d > 0.0f) {
                sum = fadd(sum, d);
                ++n;
            }
        }
        out[o] = n > 0 ? fdiv(sum, (float)n) : 0.0f;
    }
}

struct IcpState {
    float T[16];  // current camera-to-world estimate
    int done;     // the level stopped (too few pixels or no solution)
    int steps;    // steps applied
};

// Partial sums of CTA blockIdx.x: partials[b * kIcpSums + k].  The pose is
// read from the tracker state st (or T_arg when st is null).
__global__ void __launch_bounds__(kIcpThreads) icp_partial_kernel(
    const float *__restrict__ depth, int W, int H, Intr in, const IcpState *__restrict__ st, Mat34 T_arg,
    const float4 *__restrict__ V, const float4 *__restrict__ N, Intr ref, Mat34 M, float dist_thresh,
    double *__restrict__ partials)
{
    __shared__ double red[kIcpThreads / 32][kIcpSums];
    if (st && st->done) return;
    Mat34 T = T_arg;
    if (st) {
#pragma unroll
        for (int k = 0; k < 12; ++k) T.m[k] = st->T[k];
    }
    const float t2 = fmul(dist_thresh, dist_thresh);
    float acc[kIcpSums - 1];
#pragma unroll
    for (int k = 0; k < kIcpSums - 1; ++k) acc[k] = 0.0f;
    int count = 0;
    const int n_pix = W * H;
    // kBatch pixels per pass (p, p + stride, ...): their depth loads, then
    // their map loads, are issued together
    constexpr int kBatch = 4;
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x + threadIdx.x; p0 < n_pix; p0 += kBatch * stride) {
        float dk[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int p = p0 + b * stride;
            dk[b] = p < n_pix ? __ldg(&depth[p]) : 0.0f;
        }
        float pw[kBatch][3];
        int o[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            o[b] = -1;
            const float d = dk[b];
            if (!(d > 0.0f)) continue;
            const int p = p0 + b * stride;
            const int u = p % W, v = p / W;
            const float pcx = fmul(fdiv(fsub((float)u, in.cx), in.fx), d);
            const float pcy = fmul(fdiv(fsub((float)v, in.cy), in.fy), d);
            float pr[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) pw[b][r] = row_apply(T.m + 4 * r, pcx, pcy, d);
#pragma unroll
            for (int r = 0; r < 3; ++r) pr[r] = row_apply(M.m + 4 * r, pw[b][0], pw[b][1], pw[b][2]);
            if (!(pr[2] > 0.0f)) continue;
            const float ur = fadd(fdiv(fmul(ref.fx, pr[0]), pr[2]), ref.cx);
            const float vr = fadd(fdiv(fmul(ref.fy, pr[1]), pr[2]), ref.cy);
            if (!(ur >= 0.0f && ur <= (float)(ref.W - 1) && vr >= 0.0f && vr <= (float)(ref.H - 1))) continue;
            o[b] = (int)fadd(vr, 0.5f) * ref.W + (int)fadd(ur, 0.5f);
        }
        float4 Vk[kBatch], Nk[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            Vk[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            Nk[b] = Vk[b];
            if (o[b] >= 0) {
                Vk[b] = __ldg(&V[o[b]]);
                Nk[b] = __ldg(&N[o[b]]);
            }
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            if (o[b] < 0) continue;
            const float4 Vp = Vk[b], Np = Nk[b];
            if (!(Vp.w > 0.0f && Np.w > 0.0f)) continue;
            const float dx = fsub(pw[b][0], Vp.x), dy = fsub(pw[b][1], Vp.y), dz = fsub(pw[b][2], Vp.z);
            const float dist2 = fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
            if (!(dist2 <= t2)) continue;
            const float res = fadd(fadd(fmul(dx, Np.x), fmul(dy, Np.y)), fmul(dz, Np.z));
            const float J[6] = {fsub(fmul(pw[b][1], Np.z), fmul(pw[b][2], Np.y)),
                                fsub(fmul(pw[b][2], Np.x), fmul(pw[b][0], Np.z)),
                                fsub(fmul(pw[b][0], Np.y), fmul(pw[b][1], Np.x)), Np.x, Np.y, Np.z};
            int k = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = i; j < 6; ++j, ++k) acc[k] = fadd(acc[k], fmul(J[i], J[j]));
#pragma unroll
            for (int i = 0; i < 6; ++i) acc[21 + i] = fadd(acc[21 + i], fmul(J[i], res));
            acc[27] = fadd(acc[27], fmul(res, res));
            ++count;
        }
    }
    // warps by float shuffle trees (the count exactly, as an integer), then
    // the CTA's warp rows in double, in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kIcpSums - 1; ++k) {
        float x = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = fadd(x, __shfl_down_sync(kFull, x, off));
        if (lane == 0) red[warp][k] = (double)x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) count += __shfl_down_sync(kFull, count, off);
    if (lane == 0) red[warp][kIcpSums - 1] = (double)count;
    __syncthreads();
    if (threadIdx.x < kIcpSums) {
        double x = 0.0;
#pragma unroll
        for (int w = 0; w < kIcpThreads / 32; ++w) x += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * kIcpSums + threadIdx.x] = x;
    }
}

// Sums the n_part partial rows into sums: warp w adds column w, lane l the
// rows l, l + 32, ... in order, then a fixed shuffle tree (the result does
// not depend on scheduling); with st, thread 0 then takes the Gauss-Newton
// step.
__global__ void __launch_bounds__(1024) icp_solve_kernel(const double *__restrict__ partials, int n_part,
                                                         double *__restrict__ sums, IcpState *st)
{
    if (st && st->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < kIcpSums) {
        double x = 0.0;
        for (int b = lane; b < n_part; b += 32) x += partials[(size_t)b * kIcpSums + warp];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(kFull, x, off);
        if (lane == 0) sums[warp] = x;
    }
    __syncthreads();
    if (!st || threadIdx.x != 0) return;
    if (sums[28] < 6.0) {
        st->done = 1;
        return;
    }
    double A[6][6], L[6][6], y[6], x[6];
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++k) A[i][j] = A[j][i] = sums[k];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double a = A[i][j];
            for (int m = 0; m < j; ++m) a -= L[i][m] * L[j][m];
            if (i == j) {
                if (!(a > 0.0)) {
                    st->done = 1;
                    return;
                }
                L[i][i] = sqrt(a);
            } else {
                L[i][j] = a / L[j][j];
            }
        }
    }
    for (int i = 0; i < 6; ++i) {
        double a = -sums[21 + i];
        for (int m = 0; m < i; ++m) a -= L[i][m] * y[m];
        y[i] = a / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double a = y[i];
        for (int m = i + 1; m < 6; ++m) a -= L[m][i] * x[m];
        x[i] = a / L[i][i];
    }
    // R = I + sin(th)/th K + (1 - cos(th))/th^2 K^2, K = [omega]_x
    const double th = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    const double s1 = th > 1e-12 ? sin(th) / th : 1.0;
    const double s2 = th > 1e-12 ? (1.0 - cos(th)) / (th * th) : 0.5;
    const double K[3][3] = {{0.0, -x[2], x[1]}, {x[2], 0.0, -x[0]}, {-x[1], x[0], 0.0}};
    double R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double k2 = 0.0;
            for (int m = 0; m < 3; ++m) k2 += K[i][m] * K[m][j];
            R[i][j] = (i == j ? 1.0 : 0.0) + s1 * K[i][j] + s2 * k2;
        }
    float Tn[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int m = 0; m < 3; ++m) a += R[i][m] * (double)st->T[4 * m + j];
            Tn[4 * i + j] = (float)a;
        }
        double a = x[3 + i];
        for (int m = 0; m < 3; ++m) a += R[i][m] * (double)st->T[4 * m + 3];
        Tn[4 * i + 3] = (float)a;
    }
    for (int i = 0; i < 12; ++i) st->T[i] = Tn[i];
    st->steps += 1;
}

int icp_grid(int n_pix)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    // about eight pixels per thread, at most two CTAs per SM and kIcpMaxPartials rows
    int g = (n_pix + 8 * kIcpThreads - 1) / (8 * kIcpThreads);
    if (g > 2 * sms) g = 2 * sms;
    if (g > kIcpMaxPartials) g = kIcpMaxPartials;
    return g > 0 ? g : 1;
}

}  // namespace

cudaError_t launch_depth_halve(const float *in, int W, int H, float *out, cudaStream_t st)
{
    const int n = (W / 2) * (H / 2);
    if (n <= 0) return cudaSuccess;
    int g = (n + 255) / 256;
    if (g > 1216) g = 1216;
    depth_halve_kernel<<<g, 256, 0, st>>>(in, W, H, out);
    return cudaGetLastError();
}

cudaError_t launch_icp_reduce(const float *depth, const Intr &in, const Mat34 &T_g, const float4 *V, const float4 *N,
                              const Intr &ref, const Mat34 &M_ref, float dist_thresh, double *work, cudaStream_t st)
{
    const int g = icp_grid(in.W * in.H);
    double *partials = work + kIcpSums;
    icp_partial_kernel<<<g, kIcpThreads, 0, st>>>(depth, in.W, in.H, in, nullptr, T_g, V, N, ref, M_ref, dist_thresh,
                                                   partials);
    icp_solve_kernel<<<1, 1024, 0, st>>>(partials, g, work, nullptr);
    return cudaGetLastError();
}

size_t track_scratch_bytes(int W, int H, int levels)
{
    size_t b = sizeof(double) * (size_t)kIcpWorkDoubles + 256;  // work, then the state
    int w = W, h = H;
    for (int l = 1; l < levels; ++l) {
        w /= 2;
        h /= 2;
        b += sizeof(float) * (size_t)(w > 0 ? w : 0) * (size_t)(h > 0 ? h : 0);
        b = (b + 255) & ~(size_t)255;
    }
    return b;
}

cudaError_t launch_track(const float *depth, const Intr &in0, int levels, const int *iters, const float *thresh,
                         const float4 *V, const float4 *N, const Intr &ref, const Mat34 &M_ref, float T[16],
                         int *steps, void *scratch, cudaStream_t st)
{
    char *base = static_cast<char *>(scratch);
    double *work = reinterpret_cast<double *>(base);
    IcpState *state = reinterpret_cast<IcpState *>(base + sizeof(double) * (size_t)kIcpWorkDoubles);
    size_t off = sizeof(double) * (size_t)kIcpWorkDoubles + 256;
    const float *lev[kTrackMaxLevels];
    Intr li[kTrackMaxLevels];
    lev[0] = depth;
    li[0] = in0;
    for (int l = 1; l < levels; ++l) {
        float *out = reinterpret_cast<float *>(base + off);
        li[l].W = li[l - 1].W / 2;
        li[l].H = li[l - 1].H / 2;
        // pixel i of the next level covers pixels 2i, 2i+1: f / 2, (c - 1/2) / 2
        volatile float fx = li[l - 1].fx / 2.0f, fy = li[l - 1].fy / 2.0f;
        volatile float cxm = li[l - 1].cx - 0.5f, cym = li[l - 1].cy - 0.5f;
        li[l].fx = fx;
        li[l].fy = fy;
        li[l].cx = cxm / 2.0f;
        li[l].cy = cym / 2.0f;
        cudaError_t e = launch_depth_halve(lev[l - 1], li[l - 1].W, li[l - 1].H, out, st);
        if (e != cudaSuccess) return e;
        lev[l] = out;
        off += sizeof(float) * (size_t)li[l].W * (size_t)li[l].H;
        off = (off + 255) & ~(size_t)255;
    }
    IcpState h_state;
    memset(&h_state, 0, sizeof(h_state));
    memcpy(h_state.T, T, sizeof(h_state.T));
    cudaError_t e = cudaMemcpyAsync(state, &h_state, sizeof(h_state), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    double *partials = work + kIcpSums;
    for (int l = levels - 1; l >= 0; --l) {
        if (iters[l] <= 0 || li[l].W < 1 || li[l].H < 1) continue;
        e = cudaMemsetAsync(&state->done, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        const int g = icp_grid(li[l].W * li[l].H);
        for (int it = 0; it < iters[l]; ++it) {
            icp_partial_kernel<<<g, kIcpThreads, 0, st>>>(lev[l], li[l].W, li[l].H, li[l], state, Mat34{}, V, N, ref,
                                                           M_ref, thresh[l], partials);
            icp_solve_kernel<<<1, 1024, 0, st>>>(partials, g, work, state);
        }
    }
    e = cudaMemcpyAsync(&h_state, state, sizeof(h_state), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    memcpy(T, h_state.T, sizeof(float) * 12);
    T[12] = T[13] = T[14] = 0.0f;
    T[15] = 1.0f;
    *steps = h_state.steps;
    return cudaGetLastError();
}

}  // namespace itm
