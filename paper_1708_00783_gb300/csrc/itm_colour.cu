// Colour voxels (Sec. 3.1: the voxel types with colour carry an RGB value and
// a colour weight; the paper does not print their update).
//
// Readings: a voxel that gets a depth update this frame within the band
// -mu <= eta <= mu takes the colour of its projection into the RGB image --
// its depth-camera coordinates mapped by the depth-to-colour extrinsic,
// projected with the colour intrinsics, the image sampled bilinearly from the
// 2x2 pixels at the floor of the position (which must lie inside the image);
// each channel keeps the running mean (w c + c_obs) / (w + 1) in fp32 rounded
// half up to 8 bits, and the colour weight counts observations up to max_w.
// A point's colour is its nearest voxel's (voxel coordinates as in the
// raycast, nearest voxel floor(q + 1/2)).
//
// The colour pass runs after the depth integration over the same visible
// blocks and repeats its projection and decision arithmetic operation for
// operation (built with -fmad=false like the integration), so it colours
// exactly the voxels the integration updated within the band; the
// integration kernel itself is unchanged.  Voxel colour: one 32-bit word per
// voxel, bytes r, g, b, colour weight, in the sdf's voxel order.  Colour runs
// with the constant observation weight (weight mode 0) and without swapping.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "itm_ops.cuh"

namespace itm {

namespace {

struct ColourFrame {
    const uint8_t *rgb;  // Hc x Wc x 3 bytes, row-major
    int Wc, Hc;
    float fx, fy, cx, cy;
    Mat34 T;  // depth camera -> colour camera
};

constexpr int kThreads = 64;

// The colour observation of the voxel at depth-camera coordinates (X, Y, Z)
// fused into its word.
__device__ __forceinline__ void colour_update(uint32_t *word, float X, float Y, float Z, const ColourFrame &cf,
                                              float max_w)
{
    const float Xc = row_apply(&cf.T.m[0], X, Y, Z);
    const float Yc = row_apply(&cf.T.m[4], X, Y, Z);
    const float Zc = row_apply(&cf.T.m[8], X, Y, Z);
    if (!(Zc > 0.0f)) return;
    const float uc = fadd(fdiv(fmul(cf.fx, Xc), Zc), cf.cx);
    const float vc = fadd(fdiv(fmul(cf.fy, Yc), Zc), cf.cy);
    if (!(uc >= 0.0f && vc >= 0.0f && uc < (float)(cf.Wc - 1) && vc < (float)(cf.Hc - 1))) return;
    const int u0 = (int)uc, v0 = (int)vc;
    const float a = fsub(uc, (float)u0), b = fsub(vc, (float)v0);
    const uint32_t old = *word;
    const float wc = (float)(old >> 24);
    const size_t r0 = ((size_t)v0 * cf.Wc + u0) * 3, r1 = r0 + (size_t)cf.Wc * 3;
    uint32_t out = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float p00 = (float)__ldg(&cf.rgb[r0 + ch]), p10 = (float)__ldg(&cf.rgb[r0 + 3 + ch]);
        const float p01 = (float)__ldg(&cf.rgb[r1 + ch]), p11 = (float)__ldg(&cf.rgb[r1 + 3 + ch]);
        const float top = fadd(p00, fmul(a, fsub(p10, p00)));
        const float bot = fadd(p01, fmul(a, fsub(p11, p01)));
        const float obs = fadd(top, fmul(b, fsub(bot, top)));
        const float nc = fdiv(fadd(fmul(wc, (float)((old >> (8 * ch)) & 0xffu)), obs), fadd(wc, 1.0f));
        const int q = (int)fadd(nc, 0.5f);
        out |= (uint32_t)(q < 0 ? 0 : (q > 255 ? 255 : q)) << (8 * ch);
    }
    const float nw = fadd(wc, 1.0f);
    out |= (uint32_t)(nw < max_w ? nw : max_w) << 24;
    *word = out;
}

// One visible block per CTA iteration, thread t the x-row of voxels 8t ..
// 8t+7, with the integration's arithmetic (integrate_block) for the voxel's
// position, projection and update decision.
__global__ void __launch_bounds__(kThreads) colour_kernel(SceneDev s, const float *__restrict__ depth, Intr in,
                                                          Mat34 M, ColourFrame cf, uint32_t *__restrict__ rgbw)
{
    const int n = min(__ldcg(&s.ctr->n_visible), s.nv);
    const int t = threadIdx.x, ly = t & 7, lz = t >> 3;
    const float vs = s.voxel_size, neg_mu = -s.mu, mu = s.mu;
    const float umax = (float)(in.W - 2), vmax = (float)(in.H - 2);
    const float max_w = (float)s.max_w;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int ptr = vis_ptr(__ldg(&s.visible[i]));
        if (ptr >= s.nv) continue;
        const short4 b = __ldg(&s.block_pos[ptr]);
        const float py = fmul((float)(b.y * 8 + ly), vs);
        const float pz = fmul((float)(b.z * 8 + lz), vs);
        const float xy = fmul(M.m[1], py), xz = fmul(M.m[2], pz);
        const float yy = fmul(M.m[5], py), yz = fmul(M.m[6], pz);
        const float zy = fmul(M.m[9], py), zz = fmul(M.m[10], pz);
        const float gx0 = (float)(b.x * 8);
        // the eight voxels' pixels first, then their depth reads together, then
        // the decisions and the colour updates (as the integration orders them)
        int pix[8];
        float Zk[8];
        unsigned valid = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float px = fmul(fadd(gx0, (float)k), vs);
            const float Z = fadd(fadd(fadd(fmul(M.m[8], px), zy), zz), M.m[11]);
            Zk[k] = Z;
            pix[k] = 0;
            if (Z <= 0.0f) continue;
            const float X = fadd(fadd(fadd(fmul(M.m[0], px), xy), xz), M.m[3]);
            const float Y = fadd(fadd(fadd(fmul(M.m[4], px), yy), yz), M.m[7]);
            const float u = fadd(fdiv(fmul(in.fx, X), Z), in.cx);
            const float v = fadd(fdiv(fmul(in.fy, Y), Z), in.cy);
            if (u < 1.0f || u > umax || v < 1.0f || v > vmax) continue;
            const int p = (int)fadd(u, 0.5f) + (int)fadd(v, 0.5f) * in.W;
            if (p < 0 || p >= in.W * in.H) continue;
            pix[k] = p;
            valid |= 1u << k;
        }
        float dk[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) dk[k] = (valid & (1u << k)) ? __ldg(&depth[pix[k]]) : 0.0f;
        unsigned band = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (!(valid & (1u << k)) || !(dk[k] > 0.0f)) continue;
            const float eta = fsub(dk[k], Zk[k]);
            if (!(eta < neg_mu || eta > mu)) band |= 1u << k;
        }
        while (band) {
            const int k = __ffs(band) - 1;
            band &= band - 1;
            // the voxel's camera coordinates again, with the same operations
            const float px = fmul(fadd(gx0, (float)k), vs);
            const float X = fadd(fadd(fadd(fmul(M.m[0], px), xy), xz), M.m[3]);
            const float Y = fadd(fadd(fadd(fmul(M.m[4], px), yy), yz), M.m[7]);
            const float Z = fadd(fadd(fadd(fmul(M.m[8], px), zy), zz), M.m[11]);
            colour_update(&rgbw[(size_t)ptr * kBlockVoxels + 8 * t + k], X, Y, Z, cf, max_w);
        }
    }
}

// Colour (r, g, b, colour weight) of the voxel nearest each valid point.
__global__ void __launch_bounds__(256) colour_at_kernel(SceneDev s, const float4 *__restrict__ pts, int64_t n,
                                                        float inv_sv, const uint32_t *__restrict__ rgbw,
                                                        uint32_t *__restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const float4 p = __ldg(&pts[j]);
        uint32_t c = 0;
        if (p.w > 0.0f) {
            const float q[3] = {fmul(p.x, inv_sv), fmul(p.y, inv_sv), fmul(p.z, inv_sv)};
            if (coord_ok(q[0]) && coord_ok(q[1]) && coord_ok(q[2])) {
                const int gx = (int)floorf(fadd(q[0], 0.5f)), gy = (int)floorf(fadd(q[1], 0.5f));
                const int gz = (int)floorf(fadd(q[2], 0.5f));
                const int ptr = lookup_ro(s, gx >> 3, gy >> 3, gz >> 3);
                if (ptr >= 0) c = __ldg(&rgbw[(size_t)ptr * kBlockVoxels + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7)]);
            }
        }
        out[j] = c;
    }
}

__global__ void gather_colour_kernel(const uint32_t *__restrict__ rgbw, const int32_t *__restrict__ ptrs, int n,
                                     uint32_t *__restrict__ out)
{
    for (int j = blockIdx.x; j < n; j += gridDim.x)
        for (int i = threadIdx.x; i < kBlockVoxels; i += blockDim.x)
            out[(size_t)j * kBlockVoxels + i] = rgbw[(size_t)ptrs[j] * kBlockVoxels + i];
}

int finite16(const float *T)
{
    if (!T) return 0;
    for (int i = 0; i < 16; ++i)
        if (!isfinite(T[i])) return 0;
    return 1;
}

int grid_for(int per_sm)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * (sms > 0 ? sms : 1);
}

}  // namespace

}  // namespace itm

using namespace itm;

extern "C" {

int itm_colour_enable(itm_scene *sc)
{
    if (!sc || sc->d.rgbw || sc->d.weight_mode != 0 || sc->d.swap_state) return ITM_ERR_ARG;
    const size_t bytes = sizeof(uint32_t) * (size_t)(sc->d.nv > 0 ? sc->d.nv : 1) * kBlockVoxels;
    uint32_t *p = nullptr;
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p, bytes);
    if (e == cudaSuccess) e = cudaMemset(p, 0, bytes);
    if (e != cudaSuccess) {
        if (p) cudaFree(p);
        cudaGetLastError();
        return ITM_ERR_CUDA;
    }
    sc->d.rgbw = p;
    return ITM_OK;
}

int itm_integrate_colour(itm_scene *sc, const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                         const uint8_t *rgb_dev, const itm_intrinsics *intr_colour, const float T_d2c[16],
                         itm_stream stream)
{
    Range range_("itm_integrate_colour");
    if (!sc || !sc->d.rgbw || !depth_dev || !rgb_dev || !finite16(T_wc) || !finite16(T_d2c)) return ITM_ERR_ARG;
    if (!valid_intr(intr) || !valid_intr(intr_colour) || intr_colour->width < 2 || intr_colour->height < 2)
        return ITM_ERR_ARG;
    Mat34 M, Tc;
    rigid_inverse_rows(T_wc, M);
    pose_rows(T_d2c, Tc);
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    const Intr in = to_intr(intr);
    cudaError_t e = launch_integrate(sc->d, depth_dev, nullptr, in, M, interior_flags_hold(sc, T_wc, intr), st);
    if (e != cudaSuccess) return check_cuda(e);
    ColourFrame cf;
    cf.rgb = rgb_dev;
    cf.Wc = intr_colour->width;
    cf.Hc = intr_colour->height;
    cf.fx = intr_colour->fx;
    cf.fy = intr_colour->fy;
    cf.cx = intr_colour->cx;
    cf.cy = intr_colour->cy;
    cf.T = Tc;
    colour_kernel<<<grid_for(16), kThreads, 0, st>>>(sc->d, depth_dev, in, M, cf, sc->d.rgbw);
    return check_cuda(cudaGetLastError());
}

int itm_colour_at(itm_scene *sc, const float *points_dev, int64_t n, uint8_t *rgbw_dev, itm_stream stream)
{
    Range range_("itm_colour_at");
    if (!sc || !sc->d.rgbw || n < 0 || (n > 0 && (!points_dev || !rgbw_dev))) return ITM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(points_dev) & 15) || (reinterpret_cast<uintptr_t>(rgbw_dev) & 3))
        return ITM_ERR_ARG;
    if (n == 0) return ITM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    const float inv_sv = (float)(1.0 / (double)sc->d.voxel_size);
    const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)grid_for(8));
    colour_at_kernel<<<g, 256, 0, st>>>(sc->d, reinterpret_cast<const float4 *>(points_dev), n, inv_sv, sc->d.rgbw,
                                        reinterpret_cast<uint32_t *>(rgbw_dev));
    return check_cuda(cudaGetLastError());
}

int itm_scene_export_colour(itm_scene *sc, int16_t *coords_host, uint8_t *rgbw_host, int cap, int *n)
{
    Range range_("itm_scene_export_colour");
    if (!sc || !sc->d.rgbw || !n || cap < 0 || (cap > 0 && (!coords_host || !rgbw_host))) return ITM_ERR_ARG;
    itm_stats st;
    int r = itm_scene_stats(sc, &st);
    if (r != ITM_OK) return r;
    const int total = st.allocated_blocks, nv = sc->d.nv;
    std::vector<int32_t> order((size_t)(total > 0 ? total : 1));
    std::vector<short4> pos((size_t)(nv > 0 ? nv : 1));
    cudaError_t e = cudaSuccess;
    if (total > 0) {
        e = cudaMemcpy(order.data(), sc->d.block_free, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(pos.data(), sc->d.block_pos, sizeof(short4) * nv, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    std::vector<int32_t> keep;
    for (int i = 0; i < total; ++i) {
        if (order[i] < 0 || order[i] >= nv) return ITM_ERR_ARG;
        if (pos[order[i]].w) keep.push_back(order[i]);
    }
    const int m = (int)keep.size();
    *n = m;
    const int cnt = m < cap ? m : cap;
    if (cnt > 0) {
        int32_t *ptrs = nullptr;
        uint32_t *g = nullptr;
        e = cudaMalloc((void **)&ptrs, sizeof(int32_t) * cnt);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g, sizeof(uint32_t) * (size_t)cnt * kBlockVoxels);
        if (e == cudaSuccess) e = cudaMemcpy(ptrs, keep.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            gather_colour_kernel<<<std::min(cnt, 4096), 128>>>(sc->d.rgbw, ptrs, cnt, g);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpy(rgbw_host, g, sizeof(uint32_t) * (size_t)cnt * kBlockVoxels, cudaMemcpyDeviceToHost);
        if (ptrs) cudaFree(ptrs);
        if (g) cudaFree(g);
        if (e != cudaSuccess) return ITM_ERR_CUDA;
        for (int k = 0; k < cnt; ++k) {
            coords_host[3 * k] = pos[keep[k]].x;
            coords_host[3 * k + 1] = pos[keep[k]].y;
            coords_host[3 * k + 2] = pos[keep[k]].z;
        }
    }
    return ITM_OK;
}

}  // extern "C"
