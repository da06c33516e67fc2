// Host side of the C ABI: scene lifetime, argument checks, pose algebra,
// per-frame entry points, counters, export / import of the volume.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "itm_internal.cuh"

namespace itm {

int overflow_capacity();  // itm_alloc.cu

int check_cuda(cudaError_t e) { return e == cudaSuccess ? ITM_OK : ITM_ERR_CUDA; }

void pose_rows(const float T[16], Mat34 &out)
{
    for (int i = 0; i < 12; ++i) out.m[i] = T[i];
}

// Rows 0..2 of T^-1 for a rigid T = [R t]: [R^T, -R^T t], evaluated in double
// (the translation accumulated as 0 - r0 t0 - r1 t1 - r2 t2) and rounded once.
void rigid_inverse_rows(const float T[16], Mat34 &out)
{
    double R[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[i][j] = (double)T[4 * i + j];
        t[i] = (double)T[4 * i + 3];
    }
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) {
            out.m[4 * i + j] = (float)R[j][i];
            acc -= R[j][i] * t[j];
        }
        out.m[4 * i + 3] = (float)acc;
    }
}

int valid_intr(const itm_intrinsics *in)
{
    return in && in->width > 2 && in->height > 2 && in->width <= 32768 && in->height <= 32768 && in->fx > 0.0f &&
           in->fy > 0.0f && isfinite(in->fx) && isfinite(in->fy) && isfinite(in->cx) && isfinite(in->cy) &&
           (long long)in->width * in->height < (1ll << 30);
}

static int valid_pose(const float *T)
{
    if (!T) return 0;
    for (int i = 0; i < 16; ++i)
        if (!isfinite(T[i])) return 0;
    return 1;
}

bool interior_flags_hold(const itm_scene *sc, const float T_wc[16], const itm_intrinsics *intr)
{
    return sc->vis_ok && memcmp(sc->vis_pose, T_wc, sizeof(sc->vis_pose)) == 0 &&
           memcmp(&sc->vis_intr, intr, sizeof(itm_intrinsics)) == 0;
}

Intr to_intr(const itm_intrinsics *in)
{
    Intr r;
    r.W = in->width;
    r.H = in->height;
    r.fx = in->fx;
    r.fy = in->fy;
    r.cx = in->cx;
    r.cy = in->cy;
    return r;
}

static int valid_params(const itm_scene_params *p)
{
    if (!p) return 0;
    if (!(p->voxel_size > 0.0f) || !(p->mu > 0.0f)) return 0;
    // eta / mu is taken from RN(1 / mu) with residual corrections, exact for mu in this range
    if (!(p->mu >= 0x1p-64f && p->mu < 0x1p64f)) return 0;
    if (p->weight_mode != 0 && p->weight_mode != 1) return 0;
    if (p->max_w < 1 || (p->weight_mode == 0 && p->max_w > 255)) return 0;
    if (p->num_buckets < 1 || p->num_buckets > (1 << 30) || (p->num_buckets & (p->num_buckets - 1))) return 0;
    if (p->num_excess < 0 || p->num_excess > (1 << 28)) return 0;
    if (p->num_blocks < 0 || p->num_blocks > (1 << 24)) return 0;
    if (!(p->z_min > 0.0f) || !(p->z_max > p->z_min)) return 0;
    return 1;
}

static void free_dev(SceneDev &d)
{
    void *ptrs[] = {d.entries, d.req, d.req_list, d.overflow, d.visible, d.block_pos, d.sdf,
                    d.w8, d.w32, d.block_free, d.excess_free, d.ctr, d.range_min, d.range_max,
                    d.tile_q_hdr, d.tile_q_list};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    memset(&d, 0, sizeof(d));
}

// Copies blocks ptrs[0..n) (sdf, and weights as float) to out[j].
__global__ void gather_blocks_kernel(SceneDev s, const int32_t *__restrict__ ptrs, int n, float *__restrict__ out_sdf,
                                     float *__restrict__ out_w)
{
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const size_t src = (size_t)ptrs[j] * kBlockVoxels, dst = (size_t)j * kBlockVoxels;
        for (int i = threadIdx.x; i < kBlockVoxels; i += blockDim.x) {
            out_sdf[dst + i] = s.sdf[src + i];
            out_w[dst + i] = s.w8 ? (float)s.w8[src + i] : s.w32[src + i];
        }
    }
}

static const char kVersion[] = "itm-gb300 0.1 (sm_103a)";

}  // namespace itm

using namespace itm;

extern "C" {

const char *itm_version(void) { return kVersion; }

uint32_t itm_hash_index(int x, int y, int z, int num_buckets)
{
    return hash_bucket(x, y, z, (uint32_t)(num_buckets - 1));
}

int itm_scene_create(const itm_scene_params *params, itm_scene **out)
{
    if (!out || !valid_params(params)) return ITM_ERR_ARG;
    *out = nullptr;
    itm_scene *sc = (itm_scene *)calloc(1, sizeof(itm_scene));
    if (!sc) return ITM_ERR_ARG;
    sc->params = *params;
    cudaGetDevice(&sc->device);
    SceneDev &d = sc->d;
    d.nb = params->num_buckets;
    d.ne = params->num_excess;
    d.nv = params->num_blocks;
    d.ovf_cap = overflow_capacity();
    d.voxel_size = params->voxel_size;
    d.mu = params->mu;
    d.inv_mu = 1.0f / params->mu;  // IEEE float division: RN(1 / mu)
    d.z_min = params->z_min;
    d.z_max = params->z_max;
    d.max_w = params->max_w;
    d.weight_mode = params->weight_mode;
    const size_t nvox = (size_t)d.nv * kBlockVoxels;
    cudaError_t e = cudaSuccess;
#define ITM_ALLOC(ptr, bytes)                                         \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes) > 0 ? (bytes) : 16);
    ITM_ALLOC(d.entries, sizeof(Entry) * (size_t)(d.nb + d.ne));
    ITM_ALLOC(d.req, sizeof(unsigned long long) * (size_t)d.nb);
    ITM_ALLOC(d.req_list, sizeof(int32_t) * (size_t)d.nb);
    ITM_ALLOC(d.overflow, sizeof(unsigned long long) * (size_t)d.ovf_cap);
    ITM_ALLOC(d.visible, sizeof(int32_t) * (size_t)(d.nv > 0 ? d.nv : 1));
    ITM_ALLOC(d.block_pos, sizeof(short4) * (size_t)(d.nv > 0 ? d.nv : 1));
    ITM_ALLOC(d.sdf, sizeof(float) * nvox);
    if (d.weight_mode == 0) {
        ITM_ALLOC(d.w8, nvox);
    } else {
        ITM_ALLOC(d.w32, sizeof(float) * nvox);
    }
    ITM_ALLOC(d.block_free, sizeof(int32_t) * (size_t)(d.nv > 0 ? d.nv : 1));
    ITM_ALLOC(d.excess_free, sizeof(int32_t) * (size_t)(d.ne > 0 ? d.ne : 1));
    ITM_ALLOC(d.ctr, sizeof(Counters));
    ITM_ALLOC(d.range_min, sizeof(uint32_t) * (size_t)kRangeMaxTiles);
    ITM_ALLOC(d.range_max, sizeof(uint32_t) * (size_t)kRangeMaxTiles);
    ITM_ALLOC(d.tile_q_hdr, sizeof(int32_t) * 2 * kTileHdrInts);
    ITM_ALLOC(d.tile_q_list, sizeof(int32_t) * 2 * (size_t)kTileClasses * kOrderMaxTiles);
#undef ITM_ALLOC
    if (e == cudaSuccess && d.weight_mode == 1) {
        e = cudaStreamCreateWithFlags(&sc->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sc->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sc->ev_join, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = launch_reset(d, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        if (sc->ev_join) cudaEventDestroy(sc->ev_join);
        if (sc->ev_fork) cudaEventDestroy(sc->ev_fork);
        if (sc->aux) cudaStreamDestroy(sc->aux);
        free_dev(d);
        free(sc);
        cudaGetLastError();
        return ITM_ERR_CUDA;
    }
    sc->last_stream = 0;
    *out = sc;
    return ITM_OK;
}

int itm_scene_destroy(itm_scene *sc)
{
    if (!sc) return ITM_ERR_ARG;
    cudaDeviceSynchronize();
    swap_free(sc);
    if (sc->d.rgbw) cudaFree(sc->d.rgbw);
    if (sc->ev_join) cudaEventDestroy(sc->ev_join);
    if (sc->ev_fork) cudaEventDestroy(sc->ev_fork);
    if (sc->aux) cudaStreamDestroy(sc->aux);
    free_dev(sc->d);
    free(sc);
    return ITM_OK;
}

int itm_scene_reset(itm_scene *sc, itm_stream stream)
{
    Range range_("itm_scene_reset");
    if (!sc) return ITM_ERR_ARG;
    sc->alloc_epoch++;
    sc->vis_ok = false;
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    cudaError_t e = launch_reset(sc->d, st);
    if (e == cudaSuccess) e = swap_reset(sc, st);
    if (e == cudaSuccess && sc->d.rgbw)
        e = cudaMemsetAsync(sc->d.rgbw, 0, sizeof(uint32_t) * (size_t)(sc->d.nv > 0 ? sc->d.nv : 1) * kBlockVoxels, st);
    return check_cuda(e);
}

static int allocate_impl(itm_scene *sc, const float *depth_dev, const uint16_t *raw_dev, const itm_intrinsics *intr,
                         const float T_wc[16], itm_stream stream)
{
    if (!sc || !depth_dev || !valid_pose(T_wc) || !valid_intr(intr)) return ITM_ERR_ARG;
    Mat34 T, M;
    pose_rows(T_wc, T);
    rigid_inverse_rows(T_wc, M);
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    const Intr in = to_intr(intr);
    const bool with_range = range_fits(in);
    sc->alloc_epoch++;
    sc->vis_ok = false;
    if (sc->d.swap_state) sc->d.swap_frame++;  // Sec. 5: the blocks this allocation meets are stamped with it
    const int r = check_cuda(launch_allocate(sc->d, depth_dev, in, T, M, with_range, st, raw_dev));
    if (r == ITM_OK) {
        // the visible list's interior flags hold for this pose and these intrinsics
        sc->vis_ok = true;
        memcpy(sc->vis_pose, T_wc, sizeof(sc->vis_pose));
        sc->vis_intr = *intr;
    }
    if (r == ITM_OK && with_range) {
        // the range tiles now hold the range of a raycast from this pose
        sc->range_epoch = sc->alloc_epoch;
        memcpy(sc->range_pose, T_wc, sizeof(sc->range_pose));
        sc->range_intr = *intr;
    }
    return r;
}

int itm_allocate(itm_scene *sc, const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                 itm_stream stream)
{
    Range range_("itm_allocate");
    return allocate_impl(sc, depth_dev, nullptr, intr, T_wc, stream);
}

int itm_allocate_u16(itm_scene *sc, const uint16_t *raw_dev, float *depth_dev, const itm_intrinsics *intr,
                     const float T_wc[16], itm_stream stream)
{
    Range range_("itm_allocate_u16");
    if (!raw_dev || !depth_dev) return ITM_ERR_ARG;
    return allocate_impl(sc, depth_dev, raw_dev, intr, T_wc, stream);
}

int itm_integrate(itm_scene *sc, const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                  itm_stream stream)
{
    Range range_("itm_integrate");
    if (!sc || !depth_dev || !valid_pose(T_wc) || !valid_intr(intr)) return ITM_ERR_ARG;
    if (sc->d.weight_mode != 0) return ITM_ERR_ARG;
    Mat34 M;
    rigid_inverse_rows(T_wc, M);
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    return check_cuda(launch_integrate(sc->d, depth_dev, nullptr, to_intr(intr), M, interior_flags_hold(sc, T_wc, intr), st));
}

int itm_integrate_weighted(itm_scene *sc, const float *depth_dev, const float *wpx_dev, const itm_intrinsics *intr,
                           const float T_wc[16], itm_stream stream)
{
    Range range_("itm_integrate_weighted");
    if (!sc || !depth_dev || !wpx_dev || !valid_pose(T_wc) || !valid_intr(intr)) return ITM_ERR_ARG;
    if (sc->d.weight_mode != 1) return ITM_ERR_ARG;
    Mat34 M;
    rigid_inverse_rows(T_wc, M);
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    return check_cuda(launch_integrate(sc->d, depth_dev, wpx_dev, to_intr(intr), M, interior_flags_hold(sc, T_wc, intr), st));
}

int itm_raycast(itm_scene *sc, const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev,
                float *normal_dev, itm_stream stream)
{
    Range range_("itm_raycast");
    if (!sc || !valid_pose(T_wc) || !vertex_dev || !normal_dev || !valid_intr(intr)) return ITM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vertex_dev) & 15) || (reinterpret_cast<uintptr_t>(normal_dev) & 15))
        return ITM_ERR_ARG;
    Mat34 T, M;
    pose_rows(T_wc, T);
    rigid_inverse_rows(T_wc, M);
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    const bool ready = sc->range_epoch == sc->alloc_epoch && memcmp(sc->range_pose, T_wc, sizeof(sc->range_pose)) == 0 &&
                       memcmp(&sc->range_intr, intr, sizeof(itm_intrinsics)) == 0;
    const int r = check_cuda(launch_raycast(sc->d, to_intr(intr), T, M, reinterpret_cast<float4 *>(vertex_dev),
                                            reinterpret_cast<float4 *>(normal_dev), ready, sc->order_dims, sc->order_side, st));
    if (r == ITM_OK && range_fits(to_intr(intr))) {
        sc->range_epoch = sc->alloc_epoch;
        memcpy(sc->range_pose, T_wc, sizeof(sc->range_pose));
        sc->range_intr = *intr;
    }
    return r;
}

int itm_scene_set_shard(itm_scene *sc, int parts, int index, int slab_blocks)
{
    if (!sc || parts < 1 || index < 0 || index >= parts || slab_blocks < 2) return ITM_ERR_ARG;
    sc->d.shard_n = parts;
    sc->d.shard_i = index;
    sc->d.shard_w = slab_blocks;
    sc->alloc_epoch += 1;  // the raycast's search ranges are computed again
    return ITM_OK;
}

int itm_raycast_merge(const float *vertex_parts_dev, const float *normal_parts_dev, int parts,
                      const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev, float *normal_dev,
                      itm_stream stream)
{
    Range range_("itm_raycast_merge");
    if (!vertex_parts_dev || !normal_parts_dev || parts < 1 || !valid_intr(intr) || !valid_pose(T_wc) ||
        !vertex_dev || !normal_dev)
        return ITM_ERR_ARG;
    const uintptr_t al = reinterpret_cast<uintptr_t>(vertex_parts_dev) | reinterpret_cast<uintptr_t>(normal_parts_dev) |
                         reinterpret_cast<uintptr_t>(vertex_dev) | reinterpret_cast<uintptr_t>(normal_dev);
    if (al & 15) return ITM_ERR_ARG;
    Mat34 M;
    rigid_inverse_rows(T_wc, M);
    return check_cuda(launch_raycast_merge(reinterpret_cast<const float4 *>(vertex_parts_dev),
                                           reinterpret_cast<const float4 *>(normal_parts_dev), parts,
                                           (long long)intr->width * intr->height, M,
                                           reinterpret_cast<float4 *>(vertex_dev),
                                           reinterpret_cast<float4 *>(normal_dev), (cudaStream_t)stream));
}

int itm_raycast_range(itm_scene *sc, const itm_intrinsics *intr, const float T_wc[16], float *zmin_dev,
                      float *zmax_dev, itm_stream stream)
{
    Range range_("itm_raycast_range");
    if (!sc || !valid_pose(T_wc) || !zmin_dev || !zmax_dev || !valid_intr(intr)) return ITM_ERR_ARG;
    if (zmin_dev == reinterpret_cast<float *>(sc->d.range_min) || zmax_dev == reinterpret_cast<float *>(sc->d.range_max))
        return ITM_ERR_ARG;
    Mat34 M;
    rigid_inverse_rows(T_wc, M);
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    return check_cuda(launch_raycast_range(sc->d, to_intr(intr), M, reinterpret_cast<uint32_t *>(zmin_dev),
                                           reinterpret_cast<uint32_t *>(zmax_dev), st));
}

int itm_raycast_combined(itm_scene *const *scenes, const float *submap_from_world, int n,
                         const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev, float *normal_dev,
                         itm_stream stream)
{
    Range range_("itm_raycast_combined");
    if (!scenes || !submap_from_world || n < 1 || n > ITM_COMBINED_MAX || !valid_intr(intr) || !valid_pose(T_wc) ||
        !vertex_dev || !normal_dev)
        return ITM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vertex_dev) & 15) || (reinterpret_cast<uintptr_t>(normal_dev) & 15))
        return ITM_ERR_ARG;
    SceneDev subs[ITM_COMBINED_MAX];
    Mat34 P[ITM_COMBINED_MAX];
    for (int i = 0; i < n; ++i) {
        const itm_scene *sc = scenes[i];
        if (!sc || !valid_pose(submap_from_world + 16 * i)) return ITM_ERR_ARG;
        const itm_scene_params &a = scenes[0]->params, &b = sc->params;
        if (a.voxel_size != b.voxel_size || a.mu != b.mu || a.z_min != b.z_min || a.z_max != b.z_max ||
            a.weight_mode != b.weight_mode)
            return ITM_ERR_ARG;
        subs[i] = sc->d;
        pose_rows(submap_from_world + 16 * i, P[i]);
    }
    Mat34 T;
    pose_rows(T_wc, T);
    // the combined raycast writes its search ranges into the submaps' range
    // scratch: their next itm_raycast recomputes its own
    for (int i = 0; i < n; ++i) scenes[i]->range_epoch = -1;
    return check_cuda(launch_raycast_combined(subs, P, n, to_intr(intr), T, reinterpret_cast<float4 *>(vertex_dev),
                                              reinterpret_cast<float4 *>(normal_dev), (cudaStream_t)stream));
}

int itm_depth_halve(const float *in_dev, int width, int height, float *out_dev, itm_stream stream)
{
    Range range_("itm_depth_halve");
    if (!in_dev || !out_dev || width < 2 || height < 2 || (long long)width * height >= (1ll << 30)) return ITM_ERR_ARG;
    return check_cuda(launch_depth_halve(in_dev, width, height, out_dev, (cudaStream_t)stream));
}

static int valid_thresh(float t) { return t > 0.0f && isfinite(t); }

int itm_icp_reduce(const float *depth_dev, const itm_intrinsics *intr, const float T_g[16], const float *vertex_dev,
                   const float *normal_dev, const itm_intrinsics *ref_intr, const float T_ref[16], float dist_thresh,
                   double *work_dev, itm_stream stream)
{
    Range range_("itm_icp_reduce");
    if (!depth_dev || !valid_intr(intr) || !valid_pose(T_g) || !vertex_dev || !normal_dev || !valid_intr(ref_intr) ||
        !valid_pose(T_ref) || !valid_thresh(dist_thresh) || !work_dev)
        return ITM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vertex_dev) & 15) || (reinterpret_cast<uintptr_t>(normal_dev) & 15) ||
        (reinterpret_cast<uintptr_t>(work_dev) & 7))
        return ITM_ERR_ARG;
    Mat34 T, M;
    pose_rows(T_g, T);
    rigid_inverse_rows(T_ref, M);
    return check_cuda(launch_icp_reduce(depth_dev, to_intr(intr), T, reinterpret_cast<const float4 *>(vertex_dev),
                                        reinterpret_cast<const float4 *>(normal_dev), to_intr(ref_intr), M,
                                        dist_thresh, work_dev, (cudaStream_t)stream));
}

int itm_icp_step(const double *sums, float T_inout[16], double *step_out)
{
    if (!sums || !T_inout || !valid_pose(T_inout)) return ITM_ERR_ARG;
    if (!(sums[28] >= 6.0)) return ITM_ERR_SINGULAR;
    double A[6][6], L[6][6] = {{0.0}}, y[6], x[6];
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++k) A[i][j] = A[j][i] = sums[k];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double a = A[i][j];
            for (int m = 0; m < j; ++m) a -= L[i][m] * L[j][m];
            if (i == j) {
                if (!(a > 0.0)) return ITM_ERR_SINGULAR;
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
    const double th = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    const double s1 = th > 1e-12 ? sin(th) / th : 1.0;
    const double s2 = th > 1e-12 ? (1.0 - cos(th)) / (th * th) : 0.5;
    const double K[3][3] = {{0.0, -x[2], x[1]}, {x[2], 0.0, -x[0]}, {-x[1], x[0], 0.0}};
    double R[3][3], Tn[12];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double k2 = 0.0;
            for (int m = 0; m < 3; ++m) k2 += K[i][m] * K[m][j];
            R[i][j] = (i == j ? 1.0 : 0.0) + s1 * K[i][j] + s2 * k2;
        }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int m = 0; m < 3; ++m) a += R[i][m] * (double)T_inout[4 * m + j];
            Tn[4 * i + j] = a;
        }
        double a = x[3 + i];
        for (int m = 0; m < 3; ++m) a += R[i][m] * (double)T_inout[4 * m + 3];
        Tn[4 * i + 3] = a;
    }
    for (int i = 0; i < 12; ++i) T_inout[i] = (float)Tn[i];
    T_inout[12] = T_inout[13] = T_inout[14] = 0.0f;
    T_inout[15] = 1.0f;
    if (step_out)
        for (int i = 0; i < 6; ++i) step_out[i] = x[i];
    return ITM_OK;
}

size_t itm_track_scratch_bytes(int width, int height, int levels)
{
    if (width < 1 || height < 1 || levels < 1 || levels > ITM_TRACK_MAX_LEVELS) return 0;
    return track_scratch_bytes(width, height, levels);
}

int itm_track_depth(const float *depth_dev, const itm_intrinsics *intr, int levels, const int *iters,
                    const float *dist_thresh, const float *vertex_dev, const float *normal_dev,
                    const itm_intrinsics *ref_intr, const float T_ref[16], float T_inout[16], int *steps_out,
                    void *scratch_dev, itm_stream stream)
{
    Range range_("itm_track_depth");
    if (!depth_dev || !valid_intr(intr) || levels < 1 || levels > ITM_TRACK_MAX_LEVELS || !iters || !dist_thresh ||
        !vertex_dev || !normal_dev || !valid_intr(ref_intr) || !valid_pose(T_ref) || !T_inout ||
        !valid_pose(T_inout) || !scratch_dev)
        return ITM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vertex_dev) & 15) || (reinterpret_cast<uintptr_t>(normal_dev) & 15) ||
        (reinterpret_cast<uintptr_t>(scratch_dev) & 255))
        return ITM_ERR_ARG;
    for (int l = 0; l < levels; ++l)
        if (iters[l] < 0 || iters[l] > 1000 || !valid_thresh(dist_thresh[l])) return ITM_ERR_ARG;
    Mat34 M;
    rigid_inverse_rows(T_ref, M);
    int steps = 0;
    const int r = check_cuda(launch_track(depth_dev, to_intr(intr), levels, iters, dist_thresh,
                                          reinterpret_cast<const float4 *>(vertex_dev),
                                          reinterpret_cast<const float4 *>(normal_dev), to_intr(ref_intr), M, T_inout,
                                          &steps, scratch_dev, (cudaStream_t)stream));
    if (r == ITM_OK && steps_out) *steps_out = steps;
    return r;
}

int itm_mesh(itm_scene *sc, float *triangles_dev, int64_t capacity, int64_t *n_out, itm_stream stream)
{
    Range range_("itm_mesh");
    if (!sc || capacity < 0 || (capacity > 0 && !triangles_dev) || !n_out) return ITM_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(triangles_dev) & 3) return ITM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    sc->last_stream = st;
    unsigned long long *counter = &sc->d.ctr->mesh_tris;
    cudaError_t e = launch_mesh(sc->d, triangles_dev, (long long)capacity, counter, st);
    unsigned long long cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, counter, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return check_cuda(e);
    *n_out = (int64_t)cnt;
    return (int64_t)cnt > capacity ? ITM_ERR_TOO_LARGE : ITM_OK;
}

int itm_process_frame_u16(itm_scene *sc, const uint16_t *raw_dev, float *depth_dev, const itm_intrinsics *intr,
                          const float T_wc[16], float *vertex_dev, float *normal_dev, itm_stream stream)
{
    Range range_("itm_process_frame_u16");
    if (!sc || (vertex_dev && !normal_dev)) return ITM_ERR_ARG;
    int r = itm_allocate_u16(sc, raw_dev, depth_dev, intr, T_wc, stream);
    if (r == ITM_OK) r = itm_integrate(sc, depth_dev, intr, T_wc, stream);
    if (r == ITM_OK && vertex_dev) r = itm_raycast(sc, intr, T_wc, vertex_dev, normal_dev, stream);
    return r;
}

int itm_process_frame(itm_scene *sc, const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                      float *vertex_dev, float *normal_dev, itm_stream stream)
{
    Range range_("itm_process_frame");
    if (!sc || (vertex_dev && !normal_dev)) return ITM_ERR_ARG;
    int r = itm_allocate(sc, depth_dev, intr, T_wc, stream);
    if (r == ITM_OK) r = itm_integrate(sc, depth_dev, intr, T_wc, stream);
    if (r == ITM_OK && vertex_dev) r = itm_raycast(sc, intr, T_wc, vertex_dev, normal_dev, stream);
    return r;
}

int itm_process_frame_weighted(itm_scene *sc, const float *depth_dev, const void *packed_dev, float *wpx_dev,
                               const itm_intrinsics *intr, const float T_wc[16], float *vertex_dev,
                               float *normal_dev, itm_stream stream)
{
    Range range_("itm_process_frame_weighted");
    if (!sc || !depth_dev || !packed_dev || !wpx_dev || (vertex_dev && !normal_dev) || !valid_intr(intr) ||
        !valid_pose(T_wc))
        return ITM_ERR_ARG;
    if (sc->d.weight_mode != 1 || !sc->aux) return ITM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // fork: the per-pixel weights on the scene's second stream, beside the allocation
    cudaError_t e = cudaEventRecord(sc->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc->aux, sc->ev_fork, 0);
    if (e != cudaSuccess) return check_cuda(e);
    const int rc = itm_conf_weights(depth_dev, intr, sc->params.mu, packed_dev, wpx_dev, (itm_stream)sc->aux);
    int r = itm_allocate(sc, depth_dev, intr, T_wc, stream);
    // join, whatever failed: no work of the call stays behind on the second stream
    e = cudaEventRecord(sc->ev_join, sc->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, sc->ev_join, 0);
    if (e != cudaSuccess) return check_cuda(e);
    if (rc != ITM_OK) return rc;
    if (r == ITM_OK) r = itm_integrate_weighted(sc, depth_dev, wpx_dev, intr, T_wc, stream);
    if (r == ITM_OK && vertex_dev) r = itm_raycast(sc, intr, T_wc, vertex_dev, normal_dev, stream);
    return r;
}

int itm_depth_u16_to_f32(const uint16_t *raw_dev, float *depth_dev, int64_t n, itm_stream stream)
{
    Range range_("itm_depth_u16_to_f32");
    if (n < 0 || (n > 0 && (!raw_dev || !depth_dev))) return ITM_ERR_ARG;
    return check_cuda(launch_depth_u16(raw_dev, depth_dev, n, (cudaStream_t)stream));
}

int itm_scene_stats(itm_scene *sc, itm_stats *out)
{
    if (!sc || !out) return ITM_ERR_ARG;
    Counters c;
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(&c, sc->d.ctr, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    out->status = c.status;
    out->allocated_blocks = c.block_head < sc->d.nv ? c.block_head : sc->d.nv;
    out->excess_used = c.excess_head < sc->d.ne ? c.excess_head : sc->d.ne;
    out->visible_blocks = c.n_visible;
    out->last_requests = c.n_req;
    out->last_overflow = c.n_overflow;
    out->updated_voxels = c.updated;
    out->visited_voxels = c.visited;
    out->frames = c.frames;
    return ITM_OK;
}

int itm_scene_status(itm_scene *sc)
{
    itm_stats st;
    int r = itm_scene_stats(sc, &st);
    if (r != ITM_OK) return r;
    if (st.status & ITM_ST_HASH_FULL) return ITM_ERR_HASH_FULL;
    if (st.status & ITM_ST_VBA_FULL) return ITM_ERR_VBA_FULL;
    if (st.status & ITM_ST_RANGE) return ITM_ERR_RANGE;
    if (st.status & ITM_ST_TIMEOUT) return ITM_ERR_TIMEOUT;
    if (st.status & ITM_ST_OVERFLOW) return ITM_ERR_OVERFLOW;
    if (st.status & ITM_ST_BOUNDS) return ITM_ERR_BOUNDS;
    return ITM_OK;
}

// Blocks are handed out from the free list front to back and never returned,
// so the allocated blocks are the list's first min(block_head, nv) indices;
// at reset the list is the identity, so they are block indices 0 .. n-1.
int itm_scene_export(itm_scene *sc, int16_t *coords_host, float *sdf_host, float *w_host, int cap, int *n)
{
    Range range_("itm_scene_export");
    if (!sc || !n || cap < 0 || (cap > 0 && !coords_host)) return ITM_ERR_ARG;
    itm_stats st;
    int r = itm_scene_stats(sc, &st);
    if (r != ITM_OK) return r;
    // the allocated blocks are block_free[0 .. allocated_blocks), in the
    // order they were handed out (swap-outs fill their gaps from the end)
    const int total = st.allocated_blocks;
    const int nv = sc->d.nv;
    std::vector<int32_t> order((size_t)(total > 0 ? total : 1));
    std::vector<short4> pos((size_t)(nv > 0 ? nv : 1));
    cudaError_t e = cudaSuccess;
    if (total > 0) {
        e = cudaMemcpy(order.data(), sc->d.block_free, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(pos.data(), sc->d.block_pos, sizeof(short4) * nv, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    std::vector<int32_t> keep;
    keep.reserve(total);
    for (int i = 0; i < total; ++i) {
        if (order[i] < 0 || order[i] >= nv) return ITM_ERR_ARG;  // not a block index: a corrupted list
        if (pos[order[i]].w) keep.push_back(order[i]);
    }
    const int m = (int)keep.size();
    *n = m;
    const int cnt = m < cap ? m : cap;
    std::vector<float> sdf, wf;
    if (cnt > 0 && (sdf_host || w_host)) {
        // gather the kept blocks on the device, then one copy each
        const size_t nvox = (size_t)cnt * kBlockVoxels;
        int32_t *ptrs = nullptr;
        float *g_sdf = nullptr, *g_w = nullptr;
        e = cudaMalloc((void **)&ptrs, sizeof(int32_t) * cnt);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g_sdf, sizeof(float) * nvox);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g_w, sizeof(float) * nvox);
        if (e == cudaSuccess) e = cudaMemcpy(ptrs, keep.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            gather_blocks_kernel<<<std::min(cnt, 4096), 128>>>(sc->d, ptrs, cnt, g_sdf, g_w);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            sdf.resize(nvox);
            wf.resize(nvox);
            e = cudaMemcpy(sdf.data(), g_sdf, sizeof(float) * nvox, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(wf.data(), g_w, sizeof(float) * nvox, cudaMemcpyDeviceToHost);
        }
        if (ptrs) cudaFree(ptrs);
        if (g_sdf) cudaFree(g_sdf);
        if (g_w) cudaFree(g_w);
        if (e != cudaSuccess) return ITM_ERR_CUDA;
    }
    for (int k = 0; k < cnt; ++k) {
        const short4 b = pos[keep[k]];
        coords_host[3 * k + 0] = b.x;
        coords_host[3 * k + 1] = b.y;
        coords_host[3 * k + 2] = b.z;
        if (sdf_host) memcpy(&sdf_host[(size_t)k * kBlockVoxels], &sdf[(size_t)k * kBlockVoxels], sizeof(float) * kBlockVoxels);
        if (w_host) memcpy(&w_host[(size_t)k * kBlockVoxels], &wf[(size_t)k * kBlockVoxels], sizeof(float) * kBlockVoxels);
    }
    return ITM_OK;
}

int itm_scene_export_table(itm_scene *sc, int32_t *entries_host)
{
    if (!sc || !entries_host) return ITM_ERR_ARG;
    const size_t total = (size_t)sc->d.nb + sc->d.ne;
    std::vector<Entry> E(total);
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(E.data(), sc->d.entries, sizeof(Entry) * total, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    for (size_t i = 0; i < total; ++i) {
        entries_host[5 * i + 0] = E[i].x;
        entries_host[5 * i + 1] = E[i].y;
        entries_host[5 * i + 2] = E[i].z;
        entries_host[5 * i + 3] = E[i].offset;
        entries_host[5 * i + 4] = E[i].flag ? E[i].ptr : -2;
    }
    return ITM_OK;
}

int itm_scene_import(itm_scene *sc, const int16_t *coords_host, const float *sdf_host, const float *w_host, int n)
{
    Range range_("itm_scene_import");
    if (!sc || n < 0 || n > sc->d.nv || (n > 0 && (!coords_host || !sdf_host || !w_host))) return ITM_ERR_ARG;
    const SceneDev &d = sc->d;
    // Sec. 3.3 insertion, sequentially on the host: bucket first, then the
    // excess chain; block i of the input becomes block index i.
    std::vector<Entry> E((size_t)d.nb + d.ne);
    for (auto &x : E) {
        memset(&x, 0, sizeof(x));
        x.ptr = -2;
    }
    int used_excess = 0;
    std::vector<short4> pos((size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        const int x = coords_host[3 * i], y = coords_host[3 * i + 1], z = coords_host[3 * i + 2];
        const uint32_t h = hash_bucket(x, y, z, (uint32_t)(d.nb - 1));
        Entry *e = &E[h];
        Entry fresh;
        fresh.x = (int16_t)x;
        fresh.y = (int16_t)y;
        fresh.z = (int16_t)z;
        fresh.flag = 1;
        fresh.offset = 0;
        fresh.ptr = i;
        pos[i] = make_short4((short)x, (short)y, (short)z, 1);
        if (!e->flag) {
            *e = fresh;
            continue;
        }
        for (;;) {
            if (e->x == x && e->y == y && e->z == z) return ITM_ERR_ARG;  // duplicate
            if (e->offset < 1) break;
            e = &E[(size_t)d.nb + e->offset - 1];
        }
        if (used_excess >= d.ne) return ITM_ERR_HASH_FULL;
        E[(size_t)d.nb + used_excess] = fresh;
        e->offset = used_excess + 1;
        ++used_excess;
    }
    const size_t nvox = (size_t)n * kBlockVoxels;
    std::vector<uint8_t> w8;
    if (d.weight_mode == 0 && n > 0) {
        w8.resize(nvox);
        for (size_t i = 0; i < nvox; ++i) {
            const float w = w_host[i];
            if (!(w >= 0.0f && w <= (float)d.max_w) || w != (float)(int)w) return ITM_ERR_ARG;
            w8[i] = (uint8_t)w;
        }
    }
    sc->alloc_epoch++;
    sc->vis_ok = false;
    cudaError_t e = cudaStreamSynchronize(sc->last_stream);
    if (e == cudaSuccess) e = launch_reset(d, 0);
    if (e == cudaSuccess) e = swap_reset(sc, 0);
    if (e == cudaSuccess && d.rgbw)
        e = cudaMemsetAsync(d.rgbw, 0, sizeof(uint32_t) * (size_t)(d.nv > 0 ? d.nv : 1) * kBlockVoxels, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e == cudaSuccess)
        e = cudaMemcpy(d.entries, E.data(), sizeof(Entry) * E.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n > 0) {
        e = cudaMemcpy(d.block_pos, pos.data(), sizeof(short4) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d.sdf, sdf_host, sizeof(float) * nvox, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            if (d.weight_mode == 0) e = cudaMemcpy(d.w8, w8.data(), nvox, cudaMemcpyHostToDevice);
            else e = cudaMemcpy(d.w32, w_host, sizeof(float) * nvox, cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) {
        Counters c;
        memset(&c, 0, sizeof(c));
        c.block_head = n;
        c.excess_head = used_excess;
        e = cudaMemcpy(d.ctr, &c, sizeof(c), cudaMemcpyHostToDevice);
    }
    sc->last_stream = 0;
    return check_cuda(e);
}

}  // extern "C"
