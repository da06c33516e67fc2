// Block set of one depth frame, computed without allocating any memory.
//
// Some callers cannot call cudaMalloc: a real-time loop that must not take
// the allocator's locks or latency once it runs, a host framework that hands
// out device memory only from its own fixed arenas, or a system that forbids
// dynamic allocation after start-up.  They still want to know which voxel
// blocks a frame touches (to reserve storage in their own pools, to stream
// blocks in, to schedule work).  This entry point answers that with no scene
// and no allocation: the caller passes the depth frame and the output
// buffers, and the de-duplication set lives in a fixed array below.
//
// The set is a file-scope __device__ array of kSlots 64-bit words (32 MiB),
// held by every GPU that loads the library until the process exits.  Host
// code must not pass the array's name to a kernel (on the host it names a
// stand-in, not device memory): the first call on each device looks up its
// device address with cudaGetSymbolAddress, with that device current, and
// keeps it.  Every call shares the array and clears it first; calls that
// overlap on the GPU (different streams, or a second host thread) race on it.
#include <math.h>

#include <mutex>

#include "itm_internal.cuh"

namespace itm {

namespace {

constexpr int kMaxBlocks = ITM_NOALLOC_MAX_BLOCKS;  // distinct blocks one call may hold
constexpr int kSlots = 2 * kMaxBlocks;              // open-addressing slots (load <= 1/2)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_block_set[kSlots];

std::mutex g_setup_mutex;
unsigned long long *g_set_addr[kMaxDevices] = {nullptr};

// Device address of g_block_set on the current device (looked up once).
int set_address(unsigned long long **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ITM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_set_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_block_set) != cudaSuccess || !p) {
            cudaGetLastError();
            return ITM_ERR_CUDA;
        }
        g_set_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_set_addr[dev];
    return ITM_OK;
}

__device__ __forceinline__ uint32_t slot_of(unsigned long long k)
{
    // splitmix64 finaliser: spreads neighbouring block keys over the table
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ull;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebull;
    k ^= k >> 31;
    return (uint32_t)k & (uint32_t)(kSlots - 1);
}

// One thread per pixel, 8x4-pixel warp tiles; the segment d-mu .. d+mu and
// the DDA over the blocks it crosses are the same arithmetic as
// alloc_enumerate_kernel (Sec. 4.2).  Each distinct block enters the set
// once and is appended to the caller's output.
__global__ void __launch_bounds__(256) frame_blocks_kernel(unsigned long long *__restrict__ set,
                                                           const float *__restrict__ depth, Intr in, Mat34 T,
                                                           float inv_b, float mu, float z_min, float z_max,
                                                           short *__restrict__ coords, int cap, int32_t *count)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int u = blockIdx.x * 32 + (warp & 3) * 8 + (lane & 7);
    const int v = blockIdx.y * 8 + (warp >> 2) * 4 + (lane >> 3);
    float d = 0.0f;
    if (u < in.W && v < in.H) d = __ldg(&depth[(size_t)v * in.W + u]);
    bool more = (d > 0.0f) && !(d < z_min) && !(d > z_max);
    int cur[3] = {0, 0, 0}, step[3] = {0, 0, 0}, left[3] = {0, 0, 0};
    float tmax[3] = {0.f, 0.f, 0.f}, tdelta[3] = {0.f, 0.f, 0.f};
    if (more) {
        const float rx = fdiv(fsub((float)u, in.cx), in.fx);
        const float ry = fdiv(fsub((float)v, in.cy), in.fy);
        float z0 = fsub(d, mu);
        const float z1 = fadd(d, mu);
        if (z0 < 1e-3f) z0 = 1e-3f;
        const float ax = fmul(rx, z0), ay = fmul(ry, z0);
        const float bx = fmul(rx, z1), by = fmul(ry, z1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float q0 = fmul(row_apply(&T.m[4 * i], ax, ay, z0), inv_b);
            const float q1 = fmul(row_apply(&T.m[4 * i], bx, by, z1), inv_b);
            const float f0 = floorf(q0), f1 = floorf(q1);
            if (!(f0 >= -32768.0f && f0 <= 32767.0f && f1 >= -32768.0f && f1 <= 32767.0f)) {
                more = false;
                continue;
            }
            cur[i] = (int)f0;
            const int end = (int)f1;
            const float dir = fsub(q1, q0);
            if (end > cur[i]) {
                step[i] = 1;
                left[i] = end - cur[i];
                tdelta[i] = fdiv(1.0f, dir);
                tmax[i] = fdiv(fsub((float)(cur[i] + 1), q0), dir);
            } else if (end < cur[i]) {
                step[i] = -1;
                left[i] = cur[i] - end;
                tdelta[i] = fdiv(-1.0f, dir);
                tmax[i] = fdiv(fsub((float)cur[i], q0), dir);
            }
        }
    }
    while (__any_sync(kFull, more)) {
        const unsigned long long key = more ? pack_key(cur[0], cur[1], cur[2]) : 0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        if (more && lane == __ffs(peers) - 1) {
            uint32_t s = slot_of(key);
            bool fresh = false, placed = false;
            for (int probe = 0; probe < kSlots; ++probe) {
                const unsigned long long old = atomicCAS(&set[s], 0ull, key);
                if (old == 0ull) {
                    fresh = placed = true;
                    break;
                }
                if (old == key) {
                    placed = true;
                    break;
                }
                s = (s + 1) & (uint32_t)(kSlots - 1);
            }
            if (!placed) atomicOr(reinterpret_cast<unsigned int *>(count), 0x80000000u);  // cannot happen below kMaxBlocks
            if (fresh) {
                const int p = warp_append(count);
                if (p >= 0 && p < cap) {
                    coords[3 * p + 0] = (short)cur[0];
                    coords[3 * p + 1] = (short)cur[1];
                    coords[3 * p + 2] = (short)cur[2];
                }
            }
        }
        if (more) {
            if (left[0] + left[1] + left[2] == 0) {
                more = false;
            } else {
                int a = -1;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    if (left[i] > 0 && (a < 0 || tmax[i] < tmax[a])) a = i;
                cur[a] += step[a];
                tmax[a] = fadd(tmax[a], tdelta[a]);
                left[a] -= 1;
            }
        }
    }
}

// Upper bound on the distinct blocks a frame can touch: per pixel the DDA
// visits |dbx| + |dby| + |dbz| + 1 blocks, and the segment spans at most
// 2 mu |r| / (8 s) block units, |r| largest at an image corner.
double block_bound(const itm_intrinsics *in, float voxel_size, float mu)
{
    double rmax = 0.0;
    const double us[2] = {0.0, (double)in->width - 1.0}, vs[2] = {0.0, (double)in->height - 1.0};
    for (double u : us)
        for (double v : vs) {
            const double x = (u - in->cx) / in->fx, y = (v - in->cy) / in->fy;
            const double r = sqrt(x * x + y * y + 1.0);
            rmax = r > rmax ? r : rmax;
        }
    const double len_blocks = 2.0 * (double)mu * rmax / (8.0 * (double)voxel_size);
    const double per_pixel = floor(sqrt(3.0) * len_blocks) + 4.0;
    return per_pixel * (double)in->width * (double)in->height;
}

}  // namespace

}  // namespace itm

using namespace itm;

extern "C" int itm_frame_blocks_noalloc(const float *depth_dev, const itm_intrinsics *intr, const float T_wc[16],
                                        float voxel_size, float mu, float z_min, float z_max, int16_t *coords_dev,
                                        int cap, int32_t *count_dev, itm_stream stream)
{
    if (!depth_dev || !count_dev || !T_wc || !valid_intr(intr) || cap < 0 || (cap > 0 && !coords_dev))
        return ITM_ERR_ARG;
    if (!(voxel_size > 0.0f) || !(mu > 0.0f) || !(z_min > 0.0f) || !(z_max > z_min)) return ITM_ERR_ARG;
    for (int i = 0; i < 16; ++i)
        if (!isfinite(T_wc[i])) return ITM_ERR_ARG;
    if (block_bound(intr, voxel_size, mu) > (double)kMaxBlocks) return ITM_ERR_TOO_LARGE;  // beyond the fixed scratch
    unsigned long long *set = nullptr;
    int r = set_address(&set);
    if (r != ITM_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(set, 0, sizeof(unsigned long long) * (size_t)kSlots, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(count_dev, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return ITM_ERR_CUDA;
    Mat34 T;
    pose_rows(T_wc, T);
    const float inv_b = (float)(1.0 / (8.0 * (double)voxel_size));
    dim3 grid((intr->width + 31) / 32, (intr->height + 7) / 8);
    frame_blocks_kernel<<<grid, 256, 0, st>>>(set, depth_dev, to_intr(intr), T, inv_b, mu, z_min, z_max,
                                              reinterpret_cast<short *>(coords_dev), cap, count_dev);
    return check_cuda(cudaGetLastError());
}
