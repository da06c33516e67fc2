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
// keeps it (so the entry point must not be used across a cudaDeviceReset,
// which frees the array behind that address).  Every call shares the array
// and clears it first; calls that overlap on the GPU (different streams, or a
// second host thread) race on it.
#include <math.h>

#include <mutex>

#include "itm_ops.cuh"

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

constexpr int kMaxProbes = 256;             // linear probes before a key gives up (load <= 1/2)
constexpr uint32_t kCountOverflow = 0x80000000u;  // *count bit: the fixed set overflowed
constexpr uint32_t kCountRange = 0x40000000u;     // *count bit: a pixel left the int16 block range
constexpr uint32_t kCountMask = 0x3fffffffu;

// One thread per pixel, 8x4-pixel warp tiles; the segment d-mu .. d+mu and
// the walk over the blocks it crosses are the allocation's own
// (segment_walk_setup / segment_walk_step, Sec. 4.2).  Each distinct block
// enters the set once and is appended to the caller's output.
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
    SegmentWalk g;
    const int seg = segment_walk_setup(u, v, d, in, T, inv_b, mu, z_min, z_max, g);
    if (seg == kSegRange) atomicOr(reinterpret_cast<unsigned int *>(count), kCountRange);
    bool more = seg == kSegWalk;
    while (__any_sync(kFull, more)) {
        const unsigned long long key = more ? pack_key(g.cur[0], g.cur[1], g.cur[2]) : 0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        if (more && lane == __ffs(peers) - 1) {
            uint32_t slot = slot_of(key);
            bool fresh = false, placed = false;
            for (int probe = 0; probe < kMaxProbes; ++probe) {
                const unsigned long long old = atomicCAS(&set[slot], 0ull, key);
                if (old == 0ull) {
                    fresh = placed = true;
                    break;
                }
                if (old == key) {
                    placed = true;
                    break;
                }
                slot = (slot + 1) & (uint32_t)(kSlots - 1);
            }
            if (!placed) atomicOr(reinterpret_cast<unsigned int *>(count), kCountOverflow);
            if (fresh) {
                const int p = (int)((uint32_t)warp_append(count) & kCountMask);
                if (p < cap) {
                    coords[3 * p + 0] = (short)g.cur[0];
                    coords[3 * p + 1] = (short)g.cur[1];
                    coords[3 * p + 2] = (short)g.cur[2];
                }
            }
        }
        if (more) more = segment_walk_step(g);
    }
}

// A rigid camera-to-world pose: last row 0 0 0 1 and orthonormal rotation
// rows (within float rounding); the size bound below assumes it.
bool rigid_pose(const float T[16])
{
    if (T[12] != 0.0f || T[13] != 0.0f || T[14] != 0.0f || T[15] != 1.0f) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double dot = 0.0;
            for (int k = 0; k < 3; ++k) dot += (double)T[4 * i + k] * (double)T[4 * j + k];
            if (fabs(dot - (i == j ? 1.0 : 0.0)) > 1e-4) return false;
        }
    return true;
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
    if (!rigid_pose(T_wc)) return ITM_ERR_ARG;
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
