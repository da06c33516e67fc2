// Sec. 4.3 integration over the visible blocks.
//
// Launch shape: a persistent grid of 64-thread CTAs walks the visible list
// (its length is read from device memory).  A CTA takes one 8^3 block per
// iteration; thread t owns the x-row of voxels 8t .. 8t+7 (y = t & 7,
// z = t >> 3): 32 contiguous bytes of sdf and 8 of weights, so each warp
// covers four z-slices with fully coalesced 16-byte accesses.  The next
// block's index, coordinates and row data are requested before the current
// block is processed (a two-stage software pipeline over the visible list).
//
// Each voxel runs the listing computeUpdatedVoxelDepthInfo with IEEE
// round-to-nearest results in the listing's order (no product fused into a
// sum), so the skip decisions, the pixel read, the weights and the sdf values
// are reproducible bit for bit.  The thread first projects its eight voxels
// (no memory access), then issues their eight depth reads together, then
// takes the update decisions: the reads overlap instead of waiting on each
// other.  The kernel is bound by instruction issue, so the arithmetic runs on
// voxel pairs with the packed FP32x2 add / multiply / FMA of sm_100+, and
// each of the four quotients per voxel (u, v, eta / mu, the running mean) is
// the correctly rounded quotient from a correctly rounded reciprocal plus
// FMA residual corrections (Markstein 1990) instead of an IEEE division: one
// reciprocal of Z serves both pixel coordinates, 1 / mu is computed once per
// scene and 1 / (W + 1) comes from a 256-entry table in shared memory.  The
// pixel index is truncated by a round-toward-zero add of 2^23 instead of
// conversion instructions.
//
// Blocks that the visible list marks interior (kVisInterior), when the list
// was built for this pose and intrinsics (interior_ok, decided by the host),
// skip the per-voxel image-bounds and reciprocal-range tests.
//
// The decision needs no voxel data: a thread loads a 16-byte quad of sdf
// only when one of its four voxels is updated (and its 8 bytes of weights
// when any of its eight is), and stores it back after the update.  Skipped
// voxels cost no HBM traffic.
#include "itm_ops.cuh"

namespace itm {

namespace {

constexpr int kThreads = 64;

template <int MODE>  // 0: constant weight 1, uint8 weights; 1: per-pixel weight, float weights
__global__ void __launch_bounds__(kThreads) integrate_kernel(SceneDev s, const float *__restrict__ depth,
                                                             const float *__restrict__ wpx, Intr in, Mat34 M,
                                                             float2 nz, int interior_ok)
{
    __shared__ float2 rcp_w[256];
    if (MODE == 0) {
        fill_rcp_w(rcp_w);
        __syncthreads();
    }
    grid_dep_wait();
    const int n = min(__ldcg(&s.ctr->n_visible), s.nv);
    const int t = threadIdx.x;
    unsigned updated = 0;
    int i = blockIdx.x;
    int e = 0;  // visible-list entry: block index and interior flag
    short4 b = make_short4(0, 0, 0, 0);
    RowData row;
    if (i < n) {
        e = __ldg(&s.visible[i]);
        b = __ldg(&s.block_pos[vis_ptr(e)]);
        row = load_row<MODE>(s, vis_ptr(e), t);
    }
    while (i < n) {
        // the next block's index, coordinates and row data are requested
        // before this block's update, which hides their latency
        const int i_next = i + gridDim.x;
        int e_next = 0;
        short4 b_next = b;
        RowData row_next = row;
        if (i_next < n) {
            e_next = __ldg(&s.visible[i_next]);
            b_next = __ldg(&s.block_pos[vis_ptr(e_next)]);
            row_next = load_row<MODE>(s, vis_ptr(e_next), t);
        }
        if (interior_ok && (e & kVisInterior))
            integrate_block<MODE, true>(s, depth, wpx, in, M, vis_ptr(e), b, t, updated, row, rcp_w, nz);
        else
            integrate_block<MODE, false>(s, depth, wpx, in, M, vis_ptr(e), b, t, updated, row, rcp_w, nz);
        i = i_next;
        e = e_next;
        b = b_next;
        row = row_next;
    }

    grid_dep_launch();
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
                             const Mat34 &M_d, bool interior_ok, cudaStream_t st)
{
    const float2 nz = make_float2(-0.0f, -0.0f);
    const int io = interior_ok ? 1 : 0;
    if (wpx)
        return launch_pdl(integrate_kernel<1>, dim3(integrate_grid<1>()), dim3(kThreads), 0, st, s, depth, wpx, in,
                          M_d, nz, io);
    return launch_pdl(integrate_kernel<0>, dim3(integrate_grid<0>()), dim3(kThreads), 0, st, s, depth,
                      (const float *)nullptr, in, M_d, nz, io);
}

}  // namespace itm
