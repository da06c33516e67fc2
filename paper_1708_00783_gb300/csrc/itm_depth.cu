// Sec. 4 view preparation (unsigned short millimetres -> float metres) and
// the scene reset fills.  Both are plain streaming kernels: 16-byte loads and
// stores, grid sized to a multiple of the SM count.
#include "itm_internal.cuh"

namespace itm {

namespace {

int stream_grid()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = sms * 8;
    }
    return g;
}

// d = raw / 1000, correctly rounded (IEEE division)
__global__ void __launch_bounds__(256) depth_u16_kernel(const uint16_t *__restrict__ raw, float *__restrict__ out,
                                                        int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n8 = n / 8;
    const bool aligned = ((reinterpret_cast<uintptr_t>(raw) & 15) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (aligned) {
        for (; i < n8; i += stride) {
            const uint4 r = __ldcs(reinterpret_cast<const uint4 *>(raw) + i);
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
            float f[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                f[2 * k] = __fdiv_rn((float)(w[k] & 0xffffu), 1000.0f);
                f[2 * k + 1] = __fdiv_rn((float)(w[k] >> 16), 1000.0f);
            }
            float4 *o = reinterpret_cast<float4 *>(out) + 2 * i;
            __stcs(o, make_float4(f[0], f[1], f[2], f[3]));
            __stcs(o + 1, make_float4(f[4], f[5], f[6], f[7]));
        }
        i = n8 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    }
    for (; i < n; i += stride) out[i] = __fdiv_rn((float)raw[i], 1000.0f);
}

__global__ void reset_entries_kernel(SceneDev s)
{
    const int total = s.nb + s.ne;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        reinterpret_cast<int4 *>(s.entries)[i] = make_int4(0, 0, 0, -2);
        if (i < s.nb) s.req[i] = 0ull;
        if (i < s.ne) s.excess_free[i] = i;
    }
}

__global__ void reset_blocks_kernel(SceneDev s)
{
    const int64_t total4 = (int64_t)s.nv * (kBlockVoxels / 4);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total4; i += stride) {
        reinterpret_cast<float4 *>(s.sdf)[i] = make_float4(1.f, 1.f, 1.f, 1.f);  // Sec. 3.1 initial sdf
        if (s.w8) reinterpret_cast<uint32_t *>(s.w8)[i] = 0u;
        if (s.w32) reinterpret_cast<float4 *>(s.w32)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < s.nv) {
            s.block_free[i] = (int)i;
            s.block_pos[i] = make_short4(0, 0, 0, 0);
        }
    }
}

}  // namespace

cudaError_t launch_depth_u16(const uint16_t *raw, float *out, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t need = (n + 8 * 256 - 1) / (8 * 256);
    int g = (int)(need < stream_grid() ? need : stream_grid());
    depth_u16_kernel<<<g > 0 ? g : 1, 256, 0, st>>>(raw, out, n);
    return cudaGetLastError();
}

cudaError_t launch_reset(const SceneDev &s, cudaStream_t st)
{
    reset_entries_kernel<<<stream_grid(), 256, 0, st>>>(s);
    if (s.nv > 0) reset_blocks_kernel<<<stream_grid(), 256, 0, st>>>(s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(s.ctr, 0, sizeof(Counters), st);
}

}  // namespace itm
