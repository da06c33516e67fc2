// GPU check of the integration's reciprocal: itm::rcp_rn (the hardware's
// approximate reciprocal refined by one Newton-Raphson step) must equal the
// IEEE round-to-nearest reciprocal __frcp_rn on every float of the range the
// kernels use it on, [2^-64, 2^64), and rcp_out_of_range must flag exactly
// the positive floats outside it (NaN excepted).  Prints the two mismatch counts.
#include <cstdio>

#include "itm_ops.cuh"

__global__ void check(unsigned long long n, unsigned long long *bad)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    // i enumerates the positive floats 0x00000001 .. 0x7fffffff (incl. inf, NaN)
    const unsigned bits = (unsigned)i + 1u;
    const float x = __uint_as_float(bits);
    const bool in_range = bits >= 0x1F800000u && bits < 0x5F800000u;  // [2^-64, 2^64)
    if (in_range && __float_as_uint(itm::rcp_rn(x)) != __float_as_uint(__frcp_rn(x))) atomicAdd(&bad[0], 1ull);
    // (a NaN is not > 0: the kernels' Z > 0 test rejects such a voxel already)
    if (!isnan(x) && itm::rcp_out_of_range(x) == in_range) atomicAdd(&bad[1], 1ull);
}

int main()
{
    unsigned long long *bad = nullptr, h[2] = {1, 1};
    if (cudaMalloc(&bad, sizeof(h)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, sizeof(h));
    const unsigned long long n = 0x7fffffffull;
    check<<<(unsigned)((n + 255) / 256), 256>>>(n, bad);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    printf("%llu %llu\n", h[0], h[1]);
    return 0;
}
