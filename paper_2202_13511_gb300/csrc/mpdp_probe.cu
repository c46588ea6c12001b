// Read bandwidth of this GPU's memory hierarchy, measured in one launch:
// the roofline denominator for kernels whose memo reads are served by the
// L2 cache (a buffer smaller than the L2 read many times) or by HBM (a
// buffer far larger than it).  Not part of the join-order method.
#include <cuda_runtime.h>

#include "../../include/mpdp.h"

namespace {

// Every thread reads 16-byte words with a grid stride, `passes` times over
// the buffer; the xor of everything read goes to one word so that no read
// can be dropped.
__global__ void __launch_bounds__(512) k_probe_read(const uint4* __restrict__ buf, size_t words, int passes,
                                                    unsigned* __restrict__ sink)
{
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; p++)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc.x ^= v.x;
            acc.y ^= v.y;
            acc.z ^= v.z;
            acc.w ^= v.w;
        }
    const unsigned r = acc.x ^ acc.y ^ acc.z ^ acc.w;
    if (r == 0x9e3779b9u) sink[0] = r;  // practically never taken, but not provably
}

}  // namespace

extern "C" int mpdp_probe_read_gbs(int device, size_t bytes, int passes, double* gbs)
{
    if (!gbs || bytes < 4096 || passes < 1) return MPDP_ERR_INVALID_ARG;
    *gbs = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t words = bytes / sizeof(uint4);
    uint4* buf = nullptr;
    unsigned* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MPDP_OK;
    if (cudaMalloc(&buf, words * sizeof(uint4)) != cudaSuccess || cudaMalloc(&sink, sizeof(unsigned)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MPDP_ERR_OOM;
    }
    if (rc == MPDP_OK && cudaMemset(buf, 0x5a, words * sizeof(uint4)) != cudaSuccess) rc = MPDP_ERR_CUDA;
    float best = 0.f;
    if (rc == MPDP_OK) {
        const int grid = sms * 4;
        k_probe_read<<<grid, 512>>>(buf, words, 1, sink);  // warm: brings a small buffer into the L2
        for (int rep = 0; rep < 5 && rc == MPDP_OK; rep++) {
            cudaEventRecord(e0);
            k_probe_read<<<grid, 512>>>(buf, words, passes, sink);
            cudaEventRecord(e1);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = MPDP_ERR_CUDA;
            else if (ms > 0.f) {
                const float g = (float)((double)words * sizeof(uint4) * passes / (ms * 1e-3) / 1e9);
                if (g > best) best = g;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    cudaGetLastError();
    *gbs = best;
    return rc;
}
