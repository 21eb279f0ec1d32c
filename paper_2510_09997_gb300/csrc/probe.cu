// probe.cu -- FP32 fused multiply-add throughput of this GPU (a measurement
// aid: the roofline peak of the FP32-bound blend is measured rather than
// taken from the data sheet).  Each thread runs 8 independent FMA chains;
// the caller times the launch.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

clod_status fail(clod_status s, const char* fmt, ...);
clod_status cuda_fail(cudaError_t e, const char* what);
clod_status device_ready(int* n_sm);

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(float* __restrict__ sink, int iters)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    const float b = 0.99993f, c = 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == -1.0f) sink[0] = s;   // never true (every chain stays positive); keeps the chains live
}

}  // namespace clod

using namespace clod;

extern "C" clod_status clod_probe_fma(int32_t iters, float* sink, uint64_t* flops, clod_stream stream)
{
    if (iters < 1 || !sink || !flops) return fail(CLOD_ERR_ARG, "bad argument to clod_probe_fma");
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    const int blocks = n_sm * (2048 / PROBE_THREADS);   // a full wave at the SM's thread limit
    k_fma_probe<<<blocks, PROBE_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(sink, iters);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_probe_fma launch");
    *flops = 2ull * PROBE_CHAINS * (uint64_t)iters * (uint64_t)blocks * PROBE_THREADS;
    return CLOD_OK;
}
