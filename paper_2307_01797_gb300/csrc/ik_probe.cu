// ik_probe.cu -- the FP64 arithmetic peak of the device, measured.
//
// The FP64 form of the step is bound by the device's FP64 units, not by its
// memory.  The denominator of that roofline is measured here: every SM runs
// blocks of independent fused-multiply-add chains held in registers (no
// memory traffic inside the timed loop), timed with CUDA events.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/itokmc.h"
#include "ik_state.h"

namespace ik {
namespace {

constexpr int PROBE_CHAINS = 8;      // independent accumulators per thread (hide the FMA latency)

__global__ void __launch_bounds__(256) k_dfma_loop(double* __restrict__ out, int iters, double a, double b)
{
    double c[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) c[k] = (double)(threadIdx.x + k) * 1e-9;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) c[k] = __fma_rn(c[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += c[k];
    if (s == 12345.678) out[blockIdx.x] = s;          // keeps the loop live; never true for a, b below
}

}  // namespace
}  // namespace ik

extern "C" int itokmc_probe_fp64_peak(void* stream, double* tflops_out, double* ms_out)
{
    using namespace ik;
    if (!tflops_out) { set_global_error("probe_fp64_peak: NULL output"); return ITOKMC_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("probe_fp64_peak: no CUDA device");
        return ITOKMC_ERR_CUDA;
    }
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * 8192) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("probe_fp64_peak: device allocation failed");
        return ITOKMC_ERR_OOM;
    }
    const int blocks = sms * 8, tpb = 256, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    g_launches += 4;
    k_dfma_loop<<<blocks, tpb, 0, s>>>(out, iters, 0.999999, 1e-7);       // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        k_dfma_loop<<<blocks, tpb, 0, s>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f && ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) {
        set_global_error("probe_fp64_peak: CUDA error");
        return ITOKMC_ERR_CUDA;
    }
    const double flop = 2.0 * PROBE_CHAINS * (double)iters * (double)blocks * tpb;
    *tflops_out = flop / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return ITOKMC_OK;
}
