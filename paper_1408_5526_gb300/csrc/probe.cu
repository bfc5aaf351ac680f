// probe.cu -- issue-rate microbenchmarks of the pipes the path kernels are bound by (not in
// the paper): ex2, rcp and lg2 on the SFU, the forward update's ex2 + rcp pair, and FP32
// FMA, each as operations per SM per clock.  The ALU/SFU rooflines of the path kernels are
// derived from unit counts and clocks; these measured rates stand beside them.
//
// Each probe thread keeps 8 independent chains and runs a fixed number of iterations (no
// waits, no data-dependent exits), with 64 warps per SM; the result feeds a store so the
// work cannot be removed.
#include <cmath>

#include "rqmc_internal.h"

namespace rqmc {

enum ProbeOp { kProbeEx2 = 0, kProbeRcp = 1, kProbeLg2 = 2, kProbePair = 3, kProbeFma = 4, kProbeOps = 5 };

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(float *out, int iters) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = -6.0f + 0.01f * (float)(threadIdx.x & 31) + 0.1f * (float)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (OP == kProbeEx2) x[k] = ex2_approx(-x[k]) - 6.0f;
            else if constexpr (OP == kProbeRcp) x[k] = rcp_approx(x[k]) - 6.0f;
            else if constexpr (OP == kProbeLg2) x[k] = lg2_approx(-x[k]) - 9.0f;
            else if constexpr (OP == kProbePair) x[k] = fmaf(rcp_approx(1.0f + ex2_approx(-x[k])), 1e-3f, x[k]);
            else x[k] = fmaf(x[k], 0.9999f, 1e-4f);
        }
    }
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <int OP>
static cudaError_t run_probe(float *buf, int blocks, int iters, cudaEvent_t a, cudaEvent_t b, float *ms) {
    probe_kernel<OP><<<blocks, 256>>>(buf, iters / 8);   // warm-up
    cudaEventRecord(a);
    probe_kernel<OP><<<blocks, 256>>>(buf, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace rqmc

using namespace rqmc;

extern "C" rqmc_status rqmc_probe_pipes(double *rates_host, int n) {
    if (!rates_host || n < kProbeOps) {
        set_error("rates_host must hold 5 values");
        return RQMC_EINVAL;
    }
    int dev = 0, sms = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || sms < 1 || khz < 1) {
        set_error("device query failed");
        return RQMC_ECUDA;
    }
    const int blocks = 8 * sms, iters = 2048;   // 64 warps per SM
    float *buf = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(float) * blocks * 256);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms[kProbeOps] = {0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = run_probe<kProbeEx2>(buf, blocks, iters, a, b, &ms[0]);
    if (e == cudaSuccess) e = run_probe<kProbeRcp>(buf, blocks, iters, a, b, &ms[1]);
    if (e == cudaSuccess) e = run_probe<kProbeLg2>(buf, blocks, iters, a, b, &ms[2]);
    if (e == cudaSuccess) e = run_probe<kProbePair>(buf, blocks, iters, a, b, &ms[3]);
    if (e == cudaSuccess) e = run_probe<kProbeFma>(buf, blocks, iters, a, b, &ms[4]);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) {
        set_error(std::string("probe failed: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    // operations per SM per clock at the device's rated clock (the pair counts one update)
    const double ops = (double)blocks * 256.0 * iters * 8.0;
    for (int k = 0; k < kProbeOps; ++k)
        rates_host[k] = ms[k] > 0.0f ? ops / (ms[k] * 1e-3) / sms / (khz * 1e3) : 0.0;
    return RQMC_OK;
}
