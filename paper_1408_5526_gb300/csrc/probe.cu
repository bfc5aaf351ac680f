// probe.cu -- issue-rate microbenchmarks of the pipes the path kernels are bound by (not in
// the paper): ex2, rcp and lg2 on the SFU, the forward update's ex2 + rcp pair, FP32 FMA,
// FP64 FMA and the FP64 forward update's exp + reciprocal pair, each as operations per SM
// per clock.  The ALU/SFU rooflines of the path kernels are derived from unit counts and
// clocks; these measured rates stand beside them.
//
// Each probe thread keeps 8 independent chains and runs a fixed number of iterations (no
// waits, no data-dependent exits), with 64 warps per SM; the result feeds a store so the
// work cannot be removed.  The SM clock is measured inside the probe kernels themselves:
// thread 0 of every block reads the SM cycle counter and the global nanosecond timer at
// the start and the end of its block, so the rates are per clock at the clock the probes
// actually ran at, not at the device's rated clock.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rqmc_internal.h"

namespace rqmc {

enum ProbeOp {
    kProbeEx2 = 0, kProbeRcp = 1, kProbeLg2 = 2, kProbePair = 3, kProbeFma = 4, kProbeDfma = 5, kProbeDpair = 6,
    kProbeOps = 7
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(float *out, unsigned long long *clk, int iters) {
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        t0 = global_ns();
        c0 = clock64();
    }
    if constexpr (OP == kProbeDfma || OP == kProbeDpair) {
        double x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = -6.0 + 0.01 * (double)(threadIdx.x & 31) + 0.1 * (double)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (OP == kProbeDfma) x[k] = fma(x[k], 0.9999, 1e-4);
                else x[k] = fma(1.0 / (1.0 + exp(-x[k])), 1e-3, x[k]);
            }
        }
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += x[k];
        out[blockIdx.x * blockDim.x + threadIdx.x] = (float)t;
    } else {
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
    __syncthreads();
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = clock64() - c0;
        clk[2 * blockIdx.x + 1] = global_ns() - t0;
    }
}

template <int OP>
static cudaError_t run_probe(float *buf, unsigned long long *clk, int blocks, int iters, cudaEvent_t a, cudaEvent_t b,
                             float *ms, std::vector<double> &mhz) {
    probe_kernel<OP><<<blocks, 256>>>(buf, clk, iters / 8);   // warm-up
    cudaEventRecord(a);
    probe_kernel<OP><<<blocks, 256>>>(buf, clk, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<unsigned long long> h(2 * (size_t)blocks);
    if ((e = cudaMemcpy(h.data(), clk, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    for (int k = 0; k < blocks; ++k)
        if (h[2 * k + 1] > 0) mhz.push_back(1e3 * (double)h[2 * k] / (double)h[2 * k + 1]);
    return cudaSuccess;
}

}  // namespace rqmc

using namespace rqmc;

extern "C" rqmc_status rqmc_probe_pipes(double *rates_host, int n) {
    if (!rates_host || n < 5) {
        set_error("rates_host must hold at least 5 values");
        return RQMC_EINVAL;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        set_error("device query failed");
        return RQMC_ECUDA;
    }
    const int blocks = 8 * sms, iters = 2048;   // 64 warps per SM
    float *buf = nullptr;
    unsigned long long *clk = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(float) * blocks * 256);
    if (e == cudaSuccess) e = cudaMalloc(&clk, sizeof(unsigned long long) * 2 * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms[kProbeOps] = {0, 0, 0, 0, 0, 0, 0};
    std::vector<double> mhz;
    // the FP64 probes run fewer iterations: GB300's FP64 rate is a small fraction of FP32's
    if (e == cudaSuccess) e = run_probe<kProbeEx2>(buf, clk, blocks, iters, a, b, &ms[0], mhz);
    if (e == cudaSuccess) e = run_probe<kProbeRcp>(buf, clk, blocks, iters, a, b, &ms[1], mhz);
    if (e == cudaSuccess) e = run_probe<kProbeLg2>(buf, clk, blocks, iters, a, b, &ms[2], mhz);
    if (e == cudaSuccess) e = run_probe<kProbePair>(buf, clk, blocks, iters, a, b, &ms[3], mhz);
    if (e == cudaSuccess) e = run_probe<kProbeFma>(buf, clk, blocks, iters, a, b, &ms[4], mhz);
    if (e == cudaSuccess && n > kProbeDfma) e = run_probe<kProbeDfma>(buf, clk, blocks, iters / 8, a, b, &ms[5], mhz);
    if (e == cudaSuccess && n > kProbeDpair) e = run_probe<kProbeDpair>(buf, clk, blocks, iters / 64, a, b, &ms[6], mhz);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (buf) cudaFree(buf);
    if (clk) cudaFree(clk);
    if (e != cudaSuccess || mhz.empty()) {
        set_error(std::string("probe failed: ") + cudaGetErrorString(e));
        return RQMC_ECUDA;
    }
    // SM clock the probes ran at: median over every block of every probe
    std::nth_element(mhz.begin(), mhz.begin() + mhz.size() / 2, mhz.end());
    const double clock_mhz = mhz[mhz.size() / 2];
    const int iters_of[kProbeOps] = {iters, iters, iters, iters, iters, iters / 8, iters / 64};
    for (int k = 0; k < kProbeOps && k < n; ++k) {
        const double ops = (double)blocks * 256.0 * iters_of[k] * 8.0;   // the pairs count one update
        rates_host[k] = ms[k] > 0.0f ? ops / (ms[k] * 1e-3) / sms / (clock_mhz * 1e6) : 0.0;
    }
    if (n > kProbeOps) rates_host[kProbeOps] = clock_mhz;
    return RQMC_OK;
}
