// k_batch.cu -- batched launch: ticket reset, the persistent kernel of the sequence, and the
// per-instrument theta reduction.
#include "rqmc_internal.h"

namespace rqmc {

template <int SEQ>
cudaError_t launch_batch_seq(const BatchLaunch &bl, int kind, cudaStream_t st);

// theta of every instrument: block = instrument, threads over (m, o), tiles summed in order
__global__ void batch_theta_kernel(const BatchInst *__restrict__ insts, const double *__restrict__ partials,
                                   double *__restrict__ theta) {
    const BatchInst &bi = insts[blockIdx.x];
    const int nout = bi.nout, M = bi.g.M;
    const double *pb = partials + bi.part_off;
    for (int idx = threadIdx.x; idx < M * nout; idx += blockDim.x) {
        const int m = idx / nout, o = idx % nout;
        const double *p = pb + (size_t)m * bi.tiles_per_m * nout + o;
        double s = 0.0;
        for (uint32_t t = 0; t < bi.tiles_per_m; ++t) s += p[(size_t)t * nout];
        theta[bi.theta_off + idx] = s / (double)bi.N;
    }
}

// [reset the tickets] -> fork: classes 1.. on side streams | class 0 on st -> join ->
// theta.  No kernel waits on another, so any co-scheduling of them is safe.
cudaError_t launch_batch(const BatchLaunch &bl, int seq, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bl.counter, 0, kBatchClasses * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bl.stats, 0, sizeof(unsigned long long) * 3 * kBatchClasses * bl.stats_cap, st)) !=
        cudaSuccess)
        return e;
    bool forked[kBatchClasses] = {};
    if ((e = cudaEventRecord(bl.fork, st)) != cudaSuccess) return e;
    for (int k = 1; k < kBatchClasses; ++k) {
        if (bl.n_items[k] == 0) continue;
        cudaStream_t sk = bl.side[k - 1];
        if ((e = cudaStreamWaitEvent(sk, bl.fork, 0)) != cudaSuccess) return e;
#define RQMC_L(S) launch_batch_seq<S>(bl, k, sk)
        e = RQMC_SEQ_DISPATCH(seq, RQMC_L);
#undef RQMC_L
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(bl.join[k - 1], sk)) != cudaSuccess) return e;
        forked[k] = true;
    }
    if (bl.n_items[0] > 0) {
#define RQMC_L(S) launch_batch_seq<S>(bl, 0, st)
        e = RQMC_SEQ_DISPATCH(seq, RQMC_L);
#undef RQMC_L
        if (e != cudaSuccess) return e;
    }
    for (int k = 1; k < kBatchClasses; ++k)
        if (forked[k] && (e = cudaStreamWaitEvent(st, bl.join[k - 1], 0)) != cudaSuccess) return e;
    batch_theta_kernel<<<bl.n_inst, 256, 0, st>>>(bl.insts, bl.partials, bl.theta);
    return cudaGetLastError();
}

}  // namespace rqmc
