// k_batch.cuh -- one persistent launch over a batch of heterogeneous instruments (LMM caplet
// strips of 8..160 forwards and MBS of up to 4096 months), instantiated per sequence by
// k_batch_{halton,sobol,philox}.cu.
//
// Work items are (instrument, replication m, tile of consecutive points), listed longest
// first (LPT).  Each CTA takes the next item with one atomicAdd on a ticket counter -- no
// CTA ever waits on another, so the loop cannot deadlock -- stages that instrument's tables
// for m into shared memory, runs the tile's paths with the same path code as the
// single-instrument kernels (FP32 paths, Kahan sums) and writes the item's own partial
// row.  Results therefore do not depend on which CTA took which item.
#pragma once
#include "k_lmm.cuh"
#include "k_mbs.cuh"

namespace rqmc {

template <int NF, int SEQ>
__device__ __forceinline__ void batch_lmm(const BatchInst &bi, const BatchItem &it, const GenView &gv,
                                          const RedParams &r, unsigned char *smem_raw) {
    using V2 = float2;
    constexpr int PAD = LmmMath<float>::PAD;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LmmModel<float> *md = bi.lmm;
    const int nK = md->nK, nout = r.nout;
    size_t o_cst, o_x0, o_z, o_buf, o_acc;
    lmm_smem_layout<NF, float>(bi.g, nw, nK, nout, &o_cst, &o_x0, &o_z, &o_buf, &o_acc);
    float *zb = reinterpret_cast<float *>(smem_raw + o_z) + threadIdx.x;
    V2 *cst = reinterpret_cast<V2 *>(smem_raw + o_cst);
    float *X0 = reinterpret_cast<float *>(smem_raw + o_x0);
    float *Ks = X0 + NF;
    float *wbuf = reinterpret_cast<float *>(smem_raw + o_buf) + (size_t)warp * 8 * nK * PAD;
    float *acc = reinterpret_cast<float *>(smem_raw + o_acc);
    float *cmp = acc + nw * nout;
    for (int k = threadIdx.x; k < NF; k += blockDim.x) {
        cst[k] = V2{md->sig[k], md->cc[k]};
        X0[k] = md->X0[k];
    }
    if (threadIdx.x < kMaxStrikes) Ks[threadIdx.x] = md->K[threadIdx.x];
    zero_acc(acc, cmp, nw * nout);
    const LmmScal<float> sc{md->nf, md->nK, md->dl, md->inv_dl, md->disc0, md->hc, md->sqhc};
    __syncthreads();
    for (int pp = 0; pp < r.ppt; ++pp) {
        const uint32_t i = it.tile * r.tile + (uint32_t)(pp * blockDim.x + threadIdx.x);
        const bool active = i < r.N;
        if (!__any_sync(0xffffffffu, active)) break;
        PathGen<SEQ> pg[1];
        pg[0].init(gv, active ? i : 0u);
        const bool act[1] = {active};
        lmm_path<NF, SEQ, float, 1>(pg, act, sc, cst, X0, Ks, zb, wbuf, acc + warp * nout, cmp + warp * nout, lane);
    }
    flush_unit(r, it.m * bi.tiles_per_m + it.tile, acc, cmp);
}

template <int SEQ>
__device__ __forceinline__ void batch_mbs(const BatchInst &bi, const BatchItem &it, const GenView &gv,
                                          const RedParams &r, unsigned char *smem_raw) {
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const MbsModel<float> md = *bi.mbs;
    float *acc = reinterpret_cast<float *>(smem_raw + stage_bytes(bi.g));
    float *cmp = acc + nw;
    float *ck = cmp + nw;
    for (int k = threadIdx.x; k <= md.months; k += blockDim.x) ck[k] = md.ck[k];
    zero_acc(acc, cmp, nw);
    __syncthreads();
    for (int pp = 0; pp < r.ppt; ++pp) {
        const uint32_t i = it.tile * r.tile + (uint32_t)(pp * blockDim.x + threadIdx.x);
        const bool active = i < r.N;
        if (!__any_sync(0xffffffffu, active)) break;
        PathGen<SEQ> pg;
        pg.init(gv, active ? i : 0u);
        const float v = mbs_path<float, SEQ>(pg, md, ck);
        warp_accumulate<float>(active ? v : 0.0f, acc + warp, cmp + warp, 0, lane);
    }
    flush_unit(r, it.m * bi.tiles_per_m + it.tile, acc, cmp);
}

template <int SEQ>
__global__ void __launch_bounds__(256, 1) batch_kernel(const BatchInst *__restrict__ insts,
                                                       const BatchItem *__restrict__ items, uint32_t n_items,
                                                       uint32_t *counter, double *partials, int ppt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_ticket;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = s_ticket;
        __syncthreads();   // every thread has read the ticket before thread 0 takes the next one
        if (t >= n_items) break;
        const BatchItem it = items[t];
        const BatchInst &bi = insts[it.inst];
        GenView gv;
        stage_tables(bi.g, (int)it.m, smem_raw, gv);
        RedParams r;
        r.nout = bi.nout;
        r.ppt = ppt;
        r.tile = blockDim.x * (uint32_t)ppt;
        r.tiles_per_m = bi.tiles_per_m;
        r.units = bi.tiles_per_m * (uint32_t)bi.g.M;
        r.N = bi.N;
        r.partials = partials + bi.part_off;
        r.status = nullptr;
        if (bi.kind == 0) {
            switch (bi.bucket) {
                case 16: batch_lmm<16, SEQ>(bi, it, gv, r, smem_raw); break;
                case 40: batch_lmm<40, SEQ>(bi, it, gv, r, smem_raw); break;
                case 80: batch_lmm<80, SEQ>(bi, it, gv, r, smem_raw); break;
                default: batch_lmm<160, SEQ>(bi, it, gv, r, smem_raw); break;
            }
        } else {
            batch_mbs<SEQ>(bi, it, gv, r, smem_raw);
        }
    }
}

template <int SEQ>
cudaError_t launch_batch_seq(const BatchLaunch &bl, cudaStream_t st) {
    auto kern = batch_kernel<SEQ>;
    if (bl.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bl.smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bl.threads, bl.smem);
    if (occ < 1) occ = 1;
    const unsigned grid = (unsigned)std::min<unsigned long long>(bl.n_items, (unsigned long long)occ * sms);
    kern<<<grid, bl.threads, bl.smem, st>>>(bl.insts, bl.items, bl.n_items, bl.counter, bl.partials, bl.ppt);
    return cudaGetLastError();
}

}  // namespace rqmc
