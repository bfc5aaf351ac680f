// k_batch.cuh -- persistent kernels over a batch of heterogeneous instruments (LMM caplet
// strips of 8..160 forwards and MBS of up to 4096 months), one kernel per work class
// (160-forward strips, MBS, smaller strips; see BatchLaunch), instantiated per sequence by
// k_batch_{halton,sobol,philox}.cu.
//
// Work items are (instrument, replication m, tile of consecutive points), listed longest
// first (LPT) per class.  Each CTA takes its class's next item with one atomicAdd on a
// ticket counter -- no
// CTA ever waits on another, so the loop cannot deadlock -- stages that instrument's tables
// for m into shared memory, runs the tile's paths with the same path code as the
// single-instrument kernels (FP32 paths, Kahan sums) and writes the item's own partial
// row.  Results therefore do not depend on which CTA took which item.
#pragma once
#include "k_lmm.cuh"
#include "k_mbs.cuh"

namespace rqmc {

// Paths per thread in lockstep per bucket, sized to the register budget of the bucket's
// work class (16/40/80 forwards: 2 CTAs per SM, 128 registers; 160: 1 CTA per SM).  MBS
// paths go mbs_paths32(SEQ) per thread, as in the MBS kernel: their coordinates and the
// central inverse-CDF branch are generated together.
template <int NF>
__host__ __device__ constexpr int batch_ilp() {
    return NF <= 16 ? 4 : NF <= 40 ? 2 : 1;
}


// Work class of an instrument (see BatchLaunch).
__host__ __device__ inline int batch_class(const BatchInst &bi) { return bi.kind != 0 ? 1 : bi.bucket == 160 ? 0 : 2; }

// Strips of 40 and more forwards draw an item's normals before its paths (batch_item_normals)
// and read them like the normals-loaded caplet kernel; 16-forward strips draw them in the
// step loop (their four lockstep paths would need a 64 KB double buffer).  Measured on the
// 512-instrument batch (Sobol'): the 81..160-forward class 6 % faster.  Leaving only the
// 80-forward strips on in-loop generation measured 7 % slower for them (one strip, N = 65536,
// M = 16) than this choice.
__host__ __device__ constexpr bool batch_zg_bucket(int bucket) { return bucket >= 40; }
template <int NF>
__host__ __device__ constexpr bool batch_zg() {
    return batch_zg_bucket(NF);
}

// The normals of the item's points i0 .. i0 + np - 1 (np <= ld) in dimensions 0 .. nd - 1, by
// all threads of the CTA: z[j ld + (i - i0)].  A task is one lane-run of 8 consecutive points
// in a block of 4 dimensions (the Philox counter block); the 8 points are drawn in lockstep,
// each value bit-identical to the path's own draw.  Points past N repeat point N - 1 (never
// read: a path past N reads slot 0).
template <int SEQ>
__device__ __forceinline__ void batch_item_normals(const GenView &gv, uint32_t i0, uint32_t np, uint32_t N, int nd,
                                                   float *__restrict__ z, uint32_t ld) {
    const uint32_t nrun = (np + 7) >> 3, nblk = (uint32_t)(nd + 3) >> 2;
    for (uint32_t t = threadIdx.x; t < nrun * nblk; t += blockDim.x) {
        const uint32_t jb = t / nrun, r = t % nrun;
        PathGen<SEQ> pg[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) pg[k].init(gv, min(i0 + 8 * r + (uint32_t)k, N - 1));
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * (int)jb + jj;
            if (j >= nd) break;
            float v[8];
            normals32<SEQ, 8>(pg, j, v);
            float4 *dst = reinterpret_cast<float4 *>(z + (size_t)j * ld + 8 * r);
            dst[0] = make_float4(v[0], v[1], v[2], v[3]);
            dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
    }
}

// zs: this CTA's normals buffer (batch_zg<NF> strips), at least NF x r.tile floats.
template <int NF, int SEQ>
__device__ __forceinline__ void batch_lmm(const BatchInst &bi, const BatchItem &it, const GenView &gv,
                                          const RedParams &r, unsigned char *smem_raw, float *zs) {
    using CC = float4;
    constexpr int PAD = LmmMath<float>::PAD;
    constexpr bool ZG = batch_zg<NF>();
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LmmModel<float> *md = bi.lmm;
    const int nK = md->nK, nout = r.nout;
    constexpr int P = batch_ilp<NF>();
    size_t o_cst, o_x0, o_z, o_buf, o_acc;
    lmm_smem_layout<NF, float, P>(bi.g, nw, nK, nout, &o_cst, &o_x0, &o_z, &o_buf, &o_acc, ZG ? 2 : 1);
    float *zb = reinterpret_cast<float *>(smem_raw + o_z) + threadIdx.x;
    CC *cst = reinterpret_cast<CC *>(smem_raw + o_cst);
    float *X0 = reinterpret_cast<float *>(smem_raw + o_x0);
    float *Ks = X0 + NF;
    float *wbuf = reinterpret_cast<float *>(smem_raw + o_buf) + (size_t)warp * 8 * nK * PAD;
    float *acc = reinterpret_cast<float *>(smem_raw + o_acc);
    float *cmp = acc + nw * nout;
    lmm_fill_constants<NF, float>(*md, cst, X0);
    if (threadIdx.x < kMaxStrikes) Ks[threadIdx.x] = md->K[threadIdx.x];
    zero_acc(acc, cmp, nw * nout);
    const LmmScal<float> sc{md->nf, md->nK, md->dl, md->inv_dl, md->disc0, md->hc, md->sqhc};
    const uint32_t i0 = it.tile * r.tile;   // the item's first point
    if constexpr (ZG) batch_item_normals<SEQ>(gv, i0, min(r.tile, r.N - i0), r.N, md->nf, zs, r.tile);
    __syncthreads();
    for (int pp = 0; pp < r.ppt; pp += P) {
        PathGen<SEQ> pg[P];
        bool act[P];
        bool any = false;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t i = i0 + (uint32_t)((pp + p) * blockDim.x + threadIdx.x);
            act[p] = pp + p < r.ppt && i < r.N;
            any = any || act[p];
            pg[p].init(gv, act[p] ? i : i0);
        }
        if (!__any_sync(0xffffffffu, any)) break;
        // payoff with delta applied per step (DK = false): the (delta L - delta K) form makes the
        // small-strip class spill under its 128-register budget (measured 10 % slower)
        lmm_path<NF, SEQ, float, P, false, ZG, false>(pg, act, sc, cst, X0, Ks, zb, wbuf, acc + warp * nout,
                                                      cmp + warp * nout, lane, zs, r.tile, i0);
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
    constexpr int P = mbs_paths32(SEQ);
    for (int pp = 0; pp < r.ppt; pp += P) {
        PathGen<SEQ> pg[P];
        bool act[P];
        bool any = false;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t i = it.tile * r.tile + (uint32_t)((pp + p) * blockDim.x + threadIdx.x);
            act[p] = pp + p < r.ppt && i < r.N;
            any = any || act[p];
            pg[p].init(gv, act[p] ? i : 0u);
        }
        if (!__any_sync(0xffffffffu, any)) break;
        float v[P];
        mbs_paths<float, SEQ, P>(pg, md, ck, v);
#pragma unroll
        for (int p = 0; p < P; ++p) warp_accumulate<float>(act[p] ? v[p] : 0.0f, acc + warp, cmp + warp, 0, lane);
    }
    flush_unit(r, it.m * bi.tiles_per_m + it.tile, acc, cmp);
}

// One persistent kernel per work class KIND (see BatchLaunch).
// CTA timing record: SM id, global-timer start and end of the CTA's item loop.
__device__ __forceinline__ unsigned long long batch_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t batch_smid() {
    uint32_t id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

template <int SEQ, int KIND>
__global__ void __launch_bounds__(256, KIND == 0 ? 1 : KIND == 1 ? 4 : 2) batch_kernel(const BatchInst *__restrict__ insts,
                                                                    const BatchItem *__restrict__ items,
                                                                    uint32_t n_items, uint32_t *counter,
                                                                    double *partials, int ppt,
                                                                    unsigned long long *stats, uint32_t stats_cap,
                                                                    float *znorm, size_t zstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_ticket;
    const unsigned long long t_start = batch_clock();
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
        float *zs = znorm ? znorm + (size_t)blockIdx.x * zstride : nullptr;   // the CTA's normals buffer
        if constexpr (KIND == 0) {
            batch_lmm<160, SEQ>(bi, it, gv, r, smem_raw, zs);
        } else if constexpr (KIND == 2) {
            switch (bi.bucket) {
                case 16: batch_lmm<16, SEQ>(bi, it, gv, r, smem_raw, zs); break;
                case 40: batch_lmm<40, SEQ>(bi, it, gv, r, smem_raw, zs); break;
                default: batch_lmm<80, SEQ>(bi, it, gv, r, smem_raw, zs); break;
            }
        } else {
            batch_mbs<SEQ>(bi, it, gv, r, smem_raw);
        }
    }
    if (threadIdx.x == 0 && stats && blockIdx.x < stats_cap) {
        unsigned long long *rec = stats + 3ull * ((unsigned long long)KIND * stats_cap + blockIdx.x);
        rec[0] = batch_smid();
        rec[1] = t_start;
        rec[2] = batch_clock();
    }
}

template <int SEQ, int KIND>
cudaError_t launch_batch_class(const BatchLaunch &bl, cudaStream_t st) {
    auto kern = batch_kernel<SEQ, KIND>;
    const size_t smem = bl.smem[KIND];
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bl.threads, smem);
    if (occ < 1) occ = 1;
    unsigned grid = (unsigned)std::min<unsigned long long>(bl.n_items[KIND], (unsigned long long)occ * sms);
    if (bl.znorm[KIND]) grid = std::min<unsigned>(grid, bl.zctas[KIND]);   // one normals buffer per CTA
    kern<<<grid, bl.threads, smem, st>>>(bl.insts, bl.items[KIND], bl.n_items[KIND], bl.counter + KIND, bl.partials,
                                         bl.ppt, bl.stats, bl.stats_cap, bl.znorm[KIND], bl.zstride[KIND]);
    return cudaGetLastError();
}

template <int SEQ>
cudaError_t launch_batch_seq(const BatchLaunch &bl, int kind, cudaStream_t st) {
    return kind == 0   ? launch_batch_class<SEQ, 0>(bl, st)
           : kind == 1 ? launch_batch_class<SEQ, 1>(bl, st)
                       : launch_batch_class<SEQ, 2>(bl, st);
}

}  // namespace rqmc
