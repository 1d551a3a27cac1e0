// Block-sparse contractions in plain FP64 (the FP64 form with block_sparse = 1).
//
// The same charge-block plan as the tensor-core grouped GEMM (hotrg_blocks.cu:
// groups of the values present in both M and N, 128 x 128 tiles, offset
// tables for every sorted position), contracted with FP64 FMA on the SIMT
// pipes.  This is the per-sector contraction of the block-sparse remark of
// §2.3.1 with no change of arithmetic: every product of a block is an FP64
// dot product over the block's K elements, accumulated in K order.
//
// Each planner tile is split into four 64 x 64 sub-tiles; a persistent grid
// walks the sub-tiles (CTA b takes b, b + gridDim.x, ...).  Per sub-tile the
// 64 row offsets of A and B and, per 16-wide K chunk, the chunk's K offsets
// are staged in shared memory; the operand elements are gathered through them
// (A(m, k) = A[offM0[m] + offK0[k]], B(n, k) = B[offN0[n] + offK1[k]]) and
// each thread accumulates a 4 x 4 block of outputs, written to
// C[offM1[m] + offN1[n]] (+ pi_out[offM2[m] + offN2[n]] for an output in a pair layout).
#include "internal.cuh"

namespace hotrg {

constexpr int DG_T = 64, DG_K = 16, DG_THREADS = 256, DG_CTAS_PER_SM = 8;

__device__ __forceinline__ void dg_decode(const BsGroup* gr, int G, int t, int& g, int& tm, int& tn) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gr[mid].tile_base <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    g = lo;
    const int loc = t - gr[g].tile_base;
    tm = loc / gr[g].tiles_n;
    tn = loc % gr[g].tiles_n;
}

__global__ void __launch_bounds__(DG_THREADS) dgemm_grouped_kernel(const double* __restrict__ A,
                                                                   const double* __restrict__ B,
                                                                   double* __restrict__ C, BsPlan pl) {
    __shared__ double As[DG_K][DG_T + 1];
    __shared__ double Bs[DG_K][DG_T + 1];
    __shared__ int64_t rA[DG_T], rB[DG_T], rC[DG_T], cC[DG_T];
    __shared__ int64_t kA[DG_K], kB[DG_K];
    __shared__ int32_t rP[DG_T], cP[DG_T];
    const int32_t* __restrict__ pi = pl.pi_out;
    const int G = pl.hdr->G;
    const int total = pl.hdr->total_tiles * 4;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        int g, tm, tn;
        dg_decode(pl.groups, G, w >> 2, g, tm, tn);
        const BsGroup gr = pl.groups[g];
        const int m0 = tm * 128 + ((w >> 1) & 1) * DG_T, n0 = tn * 128 + (w & 1) * DG_T;
        if (m0 >= gr.M || n0 >= gr.N) continue;  // the whole CTA leaves this sub-tile together
        __syncthreads();  // the previous sub-tile's readers of the offset arrays are done
        if (tid < DG_T) {
            const int m = m0 + tid;
            rA[tid] = m < gr.M ? pl.offM0[gr.mbase + m] : -1;
            rC[tid] = m < gr.M ? pl.offM1[gr.mbase + m] : -1;
            rP[tid] = (m < gr.M && pi) ? pl.offM2[gr.mbase + m] : 0;
        } else if (tid < 2 * DG_T) {
            const int n = n0 + tid - DG_T;
            rB[tid - DG_T] = n < gr.N ? pl.offN0[gr.nbase + n] : -1;
            cC[tid - DG_T] = n < gr.N ? pl.offN1[gr.nbase + n] : -1;
            cP[tid - DG_T] = (n < gr.N && pi) ? pl.offN2[gr.nbase + n] : 0;
        }
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (int k0 = 0; k0 < gr.K; k0 += DG_K) {
            if (tid < DG_K) {
                const int k = k0 + tid;
                kA[tid] = k < gr.K ? pl.offK0[gr.kbase + k] : -1;
            } else if (tid < 2 * DG_K) {
                const int k = k0 + tid - DG_K;
                kB[tid - DG_K] = k < gr.K ? pl.offK1[gr.kbase + k] : -1;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < (DG_T * DG_K) / DG_THREADS; ++u) {
                const int i = tid + u * DG_THREADS;
                const int r = i / DG_K, kk = i % DG_K;
                const int64_t ra = rA[r], rb = rB[r], ka = kA[kk], kb = kB[kk];
                As[kk][r] = (ra >= 0 && ka >= 0) ? A[ra + ka] : 0.0;
                Bs[kk][r] = (rb >= 0 && kb >= 0) ? B[rb + kb] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < DG_K; ++kk) {
                double av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
        if (gr.K == 0) __syncthreads();  // the row offsets were written without a K chunk's barrier
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t ro = rC[ty + 16 * i];
            if (ro < 0) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t co = cC[tx + 16 * j];
                if (co >= 0) C[ro + co + (pi ? (int64_t)pi[rP[ty + 16 * i] + cP[tx + 16 * j]] : 0)] = acc[i][j];
            }
        }
    }
}

hotrg_status dgemm_grouped(hotrg_ctx* ctx, const BsPlan& pl, const void* A, int afmt, const void* B, int bfmt,
                           void* C, int cfmt, int prof_class) {
    if (afmt != 0 || bfmt != 0 || cfmt != 0)
        return set_err(ctx, HOTRG_EINVAL, "FP64 grouped contraction takes FP64 operands and output");
    const int h = prof_begin(ctx);
    dgemm_grouped_kernel<<<ctx->sm_count * DG_CTAS_PER_SM, DG_THREADS, 0, ctx->stream>>>(
        (const double*)A, (const double*)B, (double*)C, pl);
    prof_end(ctx, h, prof_class, 0.0);  // algorithmic flops are counted on the device by the planner
    HOTRG_COUNT(1);
    HOTRG_LAUNCH_CHECK(ctx, "dgemm_grouped_kernel");
    return HOTRG_OK;
}

}  // namespace hotrg
