// Contraction engine dispatch: every contraction of a step is C = A B^T with
// K-contiguous FP64 operands and an FP64 result (dense), or a grouped product
// over charge blocks (block-sparse).  HOTRG_FP64 runs the SIMT DFMA kernels
// (dense: hotrg_kernels.cu, grouped: hotrg_grouped_f64.cu); the tensor-core
// split forms live in hotrg_umma.cu.
#include "internal.cuh"

namespace hotrg {

hotrg_status umma_gemm(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, bool coarse);
size_t umma_workspace(int prec, int64_t M, int64_t N, int64_t K);

hotrg_status gemm_engine(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda, const double* B,
                         int64_t ldb, double* C, int64_t ldc, bool coarse) {
    if (M <= 0 || N <= 0) return HOTRG_OK;
    if (prec == HOTRG_FP64) {
        const int h = prof_begin(ctx);
        launch_gemm_tn_f64(M, N, K, A, lda, B, ldb, C, ldc, 1, 0, 0, 0, ctx->stream);
        prof_end(ctx, h, coarse ? PROF_GEMM_COARSE : PROF_GEMM_ENV, 2.0 * M * N * (double)K);
        HOTRG_LAUNCH_CHECK(ctx, "gemm_tn_f64");
        return HOTRG_OK;
    }
    // slice buffers live only until the (stream-ordered) GEMM has consumed them
    const size_t mark = ctx->ws.used;
    hotrg_status s = umma_gemm(ctx, prec, M, N, K, A, lda, B, ldb, C, ldc, coarse);
    ctx->ws.used = mark;
    return s;
}

hotrg_status grouped_engine(hotrg_ctx* ctx, int prec, const BsPlan& pl, const void* A, int afmt, const void* B,
                            int bfmt, void* C, int cfmt, int prof_class) {
    if (prec == HOTRG_FP64) return dgemm_grouped(ctx, pl, A, afmt, B, bfmt, C, cfmt, prof_class);
    return umma_grouped(ctx, prec, pl, A, afmt, B, bfmt, C, cfmt, prof_class);
}

size_t gemm_engine_workspace(int prec, int64_t M, int64_t N, int64_t K) {
    if (prec == HOTRG_FP64) return 0;
    return umma_workspace(prec, M, N, K);
}

}  // namespace hotrg
