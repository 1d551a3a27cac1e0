// Tensor-core split-precision contraction engine (sm_103a).  Placeholder
// until the tcgen05 kernels land: the split forms report HOTRG_ENOTSUP.
#include "internal.cuh"

namespace hotrg {

hotrg_status umma_gemm(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, bool coarse) {
    (void)prec; (void)M; (void)N; (void)K; (void)A; (void)lda; (void)B; (void)ldb; (void)C; (void)ldc; (void)coarse;
    return set_err(ctx, HOTRG_ENOTSUP, "split-precision engine not built");
}

size_t umma_workspace(int prec, int64_t M, int64_t N, int64_t K) {
    (void)prec; (void)M; (void)N; (void)K;
    return 0;
}

}  // namespace hotrg
