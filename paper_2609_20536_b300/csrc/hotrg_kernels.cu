// Elementwise and FP64 SIMT kernels of libhotrg: initial tensors (§3.2-§3.4),
// permutations, the FP64 reference-form GEMM, norms and traces.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace hotrg {

// ---------------------------------------------------------------------------
// Modified Bessel I_n(x), integer n, from the power series
//   I_n(x) = sum_k (x/2)^{2k+|n|} / (k! (k+|n|)!)
// (all terms positive for x >= 0).  The Jacobi-Anger expansion of §3.2 / §3.3
// (Eq. 3.3, 3.9) makes I_n the only special function the tensors need.
// ---------------------------------------------------------------------------
__device__ double bessel_in(int n, double x) {
    n = n < 0 ? -n : n;
    if (x == 0.0) return n == 0 ? 1.0 : 0.0;
    double sign = 1.0;
    if (x < 0.0) {
        x = -x;
        if (n & 1) sign = -1.0;
    }
    const double half = 0.5 * x;
    double term = 1.0;
    for (int k = 1; k <= n; ++k) {
        term *= half / (double)k;
        if (term < 1e-300) return 0.0;  // below any scale that reaches the tensor
    }
    double sum = term;
    const double q = half * half;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (double)(k + n));
        sum += term;
        if (term <= 1e-18 * sum) break;
    }
    return sign * sum;
}

// a_n(beta, Delta) = sum_{m=-M..M} I_{n-qm}(beta Delta) I_m(beta (1 - Delta))   (Eq. 3.4; q = 2 in the thesis)
// F(Q) for the pure tensor (Eq. 3.15) and the impurities (Eq. 3.20, 3.21).
// One block: first every I_k needed (k = 0 .. kmax for the four arguments
// beta Delta, beta (1 - Delta), beta h, beta h1) is tabulated in shared memory,
// one thread per value; then one thread per coefficient sums the table in the
// order of the formulas above.  All arguments are >= 0 and I_{-k} = I_k.
__global__ void coeff_kernel(const hotrg_params* __restrict__ dp, int n_max, int m_range, int kind, int q, int kmax,
                             double* a, double* F) {
    extern __shared__ double tab[];  // [4][kmax + 1]
    const double beta = dp->beta, delta = dp->delta, h = dp->h, h1 = dp->h1;
    const double xs[4] = {beta * delta, beta * (1.0 - delta), beta * h, beta * h1};
    const int w = kmax + 1;
    for (int i = threadIdx.x; i < 4 * w; i += blockDim.x) tab[i] = bessel_in(i % w, xs[i / w]);
    __syncthreads();
    const double* I1 = tab;          // I_k(beta Delta)
    const double* I2 = tab + w;      // I_k(beta (1 - Delta))
    const double* Ih = tab + 2 * w;  // I_k(beta h)
    const double* Ih1 = tab + 3 * w; // I_k(beta h1)
    auto at = [](const double* t, int k) { return t[k < 0 ? -k : k]; };
    const int na = 2 * n_max + 1;
    const int nf = 8 * n_max + 1;
    for (int t = threadIdx.x; t < na + nf; t += blockDim.x) {
        if (t < na) {
            const int n = t - n_max;
            double s = 0.0;
            for (int m = -m_range; m <= m_range; ++m) s += at(I1, n - q * m) * at(I2, m);
            a[t] = s;
        } else {
            const int Q = (t - na) - 4 * n_max;
            double s = 0.0;
            for (int j = -m_range; j <= m_range; ++j) {
                if (kind == HOTRG_T_PURE)
                    s += at(Ih, Q + 2 * j) * at(Ih1, j);
                else if (kind == HOTRG_T_IMP_M)
                    s += at(Ih1, j) * 0.5 * (at(Ih, Q + 2 * j - 1) + at(Ih, Q + 2 * j + 1));
                else
                    s += at(Ih, Q + 2 * j) * 0.5 * (at(Ih1, j + 1) + at(Ih1, j - 1));
            }
            F[t - na] = s;
        }
    }
}

// T[l,r,u,d] = sqrt(a_l a_r a_u a_d) F(n_l + n_u - n_r - n_d)   (Eq. 3.6 / 3.15)
__global__ void gxy_tensor_kernel(const double* a, const double* F, int n_max, int sym, double* T,
                                  int32_t* labels) {
    const int D0 = 2 * n_max + 1;
    const int total = D0 * D0 * D0 * D0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int d = i % D0, u = (i / D0) % D0, r = (i / (D0 * D0)) % D0, l = i / (D0 * D0 * D0);
        const int Q = l + u - r - d;
        const double f = F[Q + 4 * n_max];
        T[i] = (f == 0.0) ? 0.0 : sqrt(a[l] * a[r] * a[u] * a[d]) * f;
        if (i < D0) {
            int q = i - n_max;
            if (sym == SYM_Z2) q = ((q % 2) + 2) % 2;
            if (sym == SYM_NONE) q = 0;
            labels[i] = q;
        }
    }
}

// 2D Ising: T[l,r,u,d] = sum_s W[s,l] W[s,r] W[s,u] W[s,d], W[s,0] = sqrt(cosh b),
// W[s,1] = s sqrt(sinh b); each bond then carries exp(b s s').
__global__ void ising_tensor_kernel(const hotrg_params* __restrict__ dp, double* T, int32_t* labels) {
    const double beta = dp->beta;
    const int i = threadIdx.x;
    if (i < 16) {
        const double w[2][2] = {{sqrt(cosh(beta)), sqrt(sinh(beta))}, {sqrt(cosh(beta)), -sqrt(sinh(beta))}};
        const int d = i & 1, u = (i >> 1) & 1, r = (i >> 2) & 1, l = (i >> 3) & 1;
        double s = 0.0;
        for (int sp = 0; sp < 2; ++sp) s += w[sp][l] * w[sp][r] * w[sp][u] * w[sp][d];
        T[i] = s;
    }
    if (i < 2) labels[i] = i;
}

void launch_init_tensor(const hotrg_params* p, const hotrg_params* dp, int kind, double* T, int32_t* labels,
                        double* scratch, cudaStream_t st) {
    if (kind == HOTRG_T_ISING) {
        ising_tensor_kernel<<<1, 32, 0, st>>>(dp, T, labels);
        HOTRG_COUNT(1);
        return;
    }
    const int n_max = p->n_max;
    const int na = 2 * n_max + 1, nf = 8 * n_max + 1;
    double* a = scratch;
    double* F = scratch + na;
    const int m_range = p->m_range > 0 ? p->m_range : 50;
    int sym = SYM_U1;
    if (p->h != 0.0) sym = SYM_NONE;
    else if (p->h1 != 0.0) sym = SYM_Z2;
    // largest |order|: n_max + q m_range for a_n, 4 n_max + 2 m_range + 1 for F (q <= 4: <= 865 doubles
    // a row, 27.7 KB for the four tables)
    const int q = p->gxy_q == 0 ? 2 : p->gxy_q;
    const int kmax = std::max(n_max + q * m_range, 4 * n_max + 2 * m_range + 1) + 1;
    coeff_kernel<<<1, 256, 4 * (kmax + 1) * sizeof(double), st>>>(dp, n_max, m_range, kind, q, kmax, a, F);
    const int total = na * na * na * na;
    gxy_tensor_kernel<<<(total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024, 256, 0, st>>>(
        a, F, n_max, sym, T, labels);
    HOTRG_COUNT(2);
}

// ---------------------------------------------------------------------------
// Output-ordered permutation (up to 6 dims).
// ---------------------------------------------------------------------------
struct PermArgs {
    int nd;
    int64_t od[6];
    int64_t is[6];
    int64_t total;
};

__global__ void permute_kernel(const double* __restrict__ in, double* __restrict__ out, PermArgs a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i, off = 0;
        for (int k = a.nd - 1; k >= 0; --k) {
            const int64_t o = rem % a.od[k];
            rem /= a.od[k];
            off += o * a.is[k];
        }
        out[i] = in[off];
    }
}

void launch_permute(const double* in, double* out, int nd, const int64_t* od, const int64_t* is,
                    cudaStream_t st) {
    PermArgs a;
    a.nd = nd;
    a.total = 1;
    for (int k = 0; k < 6; ++k) {
        a.od[k] = k < nd ? od[k] : 1;
        a.is[k] = k < nd ? is[k] : 0;
        if (k < nd) a.total *= od[k];
    }
    if (a.total == 0) return;
    int64_t blocks = (a.total + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    permute_kernel<<<(int)blocks, 256, 0, st>>>(in, out, a);
    HOTRG_COUNT(1);
}

// ---------------------------------------------------------------------------
// FP64 SIMT GEMM, C = A * B^T, both operands K-contiguous.  64x64 tiles,
// 256 threads with 4x4 outputs each.  This is the plain FP64 form's engine.
// ---------------------------------------------------------------------------
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

__global__ void __launch_bounds__(256) gemm_tn_f64_kernel(int M, int N, int K, const double* __restrict__ A,
                                                          int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                          double* __restrict__ C, int64_t ldc, int64_t sA,
                                                          int64_t sB, int64_t sC) {
    __shared__ double As[GB_K][GB_M + 1];
    __shared__ double Bs[GB_K][GB_N + 1];
    const int64_t bz = blockIdx.z;
    A += bz * sA;
    B += bz * sB;
    C += bz * sC;
    const int64_t m0 = (int64_t)blockIdx.y * GB_M, n0 = (int64_t)blockIdx.x * GB_N;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += GB_K) {
        for (int i = tid; i < GB_M * GB_K; i += 256) {
            const int r = i / GB_K, kk = i % GB_K;
            const int64_t gm = m0 + r;
            const int gk = k0 + kk;
            As[kk][r] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.0;
            const int64_t gn = n0 + r;
            Bs[kk][r] = (gn < N && gk < K) ? B[gn * ldb + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
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
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gn = n0 + tx + 16 * j;
            if (gn < N) C[gm * ldc + gn] = acc[i][j];
        }
    }
}

void launch_gemm_tn_f64(int M, int N, int K, const double* A, int64_t lda, const double* B, int64_t ldb,
                        double* C, int64_t ldc, int batch, int64_t sA, int64_t sB, int64_t sC,
                        cudaStream_t st) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, batch);
    gemm_tn_f64_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, sA, sB, sC);
    HOTRG_COUNT(1);
}

// ---------------------------------------------------------------------------
// Deterministic reductions.
// ---------------------------------------------------------------------------
constexpr int NORM_BLOCKS = 592;

int norm_partials() { return NORM_BLOCKS; }

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void sumsq_partial_kernel(const double* __restrict__ x, int64_t n, double* partial) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(x[i], x[i], s);
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void sumsq_final_kernel(const double* partial, int np, double* norm) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) *norm = sqrt(t);
}

void launch_norm(const double* x, int64_t n, double* partial, double* norm, cudaStream_t st) {
    sumsq_partial_kernel<<<NORM_BLOCKS, 256, 0, st>>>(x, n, partial);
    sumsq_final_kernel<<<1, 256, 0, st>>>(partial, NORM_BLOCKS, norm);
    HOTRG_COUNT(2);
}

// x <- x / c as x (1 / c): one FP64 multiply per element instead of a division
// (B300's FP64 division made this pass 10x slower than its memory traffic).
// The divisor differs from c by at most an ulp; ln c_k is recorded from c and
// the next norm absorbs the difference.
__global__ void scale_inv_kernel(double* x, int64_t n, const double* c) {
    const double inv = 1.0 / *c;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= inv;
}

void launch_scale_inv(double* x, int64_t n, const double* c, cudaStream_t st) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (blocks < 1) blocks = 1;
    scale_inv_kernel<<<(int)blocks, 256, 0, st>>>(x, n, c);
    HOTRG_COUNT(1);
}

__global__ void axpby_kernel(double* y, const double* x, double a, double b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

void launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (blocks < 1) blocks = 1;
    axpby_kernel<<<(int)blocks, 256, 0, st>>>(y, x, a, b, n);
    HOTRG_COUNT(1);
}

__global__ void trace_kernel(const double* T, int Dx, int Dy, double* tr) {
    __shared__ double sh[32];
    double s = 0.0;
    const int64_t sx = (int64_t)Dx * Dy * Dy, sy = Dy;
    for (int i = threadIdx.x; i < Dx * Dy; i += blockDim.x) {
        const int x = i / Dy, y = i % Dy;
        s += T[x * sx + x * (int64_t)Dy * Dy + y * sy + y];
    }
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) *tr = t;
}

void launch_trace(const double* T, int Dx, int Dy, double* tr, cudaStream_t st) {
    trace_kernel<<<1, 256, 0, st>>>(T, Dx, Dy, tr);
    HOTRG_COUNT(1);
}

__global__ void step_scalars_kernel(const double* norm, hotrg_step_info* info, double* lnz_acc,
                                    double weight) {
    if (threadIdx.x == 0) {
        const double lc = log(*norm);
        if (info) info->ln_c = lc;
        if (lnz_acc) *lnz_acc += weight * lc;
    }
}

void launch_step_scalars(const double* norm, hotrg_step_info* info, double* lnz_acc, double weight,
                         cudaStream_t st) {
    step_scalars_kernel<<<1, 32, 0, st>>>(norm, info, lnz_acc, weight);
    HOTRG_COUNT(1);
}

}  // namespace hotrg
