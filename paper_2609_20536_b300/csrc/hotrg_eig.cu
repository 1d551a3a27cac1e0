// Truncation of one HOTRG step on the device (§2.4.1): per-sector FP64 Jacobi
// eigensolve of the environments E_L / E_R, the cut-cluster selection of the
// top D' eigenpairs, the eps_1 / eps_2 side rule and the projector P.
//
// Block structure (§2.3.1: conserved quantum numbers make the decomposition
// block-sparse): the fused state (a, b) of two horizontal legs carries the key
// q_h[a] + q_h[b] (U(1) charge), its parity (Z2), or 0 (no symmetry); E is
// block diagonal in the key and each block is diagonalised on its own.
//
// Selection rule (the thesis leaves ties unstated): sort all eigenvalues
// descending; those within tie_rtol * lambda_max of the D'-th largest form the
// cut cluster, filled in order of |key| ascending, key descending, lambda
// descending, slot ascending.  eps = sum of the discarded eigenvalues.  The
// right environment's projector is used only when eps_R < eps_L (1 - 1e-12).
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace hotrg {

constexpr int MAX_N = 16384;        // Dh <= 128
constexpr int SORT_THREADS = 1024;
constexpr int JAC_THREADS = 512;
constexpr int JAC_SMEM_M = 96;      // sectors up to this size run from shared memory
constexpr int JAC_MAX_PAIRS = MAX_N / 2;
// rotation parameters: 2 doubles + 2 ints per pair
constexpr size_t JAC_PAIR_BYTES = 24;
constexpr size_t JAC_SMEM_MAT = 2 * JAC_SMEM_M * JAC_SMEM_M * sizeof(double);
constexpr size_t JAC_SMEM_BYTES =
    (JAC_SMEM_MAT + (JAC_SMEM_M / 2) * JAC_PAIR_BYTES) > (JAC_MAX_PAIRS * JAC_PAIR_BYTES)
        ? (JAC_SMEM_MAT + (JAC_SMEM_M / 2) * JAC_PAIR_BYTES)
        : (JAC_MAX_PAIRS * JAC_PAIR_BYTES);

struct EigWs {
    // sector structure (shared by both sides)
    int32_t* members;   // [n] state indices grouped by key
    int32_t* sec_start; // [n + 1]
    int32_t* sec_key;   // [n]
    int64_t* sec_off;   // [n] offset of the sector's m x m block
    int32_t* nsec;      // [1]
    int32_t* slot_sec;  // [n] sector of each slot (slot = position in members)
    // per side
    double* A[2];       // packed m x m blocks (working copy of E_q, then eigenvalues on the diagonal)
    double* V[2];       // packed eigenvector blocks, V[i][j]: component i of eigenvector j
    double* lam[2];     // [n] eigenvalue of each slot
    int32_t* kept[2];   // [D'] kept slots in kept order
    double* eps[2];     // [1]
    int32_t* sweeps;    // [2]
    int32_t* status;    // [1]
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t eig_workspace_bytes(int Dh) {
    const size_t n = (size_t)Dh * Dh;
    size_t b = 0;
    b += align256(n * 4) * 4 + align256((n + 1) * 4) + align256(n * 8) + align256(64);
    for (int s = 0; s < 2; ++s) b += align256(n * n * 8) * 2 + align256(n * 8) + align256(n * 4) + align256(64);
    b += align256(64) * 2;
    return b;
}

static EigWs carve(void* base, int n) {
    char* p = (char*)base;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += align256(bytes);
        return (void*)r;
    };
    EigWs w;
    w.members = (int32_t*)take((size_t)n * 4);
    w.sec_start = (int32_t*)take((size_t)(n + 1) * 4);
    w.sec_key = (int32_t*)take((size_t)n * 4);
    w.sec_off = (int64_t*)take((size_t)n * 8);
    w.nsec = (int32_t*)take(64);
    w.slot_sec = (int32_t*)take((size_t)n * 4);
    for (int s = 0; s < 2; ++s) {
        w.A[s] = (double*)take((size_t)n * n * 8);
        w.V[s] = (double*)take((size_t)n * n * 8);
        w.lam[s] = (double*)take((size_t)n * 8);
        w.kept[s] = (int32_t*)take((size_t)n * 4);
        w.eps[s] = (double*)take(64);
    }
    w.sweeps = (int32_t*)take(64);
    w.status = (int32_t*)take(64);
    return w;
}

// ---------------------------------------------------------------------------
// Sector discovery: sort (key, state) pairs, then segment by key.
// ---------------------------------------------------------------------------
__device__ void bitonic_sort_u64(uint64_t* a, int npow2) {
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const uint64_t x = a[i], y = a[ixj];
                    if ((x > y) == up) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(SORT_THREADS) sectors_kernel(const int32_t* q_h, int Dh, int sym, EigWs w) {
    extern __shared__ uint64_t su[];
    const int n = Dh * Dh;
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
        if (i < n) {
            int key = q_h[i / Dh] + q_h[i % Dh];
            if (sym == SYM_Z2) key = ((key % 2) + 2) % 2;
            if (sym == SYM_NONE) key = 0;
            su[i] = ((uint64_t)(uint32_t)(key + (1 << 30)) << 32) | (uint32_t)i;
        } else {
            su[i] = ~0ull;
        }
    }
    __syncthreads();
    bitonic_sort_u64(su, npow2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) w.members[i] = (int32_t)(su[i] & 0xffffffffu);
    __syncthreads();
    if (threadIdx.x == 0) {
        int ns = 0;
        int64_t off = 0;
        int prev_key = 0;
        for (int i = 0; i < n; ++i) {
            const int key = (int)(su[i] >> 32) - (1 << 30);
            if (i == 0 || key != prev_key) {
                if (ns > 0) {
                    const int m = i - w.sec_start[ns - 1];
                    off += (int64_t)m * m;
                }
                w.sec_start[ns] = i;
                w.sec_key[ns] = key;
                w.sec_off[ns] = off;
                ++ns;
                prev_key = key;
            }
            w.slot_sec[i] = ns - 1;
        }
        w.sec_start[ns] = n;
        *w.nsec = ns;
        w.sweeps[0] = 0;
        w.sweeps[1] = 0;
        *w.status = HOTRG_OK;
    }
}

// ---------------------------------------------------------------------------
// Cyclic parallel Jacobi (round-robin pairing) on one symmetric block.
// A (m x m, row-major, ld m) is overwritten; V receives the eigenvectors.
// ---------------------------------------------------------------------------
__device__ double block_reduce_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// Stopping rule: a rotation is skipped when |a_pq| <= tol * ||A||_F / m
// (negligible normwise; ||A||_F is invariant under the rotations) or when
// |a_pq| <= 2^-53 sqrt(|a_pp a_qq|) (negligible against its 2x2 block).  The
// block has converged after a sweep that performs no rotation.  Returns the
// number of sweeps that rotated, or -1 when max_sweeps ran out.
__device__ int jacobi_block(double* A, double* V, int m, int max_sweeps, double tol, double* rc, double* rs,
                            int* rp, int* rq, double* red, int* s_rot) {
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) V[i] = (i / m == i % m) ? 1.0 : 0.0;
    __syncthreads();
    if (m == 1) return 0;
    double tot = 0.0;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) tot += A[i] * A[i];
    tot = block_reduce_sum(tot, red);
    const double thr = tol * sqrt(tot) / (double)m;
    const int mm = m + (m & 1);
    const int npairs = mm / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) *s_rot = 0;
        __syncthreads();
        for (int r = 0; r < mm - 1; ++r) {
            for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
                int p, q;
                if (k == 0) {
                    p = mm - 1;
                    q = r;
                } else {
                    p = (r + k) % (mm - 1);
                    q = (r - k + mm - 1) % (mm - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                double c = 1.0, s = 0.0;
                if (q < m) {
                    const double apq = A[p * m + q];
                    const double app = A[p * m + p], aqq = A[q * m + q];
                    if (fabs(apq) > thr && fabs(apq) > 1.1102230246251565e-16 * sqrt(fabs(app * aqq))) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        double t;
                        if (fabs(theta) > 1e150)
                            t = 0.5 / theta;
                        else
                            t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                        *s_rot = 1;
                    }
                } else {
                    q = -1;  // pair with the padding index: no rotation
                }
                rc[k] = c;
                rs[k] = s;
                rp[k] = p;
                rq[k] = q;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int idx = threadIdx.x; idx < npairs * m; idx += blockDim.x) {
                const int k = idx / m, j = idx % m;
                const int q = rq[k];
                if (q < 0 || rs[k] == 0.0) continue;
                const int p = rp[k];
                const double c = rc[k], s = rs[k];
                const double ap = A[p * m + j], aq = A[q * m + j];
                A[p * m + j] = c * ap - s * aq;
                A[q * m + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int idx = threadIdx.x; idx < npairs * m; idx += blockDim.x) {
                const int k = idx / m, i = idx % m;
                const int q = rq[k];
                if (q < 0 || rs[k] == 0.0) continue;
                const int p = rp[k];
                const double c = rc[k], s = rs[k];
                const double ap = A[i * m + p], aq = A[i * m + q];
                A[i * m + p] = c * ap - s * aq;
                A[i * m + q] = s * ap + c * aq;
                const double vp = V[i * m + p], vq = V[i * m + q];
                V[i * m + p] = c * vp - s * vq;
                V[i * m + q] = s * vp + c * vq;
            }
            __syncthreads();
            for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
                const int q = rq[k];
                if (q < 0 || rs[k] == 0.0) continue;
                const int p = rp[k];
                A[p * m + q] = 0.0;
                A[q * m + p] = 0.0;
            }
            __syncthreads();
        }
        const int rotated = *s_rot;
        __syncthreads();
        if (!rotated) return sweep;
    }
    return -1;
}

__global__ void __launch_bounds__(JAC_THREADS) jacobi_sectors_kernel(const double* EL, const double* ER, int n,
                                                                     int max_sweeps, double tol, EigWs w) {
    extern __shared__ double sm[];
    __shared__ double red[40];
    __shared__ int s_rot;
    const int side = blockIdx.y;
    const double* E = side == 0 ? EL : ER;
    const int nsec = *w.nsec;
    for (int sct = blockIdx.x; sct < nsec; sct += gridDim.x) {
        const int start = w.sec_start[sct];
        const int m = w.sec_start[sct + 1] - start;
        double* Ag = w.A[side] + w.sec_off[sct];
        double* Vg = w.V[side] + w.sec_off[sct];
        const bool in_smem = m <= JAC_SMEM_M;
        double* A = in_smem ? sm : Ag;
        double* V = in_smem ? sm + JAC_SMEM_M * JAC_SMEM_M : Vg;
        const int cap = in_smem ? JAC_SMEM_M / 2 : JAC_MAX_PAIRS;
        double* rc = in_smem ? sm + 2 * JAC_SMEM_M * JAC_SMEM_M : sm;
        double* rs = rc + cap;
        int* rp = (int*)(rs + cap);
        int* rq = rp + cap;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = idx / m, j = idx % m;
            A[idx] = E[(int64_t)w.members[start + i] * n + w.members[start + j]];
        }
        __syncthreads();
        const int sw = jacobi_block(A, V, m, max_sweeps, tol, rc, rs, rp, rq, red, &s_rot);
        for (int i = threadIdx.x; i < m; i += blockDim.x) w.lam[side][start + i] = A[i * m + i];
        if (in_smem)
            for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) Vg[idx] = V[idx];
        if (threadIdx.x == 0) {
            if (sw < 0)
                atomicExch(w.status, (int)HOTRG_ENOCONV);
            else
                atomicMax(&w.sweeps[side], sw);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Selection of the kept slots (one block per side).
// ---------------------------------------------------------------------------
struct SelCmp {
    const double* lam;
    const int32_t* key;  // key per slot (via sector)
    int mode;            // 0: lambda desc, slot asc; 1: |key| asc, key desc, lambda desc, slot asc
    __device__ bool less(int a, int b) const {  // "a sorts before b"
        if (mode == 0) {
            if (lam[a] != lam[b]) return lam[a] > lam[b];
            return a < b;
        }
        const int ka = key[a], kb = key[b];
        const int aa = ka < 0 ? -ka : ka, ab = kb < 0 ? -kb : kb;
        if (aa != ab) return aa < ab;
        if (ka != kb) return ka > kb;
        if (lam[a] != lam[b]) return lam[a] > lam[b];
        return a < b;
    }
};

__device__ void bitonic_sort_idx(int* a, int npow2, const SelCmp& cmp) {
    // entries < 0 are padding and sort last
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const int x = a[i], y = a[ixj];
                    bool x_after_y;
                    if (x < 0) x_after_y = y >= 0;
                    else if (y < 0) x_after_y = false;
                    else x_after_y = cmp.less(y, x);
                    if (x_after_y == up) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(SORT_THREADS) select_kernel(int n, int dprime, double tie_rtol, EigWs w) {
    extern __shared__ int si[];
    __shared__ double red[40];
    __shared__ int s_bounds[2];
    const int side = blockIdx.x;
    const double* lam = w.lam[side];
    int* slotkey = si + MAX_N;  // key per slot
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) si[i] = i < n ? i : -1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) slotkey[i] = w.sec_key[w.slot_sec[i]];
    __syncthreads();
    SelCmp cmp{lam, slotkey, 0};
    bitonic_sort_idx(si, npow2, cmp);
    int* kept = w.kept[side];
    if (n <= dprime) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) kept[i] = si[i];
        if (threadIdx.x == 0) *w.eps[side] = 0.0;
        return;
    }
    const double lmax = lam[si[0]];
    const double tol = tie_rtol * fabs(lmax);
    const double lcut = lam[si[dprime - 1]];
    if (threadIdx.x == 0) {
        int a = 0;
        while (a < n && lam[si[a]] > lcut + tol) ++a;
        int b = a;
        while (b < n && lam[si[b]] >= lcut - tol) ++b;
        s_bounds[0] = a;
        s_bounds[1] = b;
    }
    __syncthreads();
    const int n_above = s_bounds[0], n_end = s_bounds[1];
    const int need = dprime - n_above;
    const int ncl = n_end - n_above;
    // sort the cluster by the tie rule in a separate power-of-two window
    int* cl = slotkey + MAX_N;  // MAX_N ints
    int cpow2 = 1;
    while (cpow2 < ncl) cpow2 <<= 1;
    for (int i = threadIdx.x; i < cpow2; i += blockDim.x) cl[i] = i < ncl ? si[n_above + i] : -1;
    __syncthreads();
    SelCmp cmp1{lam, slotkey, 1};
    bitonic_sort_idx(cl, cpow2, cmp1);
    // kept = sorted[0, n_above) + cluster[0, need)
    for (int i = threadIdx.x; i < dprime; i += blockDim.x) kept[i] = i < n_above ? si[i] : cl[i - n_above];
    // discarded: cluster[need, ncl) and sorted[n_end, n); Kahan sums per thread
    double s = 0.0, comp = 0.0;
    for (int i = threadIdx.x; i < ncl - need; i += blockDim.x) {
        const double y = lam[cl[need + i]] - comp;
        const double t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    for (int i = n_end + threadIdx.x; i < n; i += blockDim.x) {
        const double y = lam[si[i]] - comp;
        const double t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    const double tot = block_reduce_sum(s, red);
    if (threadIdx.x == 0) *w.eps[side] = tot;
}

// ---------------------------------------------------------------------------
// Side choice and projector P[(a,b)][j] (P must be zeroed beforehand).
// ---------------------------------------------------------------------------
__global__ void projector_kernel(int n, int dprime, int policy, EigWs w, double* P, int32_t* q_out,
                                 hotrg_step_info* info) {
    const double eL = *w.eps[0];
    const double eR = policy == 0 ? *w.eps[1] : nan("");
    const int side = (policy == 0 && eR < eL * (1.0 - 1e-12)) ? 1 : 0;
    const int j = blockIdx.x;
    const int slot = w.kept[side][j];
    const int sct = w.slot_sec[slot];
    const int start = w.sec_start[sct];
    const int m = w.sec_start[sct + 1] - start;
    const int pos = slot - start;
    const double* V = w.V[side] + w.sec_off[sct];
    for (int i = threadIdx.x; i < m; i += blockDim.x) P[(int64_t)w.members[start + i] * dprime + j] = V[i * m + pos];
    if (threadIdx.x == 0) q_out[j] = w.sec_key[sct];
    if (j == 0 && threadIdx.x == 0 && info) {
        info->eps_left = eL;
        info->eps_right = eR;
        info->side = side;
        info->dprime = dprime;
        info->sweeps = max(w.sweeps[0], policy == 0 ? w.sweeps[1] : 0);
        info->status = *w.status;
    }
}

static bool g_attr_done = false;

hotrg_status eig_truncate(hotrg_ctx* ctx, const EigPlan& plan, const double* EL, const double* ER,
                          const int32_t* q_h, double* P, int32_t* q_out, hotrg_step_info* info, void* ws) {
    const int n = plan.n;
    if (n > MAX_N) return set_err(ctx, HOTRG_EINVAL, "eig_truncate: Dh^2 above 16384");
    cudaStream_t st = ctx->stream;
    if (!g_attr_done) {
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(sectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 MAX_N * 8));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(jacobi_sectors_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JAC_SMEM_BYTES));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 MAX_N * 4 * 3));
        g_attr_done = true;
    }
    EigWs w = carve(ws, n);
    sectors_kernel<<<1, SORT_THREADS, MAX_N * 8, st>>>(q_h, plan.Dh, plan.sym, w);
    HOTRG_LAUNCH_CHECK(ctx, "sectors_kernel");
    const int sides = plan.env_policy == 0 ? 2 : 1;
    int grid = n < 2 * ctx->sm_count ? n : 2 * ctx->sm_count;
    jacobi_sectors_kernel<<<dim3(grid, sides), JAC_THREADS, JAC_SMEM_BYTES, st>>>(EL, ER, n, plan.max_sweeps,
                                                                                  plan.tol, w);
    HOTRG_LAUNCH_CHECK(ctx, "jacobi_sectors_kernel");
    select_kernel<<<sides, SORT_THREADS, MAX_N * 4 * 3, st>>>(n, plan.dprime, plan.tie_rtol, w);
    HOTRG_LAUNCH_CHECK(ctx, "select_kernel");
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(P, 0, (size_t)n * plan.dprime * sizeof(double), st));
    projector_kernel<<<plan.dprime, 128, 0, st>>>(n, plan.dprime, plan.env_policy, w, P, q_out, info);
    HOTRG_LAUNCH_CHECK(ctx, "projector_kernel");
    return HOTRG_OK;
}

}  // namespace hotrg
