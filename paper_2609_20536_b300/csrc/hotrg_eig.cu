// Truncation of one HOTRG step on the device (§2.4.1): eigenpairs of the
// environments E_L / E_R per symmetry sector, the cut-cluster selection of the
// top D' eigenpairs, the eps_1 / eps_2 side rule and the projector P.
//
// Block structure (§2.3.1: conserved quantum numbers make the decomposition
// block-sparse): the fused state (a, b) of two horizontal legs carries the key
// q_h[a] + q_h[b] (U(1) charge), its parity (Z2), or 0 (no symmetry); E is
// block diagonal in the key and each block is solved on its own.
//
// Two eigensolvers:
//  * exact: cyclic parallel Jacobi in FP64 on the whole block (all m
//    eigenpairs).  Used for every block of the FP64 form and for blocks of at
//    most small_thr states in the split forms.
//  * subspace: for larger blocks of the split forms, b <= m columns of FP32
//    block subspace iteration (CGS2 orthonormalisation) followed by one FP64
//    Rayleigh-Ritz step (FP64 CGS2, Y = E_q Q on many CTAs, Jacobi on the
//    b x b projection).  Eigenvalues come out FP64-accurate; the weight of
//    the b..m-1 eigenvalues that are not listed is Tr(E_q) - sum of the
//    listed ones.  If a block's smallest listed eigenvalue reaches the cut,
//    b was too small and the step reports HOTRG_ENOCONV.
//
// Selection rule (the thesis leaves ties unstated): sort all listed
// eigenvalues descending; those within tie_rtol * lambda_max of the D'-th
// largest form the cut cluster, filled in order of |key| ascending, key
// descending, lambda descending, slot ascending.  eps = weight of everything
// not kept.  The right environment's projector is used only when
// eps_R < eps_L (1 - side_rtol), side_rtol = 1e-6 by default.
#include <math.h>

#include <algorithm>
#include <stdint.h>
#include <stdlib.h>

#include "internal.cuh"

namespace hotrg {

constexpr int MAX_N = 16384;  // Dh <= 128
constexpr int SORT_THREADS = 1024;
constexpr int JAC_THREADS = 512;
constexpr int JAC_SMEM_M = 96;  // blocks up to this size run from shared memory
constexpr int JAC_MAX_PAIRS = MAX_N / 2;
constexpr size_t JAC_PAIR_BYTES = 24;  // rotation parameters: 2 doubles + 2 ints per pair
constexpr size_t JAC_SMEM_MAT = 2 * JAC_SMEM_M * JAC_SMEM_M * sizeof(double);
constexpr size_t JAC_SMEM_BYTES =
    (JAC_SMEM_MAT + (JAC_SMEM_M / 2) * JAC_PAIR_BYTES) > (JAC_MAX_PAIRS * JAC_PAIR_BYTES)
        ? (JAC_SMEM_MAT + (JAC_SMEM_M / 2) * JAC_PAIR_BYTES)
        : (JAC_MAX_PAIRS * JAC_PAIR_BYTES);
constexpr int BCAP_MAX = 112;  // largest subspace width (Rayleigh-Ritz block in shared memory)
constexpr int SUB_THREADS = 512;
constexpr int SUB_ITERS = 12;
constexpr int SUB_ITERS_U1 = 6;
// Rayleigh-Ritz finish: H and W (b x b each), the rotation parameters, and a staging area for
// row chunks of Q and Y (24 KB: 14 rows at b = 112, 64 at b = 24)
constexpr size_t RR_STAGE_BYTES = 24 * 1024;
constexpr size_t RR_SMEM_BYTES =
    2 * BCAP_MAX * BCAP_MAX * sizeof(double) + (BCAP_MAX / 2) * JAC_PAIR_BYTES + RR_STAGE_BYTES + 1024;
constexpr size_t PREP_SMEM_BYTES = BCAP_MAX * BCAP_MAX * sizeof(double) + RR_STAGE_BYTES;      // G, staging
constexpr size_t NEXT_SMEM_BYTES = 2 * BCAP_MAX * BCAP_MAX * sizeof(double) + RR_STAGE_BYTES;  // G, W, staging
constexpr int GB_ROWS = 32;  // rows of E_q per CTA in the FP64 product

struct EigWs {
    // block structure (shared by both sides)
    int32_t* members;    // [n] state indices grouped by key (ascending within a key)
    int32_t* sec_start;  // [n + 1] start of each block in members
    int32_t* sec_key;    // [n]
    int64_t* sec_aoff;   // [n] offset of the block's m x m region
    int32_t* sec_b;      // [n] listed eigenpairs of the block
    int32_t* sec_cstart; // [n + 1] first candidate slot of the block
    int32_t* nsec;       // [1]
    int32_t* ncand;      // [1]
    int32_t* cand_sec;   // [n] block of each candidate slot
    // per side
    double* A[2];   // m x m regions: FP64 Jacobi work, or the FP32 copy of E_q
    double* V[2];   // eigenvectors of a Jacobi block (b = m), m x m, at sec_aoff
    double* S1[2];  // FP32 Q of the subspace iteration, then W (b x b: Ritz vectors Q W)
    double* S2[2];  // FP32 Y, then FP64 Q
    double* S3[2];  // FP64 E_q (packed)
    double* S4[2];  // FP64 Y = E_q Q
    double* lam[2];   // [n] eigenvalue of each candidate slot
    double* rest[2];  // [n] unlisted weight of each block
    int32_t* kept[2]; // [D'] kept slots
    double* eps[2];   // [1]
    int32_t* sweeps;  // [2]
    int32_t* status;  // [1]
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t eig_workspace_bytes(int Dh) {
    const size_t n = (size_t)Dh * Dh;
    size_t b = 0;
    b += align256(n * 4) * 5 + align256((n + 1) * 4) * 2 + align256(n * 8) + align256(64) * 2;
    for (int s = 0; s < 2; ++s) b += align256(n * n * 8) * 6 + align256(n * 8) * 2 + align256(n * 4) + align256(64);
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
    w.sec_aoff = (int64_t*)take((size_t)n * 8);
    w.sec_b = (int32_t*)take((size_t)n * 4);
    w.sec_cstart = (int32_t*)take((size_t)(n + 1) * 4);
    w.nsec = (int32_t*)take(64);
    w.ncand = (int32_t*)take(64);
    w.cand_sec = (int32_t*)take((size_t)n * 4);
    for (int s = 0; s < 2; ++s) {
        w.A[s] = (double*)take((size_t)n * n * 8);
        w.V[s] = (double*)take((size_t)n * n * 8);
        w.S1[s] = (double*)take((size_t)n * n * 8);
        w.S2[s] = (double*)take((size_t)n * n * 8);
        w.S3[s] = (double*)take((size_t)n * n * 8);
        w.S4[s] = (double*)take((size_t)n * n * 8);
        w.lam[s] = (double*)take((size_t)n * 8);
        w.rest[s] = (double*)take((size_t)n * 8);
        w.kept[s] = (int32_t*)take((size_t)n * 4);
        w.eps[s] = (double*)take(64);
    }
    w.sweeps = (int32_t*)take(64);
    w.status = (int32_t*)take(64);
    return w;
}

// ---------------------------------------------------------------------------
// Block discovery: sort (key, state) pairs, then segment by key.
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

__global__ void __launch_bounds__(SORT_THREADS) sectors_kernel(const int32_t* q_h, int Dh, int sym, int small_thr,
                                                                int bcap, EigWs w) {
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
    // block heads (a key differing from its predecessor's): each warp takes one contiguous range
    // of the sorted list, counts its heads by ballots, and writes them at its offset (an exclusive
    // scan over the warps' counts), so sec_start lists the heads in order
    __shared__ int wcount[SORT_THREADS / 32], woff[SORT_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = ((n + nw - 1) / nw + 31) / 32 * 32;
    const int lo = warp * per, hi = min(n, lo + per);
    auto key_of = [&](int i) { return (int)(su[i] >> 32) - (1 << 30); };
    int cnt = 0;
    for (int b0 = lo; b0 < hi; b0 += 32) {
        const int i = b0 + lane;
        const bool head = i < hi && (i == 0 || key_of(i) != key_of(i - 1));
        cnt += __popc(__ballot_sync(0xffffffffu, head));
    }
    if (lane == 0) wcount[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int v = 0; v < nw; ++v) {
            woff[v] = run;
            run += wcount[v];
        }
        *w.nsec = run;
    }
    __syncthreads();
    int pos = woff[warp];
    for (int b0 = lo; b0 < hi; b0 += 32) {
        const int i = b0 + lane;
        const bool head = i < hi && (i == 0 || key_of(i) != key_of(i - 1));
        const unsigned m = __ballot_sync(0xffffffffu, head);
        if (head) {
            const int slot = pos + __popc(m & ((1u << lane) - 1u));
            w.sec_start[slot] = i;
            w.sec_key[slot] = key_of(i);
        }
        pos += __popc(m);
    }
    __syncthreads();
    const int ns = *w.nsec;
    // per-block sizes and offsets (a few dozen blocks: one thread)
    if (threadIdx.x == 0) {
        w.sec_start[ns] = n;
        int64_t off = 0;
        int cs = 0;
        for (int s = 0; s < ns; ++s) {
            const int m = w.sec_start[s + 1] - w.sec_start[s];
            const int b = m <= small_thr ? m : min(m, bcap);
            w.sec_aoff[s] = off;
            w.sec_b[s] = b;
            w.sec_cstart[s] = cs;
            off += (int64_t)m * m;
            cs += b;
        }
        w.sec_cstart[ns] = cs;
        *w.ncand = cs;
        w.sweeps[0] = 0;
        w.sweeps[1] = 0;
        *w.status = HOTRG_OK;
    }
    __syncthreads();
    // candidate slot -> block, a warp per block
    for (int s = warp; s < ns; s += nw)
        for (int j = w.sec_cstart[s] + lane; j < w.sec_cstart[s + 1]; j += 32) w.cand_sec[j] = s;
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
        if (w.sec_b[sct] != m) continue;  // solved by the subspace path
        double* Ag = w.A[side] + w.sec_aoff[sct];
        double* Vg = w.V[side] + w.sec_aoff[sct];
        const bool in_smem = m <= JAC_SMEM_M;
        double* A = in_smem ? sm : Ag;
        double* V = in_smem ? sm + JAC_SMEM_M * JAC_SMEM_M : Vg;
        const int cap = in_smem ? JAC_SMEM_M / 2 : JAC_MAX_PAIRS;
        double* rc = in_smem ? sm + 2 * JAC_SMEM_M * JAC_SMEM_M : sm;
        double* rs = rc + cap;
        int* rp = (int*)(rs + cap);
        int* rq = rp + cap;
        for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5) {
            const double* erow = E + (int64_t)w.members[start + i] * n;
            for (int j = threadIdx.x & 31; j < m; j += 32) A[i * m + j] = erow[w.members[start + j]];
        }
        __syncthreads();
        const int sw = jacobi_block(A, V, m, max_sweeps, tol, rc, rs, rp, rq, red, &s_rot);
        const int cs = w.sec_cstart[sct];
        for (int i = threadIdx.x; i < m; i += blockDim.x) w.lam[side][cs + i] = A[i * m + i];
        if (in_smem)
            for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) Vg[idx] = V[idx];
        if (threadIdx.x == 0) {
            w.rest[side][sct] = 0.0;
            if (sw < 0)
                atomicExch(w.status, (int)HOTRG_ENOCONV);
            else
                atomicMax(&w.sweeps[side], sw);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Subspace path, FP32 part: b columns of block subspace iteration.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b) {
    uint32_t x = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    return (float)(x & 0xffffff) / 8388608.0f - 1.0f;  // [-1, 1)
}

// Orthonormalise the b columns of Y (m x b, ld b) in place: classical
// Gram-Schmidt applied twice per column.  A column whose remainder falls below
// dep_tol of its norm before orthogonalisation is numerically dependent on the
// previous ones (E_q is often rank deficient); it is replaced by a fresh
// pseudo-random vector (salted by the caller) and orthogonalised again, since
// normalising a round-off remainder would destroy orthogonality.
template <typename T>
__device__ void cgs2(T* Y, int m, int b, T* r, double* red, uint32_t salt, double dep_tol) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = 0; j < b; ++j) {
        bool done = false;
        for (int attempt = 0; attempt < 4 && !done; ++attempt) {
            if (attempt > 0) {
                for (int t = threadIdx.x; t < m; t += blockDim.x)
                    Y[(int64_t)t * b + j] = (T)hash_unit((uint32_t)t + 7919u * (salt + (uint32_t)attempt), (uint32_t)j);
                __syncthreads();
            }
            double n0 = 0.0;
            for (int t = threadIdx.x; t < m; t += blockDim.x)
                n0 += (double)Y[(int64_t)t * b + j] * (double)Y[(int64_t)t * b + j];
            n0 = block_reduce_sum(n0, red);
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                for (int i = warp; i < j; i += nw) {
                    T acc = 0;
                    for (int t = lane; t < m; t += 32) acc += Y[(int64_t)t * b + i] * Y[(int64_t)t * b + j];
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) r[i] = acc;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < m; t += blockDim.x) {
                    T acc = 0;
                    for (int i = 0; i < j; ++i) acc += r[i] * Y[(int64_t)t * b + i];
                    Y[(int64_t)t * b + j] -= acc;
                }
                __syncthreads();
            }
            double nrm = 0.0;
            for (int t = threadIdx.x; t < m; t += blockDim.x)
                nrm += (double)Y[(int64_t)t * b + j] * (double)Y[(int64_t)t * b + j];
            nrm = block_reduce_sum(nrm, red);
            if (nrm > dep_tol * dep_tol * n0 && nrm > 1e-280) {
                const T inv = (T)(1.0 / sqrt(nrm));
                for (int t = threadIdx.x; t < m; t += blockDim.x) Y[(int64_t)t * b + j] *= inv;
                done = true;
            }
            __syncthreads();
        }
        if (!done) {  // b exceeds the dimension that can be spanned: leave a zero column
            for (int t = threadIdx.x; t < m; t += blockDim.x) Y[(int64_t)t * b + j] = (T)0;
            __syncthreads();
        }
    }
}

// One-warp CGS2 on the b columns of Yt (stored transposed: column j is the
// contiguous row Yt[j][0..m)), with the same replacement of numerically
// dependent columns as cgs2().  Only warp-level synchronisation.
__device__ void cgs2_warp_t(float* Yt, int m, int b, uint32_t salt, float dep_tol, float* rbuf) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < b; ++j) {
        float* yj = Yt + (int64_t)j * m;
        bool done = false;
        for (int attempt = 0; attempt < 4 && !done; ++attempt) {
            if (attempt > 0) {
                for (int t = lane; t < m; t += 32)
                    yj[t] = hash_unit((uint32_t)t + 7919u * (salt + (uint32_t)attempt), (uint32_t)j);
                __syncwarp();
            }
            float n0 = 0.f;
            for (int t = lane; t < m; t += 32) n0 = fmaf(yj[t], yj[t], n0);
            for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(0xffffffffu, n0, o);
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                for (int i = 0; i < j; ++i) {
                    const float* yi = Yt + (int64_t)i * m;
                    float acc = 0.f;
                    for (int t = lane; t < m; t += 32) acc = fmaf(yi[t], yj[t], acc);
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) rbuf[i] = acc;
                }
                __syncwarp();
                for (int t = lane; t < m; t += 32) {
                    float acc = yj[t];
                    for (int i = 0; i < j; ++i) acc = fmaf(-rbuf[i], Yt[(int64_t)i * m + t], acc);
                    yj[t] = acc;
                }
                __syncwarp();
            }
            float nrm = 0.f;
            for (int t = lane; t < m; t += 32) nrm = fmaf(yj[t], yj[t], nrm);
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            if (nrm > dep_tol * dep_tol * n0 && nrm > 1e-30f) {
                const float inv = rsqrtf(nrm);
                for (int t = lane; t < m; t += 32) yj[t] *= inv;
                done = true;
            }
            __syncwarp();
        }
        if (!done) {
            for (int t = lane; t < m; t += 32) yj[t] = 0.f;
            __syncwarp();
        }
    }
}

// Blocks handled by subspace_fast_kernel (b <= 32 listed vectors, Q and Y in shared memory).
constexpr int SUBF_BMAX = 32;
constexpr int SUBF_SMEM = 200 * 1024;  // Q and Y: 2 b m floats

__device__ __forceinline__ bool subf_ok(int b, int m) {
    return b <= SUBF_BMAX && (size_t)2 * b * m * sizeof(float) <= (size_t)SUBF_SMEM;
}

// Sum of v over the block, returned to every thread (red: >= 33 floats of shared memory).
__device__ __forceinline__ float block_sum_f32(float v, float* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = lane < nw ? red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    const float r = red[32];
    __syncthreads();
    return r;
}

// cgs2_warp_t on the whole block: the j dot products of each projection are
// spread over the warps, the update and the norms over all threads.  Same
// algorithm (two classical Gram-Schmidt passes, dependent columns replaced by
// hashed random columns, at most four attempts), fixed reduction order.
__device__ void cgs2_block_t(float* Yt, int m, int b, uint32_t salt, float dep_tol, float* rbuf, float* red,
                             int attempts) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < b; ++j) {
        float* yj = Yt + (int64_t)j * m;
        bool done = false;
        for (int attempt = 0; attempt < attempts && !done; ++attempt) {
            if (attempt > 0) {
                for (int t = tid; t < m; t += blockDim.x)
                    yj[t] = hash_unit((uint32_t)t + 7919u * (salt + (uint32_t)attempt), (uint32_t)j);
                __syncthreads();
            }
            float p0 = 0.f;
            for (int t = tid; t < m; t += blockDim.x) p0 = fmaf(yj[t], yj[t], p0);
            const float n0 = block_sum_f32(p0, red);
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                for (int i = wid; i < j; i += nw) {
                    const float* yi = Yt + (int64_t)i * m;
                    float acc = 0.f;
                    for (int t = lane; t < m; t += 32) acc = fmaf(yi[t], yj[t], acc);
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) rbuf[i] = acc;
                }
                __syncthreads();
                for (int t = tid; t < m; t += blockDim.x) {
                    float acc = yj[t];
                    for (int i = 0; i < j; ++i) acc = fmaf(-rbuf[i], Yt[(int64_t)i * m + t], acc);
                    yj[t] = acc;
                }
                __syncthreads();
            }
            float p1 = 0.f;
            for (int t = tid; t < m; t += blockDim.x) p1 = fmaf(yj[t], yj[t], p1);
            const float nrm = block_sum_f32(p1, red);
            if (nrm > dep_tol * dep_tol * n0 && nrm > 1e-30f) {
                const float inv = rsqrtf(nrm);
                for (int t = tid; t < m; t += blockDim.x) yj[t] *= inv;
                done = true;
            }
            __syncthreads();
        }
        if (!done) {
            for (int t = tid; t < m; t += blockDim.x) yj[t] = 0.f;
            __syncthreads();
        }
    }
}

// FP32 block subspace iteration on one block: Qt, Yt are b x m (transposed);
// the product Yt = (E_q Q)^T and the orthonormalisation run on all warps.
__global__ void __launch_bounds__(SUB_THREADS) subspace_fp32_kernel(const double* EL, const double* ER, int n,
                                                                    int iters, int dep_attempts, EigWs w) {
    __shared__ float Es[32][65];
    __shared__ float Qs[BCAP_MAX][65];
    __shared__ float rbuf[BCAP_MAX];
    __shared__ float red[40];
    const int side = blockIdx.y;
    const double* E = side == 0 ? EL : ER;
    const int nsec = *w.nsec;
    for (int sct = blockIdx.x; sct < nsec; sct += gridDim.x) {
        const int start = w.sec_start[sct];
        const int m = w.sec_start[sct + 1] - start;
        const int b = w.sec_b[sct];
        if (b == m || subf_ok(b, m)) continue;  // Jacobi / subspace_fast_kernel
        const int64_t aoff = w.sec_aoff[sct];
        float* Ef = (float*)(w.A[side] + aoff);
        float* Q = (float*)(w.S1[side] + aoff);
        float* Y = (float*)(w.S2[side] + aoff);
        double* E64 = w.S3[side] + aoff;
        for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += blockDim.x) {
            const int i = (int)(idx / m), j = (int)(idx % m);
            const double v = E[(int64_t)w.members[start + i] * n + w.members[start + j]];
            E64[idx] = v;
            Ef[idx] = (float)v;
        }
        for (int64_t idx = threadIdx.x; idx < (int64_t)b * m; idx += blockDim.x)
            Q[idx] = hash_unit((uint32_t)(idx % m), (uint32_t)(idx / m));
        __syncthreads();
        cgs2_block_t(Q, m, b, 1u, 1e-3f, rbuf, red, 4);
        for (int it = 0; it < iters; ++it) {
            // Yt[j][i] = sum_k Ef[i][k] Qt[j][k], tiles of 32 rows x 64 k
            for (int r0 = 0; r0 < m; r0 += 32) {
                float acc[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = 0.f;
                for (int k0 = 0; k0 < m; k0 += 64) {
                    for (int idx = threadIdx.x; idx < 32 * 64; idx += blockDim.x) {
                        const int i = idx / 64, k = idx % 64;
                        Es[i][k] = (r0 + i < m && k0 + k < m) ? Ef[(int64_t)(r0 + i) * m + k0 + k] : 0.f;
                    }
                    for (int idx = threadIdx.x; idx < b * 64; idx += blockDim.x) {
                        const int j = idx / 64, k = idx % 64;
                        Qs[j][k] = (k0 + k < m) ? Q[(int64_t)j * m + k0 + k] : 0.f;
                    }
                    __syncthreads();
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int o = threadIdx.x + u * SUB_THREADS;  // output (i, j) inside the 32 x b tile
                        if (o < 32 * b) {
                            const int i = o % 32, j = o / 32;
                            float a = acc[u];
#pragma unroll 16
                            for (int k = 0; k < 64; ++k) a = fmaf(Es[i][k], Qs[j][k], a);
                            acc[u] = a;
                        }
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int o = threadIdx.x + u * SUB_THREADS;
                    if (o < 32 * b) {
                        const int i = o % 32, j = o / 32;
                        if (r0 + i < m) Y[(int64_t)j * m + r0 + i] = acc[u];
                    }
                }
            }
            __syncthreads();
            cgs2_block_t(Y, m, b, 2u + 4u * (uint32_t)it, 1e-3f, rbuf, red, dep_attempts);
            float* t = Q;  // the orthonormal Y becomes the next Q
            Q = Y;
            Y = t;
        }
        // leave the final basis (b x m, transposed) in S1
        if (Q != (float*)(w.S1[side] + aoff)) {
            float* dst = (float*)(w.S1[side] + aoff);
            for (int64_t idx = threadIdx.x; idx < (int64_t)m * b; idx += blockDim.x) dst[idx] = Q[idx];
        }
        __syncthreads();
    }
}

// Fast path of the FP32 subspace iteration for blocks with b <= 32 listed
// vectors whose Q and Y (b x m each, transposed) fit in shared memory:
//  * Y = (E_q Q)^T one warp per row of E_q, the b sums of a row in registers
//    and reduced with shuffles;
//  * block CGS2 in panels of 2 columns (bcgs2_block), with the same
//    dependent-column replacement as cgs2_warp_t.
__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block CGS2 in panels of BCGS_PW columns on Yt (b x m in shared memory, row j =
// column j).  For each panel: its columns are projected against all previous
// columns twice by the whole block (dot products spread over the warps, then
// one fused update), after which one warp runs CGS2 inside the panel.  A
// column that is numerically dependent (its norm after projection <= dep_tol x
// its norm before any projection) is replaced by a hashed random column and
// projected against every previous column again, at most three times; a
// column that stays dependent is zeroed.  R (BCGS_PW x b floats) and n0
// (BCGS_PW floats) are shared-memory scratch.  Two-column panels: the in-panel
// part runs on one warp while the rest of the block waits, so narrow panels
// leave nearly all the work to the block-wide projections (measured on the
// largest D' = 64 blocks, m ~ 400, b = 24: 142 us per call at 8 columns, 92 at
// 4, 73 at 2 and at 1; the results agree to rounding).
constexpr int BCGS_PW = 2;

// y_c -= <y_i, y_c> y_i for i = lo .. hi-1 (modified Gram-Schmidt), twice; one warp.
__device__ void proj_warp(float* Yt, int m, int c, int lo, int hi) {
    const int lane = threadIdx.x & 31;
    float* yc = Yt + c * m;
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = lo; i < hi; ++i) {
            const float* yi = Yt + i * m;
            float acc = 0.f;
            for (int t = lane; t < m; t += 32) acc = fmaf(yi[t], yc[t], acc);
            acc = warp_sum_f(acc);
            for (int t = lane; t < m; t += 32) yc[t] = fmaf(-acc, yi[t], yc[t]);
            __syncwarp();
        }
    }
}

__device__ void bcgs2_block(float* Yt, int m, int b, uint32_t salt, float dep_tol, float* R, float* n0,
                            int attempts) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int p0 = 0; p0 < b; p0 += BCGS_PW) {
        const int pw = min(BCGS_PW, b - p0);
        // norms before any projection (the dependency test's reference)
        for (int c = warp; c < pw; c += nw) {
            const float* yc = Yt + (p0 + c) * m;
            float a = 0.f;
            for (int t = lane; t < m; t += 32) a = fmaf(yc[t], yc[t], a);
            a = warp_sum_f(a);
            if (lane == 0) n0[c] = a;
        }
        __syncthreads();
        for (int pass = 0; pass < 2 && p0 > 0; ++pass) {
            for (int task = warp; task < p0 * pw; task += nw) {
                const int i = task / pw, c = task % pw;
                const float* yi = Yt + i * m;
                const float* yc = Yt + (p0 + c) * m;
                float a = 0.f;
                for (int t = lane; t < m; t += 32) a = fmaf(yi[t], yc[t], a);
                a = warp_sum_f(a);
                if (lane == 0) R[c * SUBF_BMAX + i] = a;
            }
            __syncthreads();
            for (int idx = tid; idx < pw * m; idx += blockDim.x) {
                const int c = idx / m, t = idx - c * m;
                float acc = Yt[(p0 + c) * m + t];
                for (int i = 0; i < p0; ++i) acc = fmaf(-R[c * SUBF_BMAX + i], Yt[i * m + t], acc);
                Yt[(p0 + c) * m + t] = acc;
            }
            __syncthreads();
        }
        if (warp == 0) {
            for (int c = p0; c < p0 + pw; ++c) {
                float* yc = Yt + c * m;
                float ref = n0[c - p0];
                bool done = false;
                for (int attempt = 0; attempt < attempts && !done; ++attempt) {
                    if (attempt > 0) {
                        for (int t = lane; t < m; t += 32)
                            yc[t] = hash_unit((uint32_t)t + 7919u * (salt + (uint32_t)attempt), (uint32_t)c);
                        __syncwarp();
                        float a = 0.f;
                        for (int t = lane; t < m; t += 32) a = fmaf(yc[t], yc[t], a);
                        ref = warp_sum_f(a);
                        proj_warp(Yt, m, c, 0, p0);  // a fresh column needs the earlier panels too
                    }
                    proj_warp(Yt, m, c, p0, c);
                    float a = 0.f;
                    for (int t = lane; t < m; t += 32) a = fmaf(yc[t], yc[t], a);
                    const float nrm = warp_sum_f(a);
                    if (nrm > dep_tol * dep_tol * ref && nrm > 1e-30f) {
                        const float inv = rsqrtf(nrm);
                        for (int t = lane; t < m; t += 32) yc[t] *= inv;
                        done = true;
                    }
                    __syncwarp();
                }
                if (!done) {
                    for (int t = lane; t < m; t += 32) yc[t] = 0.f;
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SUB_THREADS) subspace_fast_kernel(const double* EL, const double* ER, int n,
                                                                    int iters, int dep_attempts, EigWs w) {
    extern __shared__ float sq[];
    __shared__ float Rs[BCGS_PW * SUBF_BMAX];
    __shared__ float n0s[BCGS_PW];
    const int side = blockIdx.y;
    const double* E = side == 0 ? EL : ER;
    const int nsec = *w.nsec;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int sct = blockIdx.x; sct < nsec; sct += gridDim.x) {
        const int start = w.sec_start[sct];
        const int m = w.sec_start[sct + 1] - start;
        const int b = w.sec_b[sct];
        if (b == m || !subf_ok(b, m)) continue;
        const int64_t aoff = w.sec_aoff[sct];
        float* Ef = (float*)(w.A[side] + aoff);
        double* E64 = w.S3[side] + aoff;
        // the block's state indices go to shared memory first (Q and Y are not live yet), so that
        // each lane keeps four gathered loads of E in flight instead of a dependent pair per value
        int32_t* mem = (int32_t*)sq;
        for (int j = threadIdx.x; j < m; j += blockDim.x) mem[j] = w.members[start + j];
        __syncthreads();
        for (int i = warp; i < m; i += nwarps) {  // rows by warps, columns by lanes (no 64-bit divides)
            const double* erow = E + (int64_t)mem[i] * n;
            for (int j0 = lane; j0 < m; j0 += 128) {
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = j0 + 32 * u < m ? erow[mem[j0 + 32 * u]] : 0.0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + 32 * u;
                    if (j < m) {
                        E64[(int64_t)i * m + j] = v[u];
                        Ef[(int64_t)i * m + j] = (float)v[u];
                    }
                }
            }
        }
        __syncthreads();  // every lane has read mem[] before Q overwrites it
        float* Q = sq;
        float* Y = sq + b * m;
        for (int idx = threadIdx.x; idx < b * m; idx += blockDim.x)
            Q[idx] = hash_unit((uint32_t)(idx % m), (uint32_t)(idx / m));
        __syncthreads();
        bcgs2_block(Q, m, b, 1u, 1e-3f, Rs, n0s, 4);
        for (int it = 0; it < iters; ++it) {
            // two rows of E_q per warp; each lane keeps 4 k values of both rows in flight
            for (int i0 = 2 * warp; i0 < m; i0 += 2 * nwarps) {
                const bool two = i0 + 1 < m;
                const float* er0 = Ef + (int64_t)i0 * m;
                const float* er1 = two ? er0 + m : er0;
                float acc0[SUBF_BMAX], acc1[SUBF_BMAX];
#pragma unroll
                for (int j = 0; j < SUBF_BMAX; ++j) {
                    acc0[j] = 0.f;
                    acc1[j] = 0.f;
                }
                for (int k0 = lane; k0 < m; k0 += 128) {
                    float e0[4], e1[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + 32 * u;
                        e0[u] = k < m ? er0[k] : 0.f;
                        e1[u] = k < m ? er1[k] : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + 32 * u;
                        if (k < m) {
#pragma unroll
                            for (int j = 0; j < SUBF_BMAX; ++j)
                                if (j < b) {
                                    const float q = Q[j * m + k];
                                    acc0[j] = fmaf(e0[u], q, acc0[j]);
                                    acc1[j] = fmaf(e1[u], q, acc1[j]);
                                }
                        }
                    }
                }
                float mine0 = 0.f, mine1 = 0.f;
#pragma unroll
                for (int j = 0; j < SUBF_BMAX; ++j)
                    if (j < b) {
                        const float v0 = warp_sum_f(acc0[j]);
                        const float v1 = warp_sum_f(acc1[j]);
                        if (lane == j) {
                            mine0 = v0;
                            mine1 = v1;
                        }
                    }
                if (lane < b) {
                    Y[lane * m + i0] = mine0;
                    if (two) Y[lane * m + i0 + 1] = mine1;
                }
            }
            __syncthreads();
            bcgs2_block(Y, m, b, 2u + 4u * (uint32_t)it, 1e-3f, Rs, n0s, dep_attempts);
            float* t = Q;  // the orthonormal Y becomes the next Q
            Q = Y;
            Y = t;
        }
        // the final basis (b x m, transposed) goes to S1, as from subspace_fp32_kernel
        float* dst = (float*)(w.S1[side] + aoff);
        for (int idx = threadIdx.x; idx < b * m; idx += blockDim.x) dst[idx] = Q[idx];
        __syncthreads();
    }
}

// Entry k of the upper triangle of a b x b matrix, rows in order: row i starts at
// S(i) = i b - i (i - 1) / 2; i from the quadratic's root in FP32 (exact integers below 2^24),
// then corrected by whole rows.
__device__ __forceinline__ void tri_entry(int k, int b, int& i, int& j) {
    const float c = (float)(2 * b + 1);
    i = (int)((c - sqrtf(c * c - 8.0f * (float)k)) * 0.5f);
    i = max(0, min(i, b - 1));
    while (i + 1 < b && (i + 1) * b - (i + 1) * i / 2 <= k) ++i;
    while (i > 0 && i * b - i * (i - 1) / 2 > k) --i;
    j = i + (k - (i * b - i * (i - 1) / 2));
}

// Upper triangle of H = X^T Y (X, Y: m x b row-major in global memory; i <= j), accumulated in
// H[i * b + j] in row order.  Rows are staged R at a time (R b contiguous doubles of each
// operand, so every global read is coalesced); each thread owns a fixed set of entries, walked
// in a dense enumeration of the triangle.  Ends with a block barrier.
__device__ void gram_upper(const double* X, const double* Y, int m, int b, double* H, double* stage, int R) {
    const int ntri = b * (b + 1) / 2;
    for (int k = threadIdx.x; k < ntri; k += blockDim.x) {
        int i, j;
        tri_entry(k, b, i, j);
        H[i * b + j] = 0.0;
    }
    double* xs = stage;
    double* ys = stage + R * b;
    for (int t0 = 0; t0 < m; t0 += R) {
        const int r = min(R, m - t0);
        __syncthreads();  // the previous chunk has been consumed
        for (int e = threadIdx.x; e < r * b; e += blockDim.x) {
            xs[e] = X[(int64_t)t0 * b + e];
            ys[e] = Y[(int64_t)t0 * b + e];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < ntri; k += blockDim.x) {
            int i, j;
            tri_entry(k, b, i, j);
            double a = H[i * b + j];
            for (int u = 0; u < r; ++u) a = fma(xs[u * b + i], ys[u * b + j], a);
            H[i * b + j] = a;
        }
    }
    __syncthreads();
}

// One warp: in-place Cholesky G = R^T R of a b x b Gram matrix of unit-norm columns (R upper,
// in G's upper triangle).  A pivot at or below 1e-8 marks its column dependent or zeroed: it is
// dropped (live[j] = 0, row j of R set to e_j).  rinv[j] = 1 / R_jj, so that the solve below
// multiplies (an FP64 divide is a long instruction sequence on this part).
__device__ void chol_upper_warp(double* G, int b, int* live, double* rinv) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < b; ++j) {
        const double d = G[j * b + j];
        __syncwarp();
        const bool ok = d > 1e-8;
        const double rjj = ok ? sqrt(d) : 1.0;
        const double ri = 1.0 / rjj;
        if (lane == 0) {
            live[j] = ok ? 1 : 0;
            rinv[j] = ri;
        }
        for (int c = j + lane; c < b; c += 32)
            G[j * b + c] = ok ? (c == j ? rjj : G[j * b + c] * ri) : (c == j ? 1.0 : 0.0);
        __syncwarp();
        // trailing update: G[r][c] -= R[j][r] R[j][c] for j < r <= c
        for (int idx = lane; idx < b * b; idx += 32) {
            const int r = idx / b, c = idx % b;
            if (r > j && c >= r) G[r * b + c] -= G[j * b + r] * G[j * b + c];
        }
        __syncwarp();
    }
}

// Q <- Q R^-1 row by row (forward substitution x R = q, in place: q[i], i < j, already holds
// x_i); dropped columns become zero.  Ends with a block barrier.
__device__ void chol_solve_rows(double* Q, int m, int b, const double* G, const int* live, const double* rinv) {
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        double* q = Q + (int64_t)t * b;
        for (int j = 0; j < b; ++j) {
            if (!live[j]) {
                q[j] = 0.0;
                continue;
            }
            double a = q[j];
            for (int i = 0; i < j; ++i) a = fma(-q[i], G[i * b + j], a);
            q[j] = a * rinv[j];
        }
    }
    __syncthreads();
}

// FP64 basis from the FP32 one: Q64 = double(Q32) R^-1 with R the Cholesky
// factor of G = Q64^T Q64 (one Cholesky QR).  The FP32 basis is orthonormal
// to ~1e-7, so G is within ~1e-7 of the identity and one pass leaves Q64
// orthonormal to rounding.  A column whose pivot falls below 1e-8 of its
// diagonal (a column the FP32 stage zeroed, or a dependent one) is set to
// zero and dropped from the factorisation.  Result in S2, m x b row-major.
__global__ void __launch_bounds__(SUB_THREADS) rr_prep_kernel(EigWs w, int smem_doubles) {
    extern __shared__ double G[];  // b x b, then the row-chunk staging area (smem_doubles in all)
    __shared__ int live[BCAP_MAX];
    __shared__ double rinv[BCAP_MAX];
    const int side = blockIdx.y;
    const int nsec = *w.nsec;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int sct = blockIdx.x; sct < nsec; sct += gridDim.x) {
        const int m = w.sec_start[sct + 1] - w.sec_start[sct];
        const int b = w.sec_b[sct];
        if (b == m) continue;
        const int64_t aoff = w.sec_aoff[sct];
        const float* Q32 = (const float*)(w.S1[side] + aoff);  // b x m (transposed)
        double* Q = w.S2[side] + aoff;
        for (int t = warp; t < m; t += nw)
            for (int j = lane; j < b; j += 32) Q[(int64_t)t * b + j] = (double)Q32[(int64_t)j * m + t];
        __syncthreads();
        // G = Q^T Q, upper triangle (all the Cholesky reads), from row chunks staged in shared
        // memory, FP64 FMAs only (widening the FP32 basis inside this loop made the kernel 30%
        // slower: each conversion is one more FP64-pipe instruction)
        gram_upper(Q, Q, m, b, G, G + b * b, min(128, (smem_doubles - b * b) / (2 * b)));
        if (warp == 0) chol_upper_warp(G, b, live, rinv);
        __syncthreads();
        chol_solve_rows(Q, m, b, G, live, rinv);
    }
}

// Y = E_q Q (FP64) for all subspace blocks: CTA (row tile, block); 32 rows x b columns.
__global__ void __launch_bounds__(256) rr_product_kernel(EigWs w) {
    __shared__ double Es[GB_ROWS][33];
    __shared__ double Qs[32][BCAP_MAX + 1];
    const int side = blockIdx.z;
    const int nsec = *w.nsec;
    for (int sct = blockIdx.y; sct < nsec; sct += gridDim.y) {
        const int m = w.sec_start[sct + 1] - w.sec_start[sct];
        const int b = w.sec_b[sct];
        if (b == m) continue;
        const int64_t aoff = w.sec_aoff[sct];
        const double* E = w.S3[side] + aoff;
        const double* Q = w.S2[side] + aoff;
        double* Y = w.S4[side] + aoff;
        for (int r0 = blockIdx.x * GB_ROWS; r0 < m; r0 += gridDim.x * GB_ROWS) {
            double acc[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u] = 0.0;
            for (int k0 = 0; k0 < m; k0 += 32) {
                for (int idx = threadIdx.x; idx < GB_ROWS * 32; idx += blockDim.x) {
                    const int i = idx / 32, k = idx % 32;
                    Es[i][k] = (r0 + i < m && k0 + k < m) ? E[(int64_t)(r0 + i) * m + k0 + k] : 0.0;
                }
                for (int idx = threadIdx.x; idx < 32 * b; idx += blockDim.x) {
                    const int k = idx / b, j = idx % b;
                    Qs[k][j] = (k0 + k < m) ? Q[(int64_t)(k0 + k) * b + j] : 0.0;
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int o = threadIdx.x + u * 256;
                    if (o < GB_ROWS * b) {
                        const int i = o / b, j = o % b;
                        double a = acc[u];
                        for (int k = 0; k < 32; ++k) a = fma(Es[i][k], Qs[k][j], a);
                        acc[u] = a;
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int o = threadIdx.x + u * 256;
                if (o < GB_ROWS * b) {
                    const int i = o / b, j = o % b;
                    if (r0 + i < m) Y[(int64_t)(r0 + i) * b + j] = acc[u];
                }
            }
        }
    }
}

// H = Q^T Y (Y = E_q Q; exactly symmetric: the upper triangle is mirrored), Jacobi on H, W to
// S1; eigenvalues and the unlisted weight.  The Ritz vectors Q W are formed by the projector,
// for the kept columns only.
__global__ void __launch_bounds__(JAC_THREADS) rr_finish_kernel(int max_sweeps, double tol, EigWs w) {
    extern __shared__ double sm[];
    __shared__ double red[40];
    __shared__ int s_rot;
    const int side = blockIdx.y;
    const int nsec = *w.nsec;
    for (int sct = blockIdx.x; sct < nsec; sct += gridDim.x) {
        const int m = w.sec_start[sct + 1] - w.sec_start[sct];
        const int b = w.sec_b[sct];
        if (b == m) continue;
        const int64_t aoff = w.sec_aoff[sct];
        const double* Q = w.S2[side] + aoff;
        const double* Y = w.S4[side] + aoff;
        const double* E = w.S3[side] + aoff;
        double* H = sm;
        double* W = sm + b * b;
        double* rc = sm + 2 * b * b;
        double* rs = rc + BCAP_MAX / 2;
        int* rp = (int*)(rs + BCAP_MAX / 2);
        int* rq = rp + BCAP_MAX / 2;
        double* stage = (double*)(rq + BCAP_MAX / 2);
        const int avail = (int)(RR_SMEM_BYTES / sizeof(double)) - (int)(stage - sm);
        const int R = min(128, avail / (2 * b));
        gram_upper(Q, Y, m, b, H, stage, R);
        for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
            const int i = idx / b, j = idx % b;
            if (i > j) H[idx] = H[j * b + i];
        }
        __syncthreads();
        const int sw = jacobi_block(H, W, b, max_sweeps, tol, rc, rs, rp, rq, red, &s_rot);
        // W (b x b) to S1, for the projector (Ritz vectors) and for a further FP64 iteration
        // (rr_next_kernel): the FP32 basis that S1 held has been consumed by rr_prep_kernel
        double* Wg = w.S1[side] + aoff;
        for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) Wg[idx] = W[idx];
        const int cs = w.sec_cstart[sct];
        for (int j = threadIdx.x; j < b; j += blockDim.x) w.lam[side][cs + j] = H[j * b + j];
        // unlisted weight: Tr(E_q) - sum of the listed eigenvalues
        double tr = 0.0;
        for (int t = threadIdx.x; t < m; t += blockDim.x) tr += E[(int64_t)t * m + t];
        for (int j = threadIdx.x; j < b; j += blockDim.x) tr -= H[j * b + j];
        tr = block_reduce_sum(tr, red);
        if (threadIdx.x == 0) {
            w.rest[side][sct] = tr > 0.0 ? tr : 0.0;
            if (sw < 0)
                atomicExch(w.status, (int)HOTRG_ENOCONV);
            else
                atomicMax(&w.sweeps[side], sw);
        }
        __syncthreads();
    }
}

// One more FP64 subspace iteration after a Rayleigh-Ritz step: the Ritz basis
// V = Q W has E_q V = Y W (Y = E_q Q from rr_product_kernel, W from
// rr_finish_kernel), so the next basis is the orthonormalised Z = Y W.  Its
// columns are E_q v_j ~ theta_j v_j, nearly orthogonal once normalised, so one
// Cholesky QR (as in rr_prep_kernel, dropping columns whose pivot falls below
// 1e-8 of their unit norm) orthonormalises them to rounding.  Each such
// iteration shrinks the error of the j-th Ritz vector by lambda_{b+1} /
// lambda_j.  Result in S2 (m x b row-major), ready for rr_product_kernel.
__global__ void __launch_bounds__(SUB_THREADS) rr_next_kernel(EigWs w, int smem_doubles) {
    extern __shared__ double G[];  // b x b (the Gram matrix), b x b (W), then row-chunk staging
    __shared__ int live[BCAP_MAX];
    __shared__ double rinv[BCAP_MAX];
    __shared__ double cn[BCAP_MAX];
    const int side = blockIdx.y;
    const int nsec = *w.nsec;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int sct = blockIdx.x; sct < nsec; sct += gridDim.x) {
        const int m = w.sec_start[sct + 1] - w.sec_start[sct];
        const int b = w.sec_b[sct];
        if (b == m) continue;
        const int64_t aoff = w.sec_aoff[sct];
        const double* Y = w.S4[side] + aoff;
        double* Z = w.S2[side] + aoff;
        double* Ws = G + b * b;
        for (int idx = tid; idx < b * b; idx += blockDim.x) Ws[idx] = w.S1[side][aoff + idx];
        __syncthreads();
        for (int64_t idx = tid; idx < (int64_t)m * b; idx += blockDim.x) {
            const int t = (int)(idx / b), j = (int)(idx % b);
            double a = 0.0;
            for (int i = 0; i < b; ++i) a = fma(Y[(int64_t)t * b + i], Ws[i * b + j], a);
            Z[idx] = a;
        }
        __syncthreads();
        // unit column norms (a zero column stays zero and is dropped below)
        for (int j = warp; j < b; j += nw) {
            double a = 0.0;
            for (int t = lane; t < m; t += 32) a = fma(Z[(int64_t)t * b + j], Z[(int64_t)t * b + j], a);
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) cn[j] = a > 1e-280 ? 1.0 / sqrt(a) : 0.0;
        }
        __syncthreads();
        for (int64_t idx = tid; idx < (int64_t)m * b; idx += blockDim.x) Z[idx] *= cn[(int)(idx % b)];
        __syncthreads();
        gram_upper(Z, Z, m, b, G, G + 2 * b * b, min(128, (smem_doubles - 2 * b * b) / (2 * b)));
        if (warp == 0) chol_upper_warp(G, b, live, rinv);
        __syncthreads();
        chol_solve_rows(Z, m, b, G, live, rinv);
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

// Reorders kept[0, k) by block key ascending, keeping the selection order
// within a key (a gauge choice: the kept basis is only defined up to an
// orthogonal map, and the next step's labels come out sorted, so every
// charge-constrained index range of the next contractions is contiguous).
__device__ void sort_kept_by_key(int* kept, int k, const int* slotkey, int* tmp) {
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int ki = slotkey[kept[i]];
        int r = 0;
        for (int j = 0; j < k; ++j) {
            const int kj = slotkey[kept[j]];
            r += (kj < ki) || (kj == ki && j < i);
        }
        tmp[r] = kept[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) kept[i] = tmp[i];
}

__global__ void __launch_bounds__(SORT_THREADS) select_kernel(int dprime, double tie_rtol, EigWs w) {
    extern __shared__ int si[];
    __shared__ double red[40];
    __shared__ int s_bounds[2];
    const int side = blockIdx.x;
    const double* lam = w.lam[side];
    const int n = *w.ncand;
    const int nsec = *w.nsec;
    int* slotkey = si + MAX_N;  // key per slot
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) si[i] = i < n ? i : -1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) slotkey[i] = w.sec_key[w.cand_sec[i]];
    __syncthreads();
    SelCmp cmp{lam, slotkey, 0};
    bitonic_sort_idx(si, npow2, cmp);
    int* kept = w.kept[side];
    // weight of the eigenvalues no block listed
    double unl = 0.0;
    for (int s = threadIdx.x; s < nsec; s += blockDim.x) unl += w.rest[side][s];
    unl = block_reduce_sum(unl, red);
    if (n <= dprime) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) kept[i] = si[i];
        if (threadIdx.x == 0) *w.eps[side] = unl;
        sort_kept_by_key(kept, n, slotkey, slotkey + MAX_N);
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
    // a block whose smallest listed eigenvalue reaches the cut listed too few -- unless the
    // cut itself lies within the cluster width of zero: then the cluster is the noise floor of
    // the spectrum and which of its near-null states fill it does not matter
    for (int s = threadIdx.x; s < nsec; s += blockDim.x) {
        const int m = w.sec_start[s + 1] - w.sec_start[s];
        const int b = w.sec_b[s];
        if (b < m) {
            double lo = 1e300;
            for (int j = 0; j < b; ++j) lo = fmin(lo, lam[w.sec_cstart[s] + j]);
            if (lo >= lcut - tol && lcut > tol) atomicExch(w.status, (int)HOTRG_ENOCONV);
        }
    }
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
    if (threadIdx.x == 0) *w.eps[side] = tot + unl;
    sort_kept_by_key(kept, dprime, slotkey, si);
}

// ---------------------------------------------------------------------------
// Side choice and projector P[(a,b)][j] (P must be zeroed beforehand).
// ---------------------------------------------------------------------------
__global__ void projector_kernel(int dprime, int policy, double side_rtol, EigWs w, double* P, int32_t* q_out,
                                 hotrg_step_info* info) {
    const double eL = *w.eps[0];
    const double eR = policy == 0 ? *w.eps[1] : nan("");
    const int side = (policy == 0 && eR < eL * (1.0 - side_rtol)) ? 1 : 0;
    const int j = blockIdx.x;
    const int slot = w.kept[side][j];
    const int sct = w.cand_sec[slot];
    const int start = w.sec_start[sct];
    const int m = w.sec_start[sct + 1] - start;
    const int b = w.sec_b[sct];
    const int pos = slot - w.sec_cstart[sct];
    const int64_t aoff = w.sec_aoff[sct];
    if (b == m) {  // a Jacobi block: its eigenvectors are stored
        const double* V = w.V[side] + aoff;
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            P[(int64_t)w.members[start + i] * dprime + j] = V[(int64_t)i * b + pos];
    } else {  // a subspace block: Ritz vector Q W[:, pos] (Q in S2, m x b; W in S1, b x b)
        const double* Q = w.S2[side] + aoff;
        const double* Wc = w.S1[side] + aoff + pos;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double* q = Q + (int64_t)i * b;
            double a = 0.0;
            for (int c = 0; c < b; ++c) a = fma(q[c], Wc[(int64_t)c * b], a);
            P[(int64_t)w.members[start + i] * dprime + j] = a;
        }
    }
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

hotrg_status eig_truncate(hotrg_ctx* ctx, const EigPlan& plan, const double* EL, const double* ER,
                          const int32_t* q_h, double* P, int32_t* q_out, hotrg_step_info* info, void* ws) {
    const int n = plan.n;
    if (n > MAX_N) return set_err(ctx, HOTRG_EINVAL, "eig_truncate: Dh^2 above 16384");
    cudaStream_t st = ctx->stream;
    if (attr_once((const void*)sectors_kernel, ctx->device)) {
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(sectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 MAX_N * 8));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(jacobi_sectors_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JAC_SMEM_BYTES));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 MAX_N * 4 * 3));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(rr_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)RR_SMEM_BYTES));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(subspace_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 SUBF_SMEM));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(rr_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)PREP_SMEM_BYTES));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(rr_next_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)NEXT_SMEM_BYTES));
    }
    EigWs w = carve(ws, n);
    // listed width of large blocks in the split forms
    int bcap;
    if (plan.sym == SYM_NONE)
        bcap = plan.dprime + 16;
    else if (plan.sym == SYM_Z2)
        bcap = plan.dprime / 2 + 24;
    else  // U(1): many small blocks, each keeping far fewer than D' states (b = 16 at D' = 64 was
          // measured: 30 % less eigensolve time, but at high temperature and Delta ~ 0.9 some
          // blocks keep more than 16 states there and the check below reported HOTRG_ENOCONV)
        bcap = std::min(plan.dprime + 8, std::max(24, plan.dprime / 3));
    if (bcap > BCAP_MAX) bcap = BCAP_MAX;
    // tuning / diagnosis overrides: HOTRG_EIG_EXACT=1 forces FP64 Jacobi on every
    // block, HOTRG_SUB_ITERS sets the FP32 subspace iterations
    static int force_exact = -1, iters_override = 0, thr_override = 0, bcap_override = 0, dep_attempts_override = 0;
    if (force_exact < 0) {
        const char* v = getenv("HOTRG_EIG_EXACT");
        force_exact = (v && v[0] == '1') ? 1 : 0;
        const char* it = getenv("HOTRG_SUB_ITERS");
        if (it && atoi(it) > 0 && atoi(it) <= 200) iters_override = atoi(it);
        const char* th = getenv("HOTRG_SMALL_THR");
        if (th && atoi(th) > 0) thr_override = atoi(th);
        const char* bc = getenv("HOTRG_BCAP");
        if (bc && atoi(bc) > 0 && atoi(bc) <= BCAP_MAX) bcap_override = atoi(bc);
        const char* da = getenv("HOTRG_DEP_ATTEMPTS");
        if (da && atoi(da) >= 1 && atoi(da) <= 4) dep_attempts_override = atoi(da);
    }
    if (bcap_override) bcap = bcap_override;
    // U(1) blocks list >= 2x their kept count, so the ratio lambda_{b+1} / lambda_kept is
    // tiny and 6 iterations converge (measured at D' = 64: within 3e-12 of FP64 Jacobi
    // on every block); the wider Z2 / no-symmetry blocks keep 12
    const int sub_iters = iters_override ? iters_override : (plan.sym == SYM_U1 ? SUB_ITERS_U1 : SUB_ITERS);
    // attempts per column in the iterations' Gram-Schmidt before a numerically dependent column is
    // zeroed (1: zeroed at once; the initial random basis always gets 4)
    const int dep_attempts = dep_attempts_override ? dep_attempts_override : 4;
    const bool exact = plan.exact || force_exact == 1;
    // blocks of at most bcap states get every eigenpair from FP64 Jacobi (b = m);
    // larger ones list bcap through the subspace path
    int small_thr = exact ? n : bcap;
    if (!exact && thr_override) small_thr = thr_override;
    const int hp0 = prof_begin(ctx);
    sectors_kernel<<<1, SORT_THREADS, MAX_N * 8, st>>>(q_h, plan.Dh, plan.sym, small_thr, bcap, w);
    HOTRG_COUNT(3);  // sectors, jacobi, select
    HOTRG_COUNT(exact ? 1 : 6);  // projector (+ two subspace kernels, rr_prep, rr_product, rr_finish)
    HOTRG_LAUNCH_CHECK(ctx, "sectors_kernel");
    const int sides = plan.env_policy == 0 ? 2 : 1;
    const int grid = n < 2 * ctx->sm_count ? n : 2 * ctx->sm_count;
    jacobi_sectors_kernel<<<dim3(grid, sides), JAC_THREADS, JAC_SMEM_BYTES, st>>>(EL, ER, n, plan.max_sweeps,
                                                                                  plan.tol, w);
    HOTRG_LAUNCH_CHECK(ctx, "jacobi_sectors_kernel");
    prof_end(ctx, hp0, PROF_EIG_PART0 + 0, 0.0);
    if (!exact) {
        const int sgrid = n < ctx->sm_count ? n : ctx->sm_count;
        const int hp1 = prof_begin(ctx);
        subspace_fast_kernel<<<dim3(sgrid, sides), SUB_THREADS, SUBF_SMEM, st>>>(EL, ER, n, sub_iters, dep_attempts,
                                                                                  w);
        subspace_fp32_kernel<<<dim3(sgrid, sides), SUB_THREADS, 0, st>>>(EL, ER, n, sub_iters, dep_attempts, w);
        prof_end(ctx, hp1, PROF_EIG_PART0 + 1, 0.0);
        HOTRG_LAUNCH_CHECK(ctx, "subspace_fp32_kernel");
        const int hp2 = prof_begin(ctx);
        const size_t prep_smem = (size_t)bcap * bcap * sizeof(double) + RR_STAGE_BYTES;
        rr_prep_kernel<<<dim3(sgrid, sides), SUB_THREADS, prep_smem, st>>>(w, (int)(prep_smem / sizeof(double)));
        HOTRG_LAUNCH_CHECK(ctx, "rr_prep_kernel");
        const int tiles = (n + GB_ROWS - 1) / GB_ROWS;
        rr_product_kernel<<<dim3(tiles < 64 ? tiles : 64, sgrid < 32 ? sgrid : 32, sides), 256, 0, st>>>(w);
        HOTRG_LAUNCH_CHECK(ctx, "rr_product_kernel");
        rr_finish_kernel<<<dim3(sgrid, sides), JAC_THREADS, RR_SMEM_BYTES, st>>>(plan.max_sweeps, plan.tol, w);
        HOTRG_LAUNCH_CHECK(ctx, "rr_finish_kernel");
        // further FP64 subspace iterations, each followed by its Rayleigh-Ritz step
        for (int r = 0; r < plan.fp64_iters; ++r) {
            const size_t next_smem = (size_t)2 * bcap * bcap * sizeof(double) + RR_STAGE_BYTES;
            rr_next_kernel<<<dim3(sgrid, sides), SUB_THREADS, next_smem, st>>>(w, (int)(next_smem / sizeof(double)));
            rr_product_kernel<<<dim3(tiles < 64 ? tiles : 64, sgrid < 32 ? sgrid : 32, sides), 256, 0, st>>>(w);
            rr_finish_kernel<<<dim3(sgrid, sides), JAC_THREADS, RR_SMEM_BYTES, st>>>(plan.max_sweeps, plan.tol, w);
            HOTRG_COUNT(3);
            HOTRG_LAUNCH_CHECK(ctx, "FP64 subspace iteration");
        }
        prof_end(ctx, hp2, PROF_EIG_PART0 + 2, 0.0);
    }
    const int hp3 = prof_begin(ctx);
    select_kernel<<<sides, SORT_THREADS, MAX_N * 4 * 3, st>>>(plan.dprime, plan.tie_rtol, w);
    HOTRG_LAUNCH_CHECK(ctx, "select_kernel");
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(P, 0, (size_t)n * plan.dprime * sizeof(double), st));
    projector_kernel<<<plan.dprime, 128, 0, st>>>(plan.dprime, plan.env_policy, plan.side_rtol, w, P, q_out, info);
    HOTRG_LAUNCH_CHECK(ctx, "projector_kernel");
    prof_end(ctx, hp3, PROF_EIG_PART0 + 3, 0.0);
    return HOTRG_OK;
}

}  // namespace hotrg
