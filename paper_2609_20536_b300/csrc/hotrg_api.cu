// C ABI of libhotrg and the host-side orchestration of one HOTRG step.
//
// One step (§2.4.1), for T[l][r][u][d] with Dh = dim(l) = dim(r), Dv = dim(u) = dim(d):
//   environments (Eq. 2.12 via E = M_(l) M_(l)^T without forming M of Eq. 2.11)
//     A[(l1,i),(l1',j)] = sum_{r,u} T[l1,r,u,i] T[l1',r,u,j]
//     B[(l2,i),(l2',j)] = sum_{r,d} T[l2,r,i,d] T[l2',r,j,d]
//     E_L[(l1,l2),(l1',l2')] = sum_{i,j} A[l1,i,l1',j] B[l2,i,l2',j]     (E_R on the r legs)
//   truncation: sector eigensolve, cut cluster, eps_1 / eps_2 rule, projector P (Eq. 2.15)
//   coarse tensor (Eq. 2.16) as s1 -> s2 -> s3:
//     W[x,l2,r1,u,i]  = sum_{l1}    P[l1,l2,x] T[l1,r1,u,i]
//     Z[x,r1,u,r2,d]  = sum_{l2,i}  W[x,l2,r1,u,i] T[l2,r2,i,d]          (O(D^7))
//     T'[x,x',u,d]    = sum_{r1,r2} Z[x,r1,u,r2,d] P[r1,r2,x']
//   normalisation c_k = ||T'||_F, relabel (l,r,u,d) <- (u,d,x,x') for the other axis.
// Every contraction is a GEMM C = A B^T over K-contiguous operands; the
// operands are laid out by permutation kernels.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace hotrg {

std::atomic<long long> g_launches{0};

bool attr_once(const void* kernel, int device) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    return done.insert({kernel, device}).second;
}

hotrg_status set_err(hotrg_ctx* ctx, hotrg_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

// ---- profiling ------------------------------------------------------------
int prof_begin(hotrg_ctx* ctx) {
    Profiler& P = ctx->prof;
    if (!P.on) return -1;
    while (P.pool.size() < 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        P.pool.push_back(e);
    }
    ProfMark m;
    m.a = P.pool.back();
    P.pool.pop_back();
    m.b = P.pool.back();
    P.pool.pop_back();
    m.cls = -1;
    m.flops = 0.0;
    cudaEventRecord(m.a, ctx->stream);
    P.pending.push_back(m);
    return (int)P.pending.size() - 1;
}

void prof_end(hotrg_ctx* ctx, int handle, int cls, double flops) {
    if (handle < 0) return;
    ProfMark& m = ctx->prof.pending[handle];
    cudaEventRecord(m.b, ctx->stream);
    m.cls = cls;
    m.flops = flops;
}

// Device-side flop counter of the block planner (its group sizes live on the device).
hotrg_status prof_ensure_dflops(hotrg_ctx* ctx) {
    if (ctx->prof.dflops) return HOTRG_OK;
    HOTRG_CUDA_TRY(ctx, cudaMalloc(&ctx->prof.dflops, 128));
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->prof.dflops, 0, 128, ctx->stream));
    return HOTRG_OK;
}

hotrg_status prof_fold(hotrg_ctx* ctx) {
    Profiler& P = ctx->prof;
    if (P.on && P.dflops) {  // called after a stream synchronisation: the counter is final
        double h[9] = {0.0};
        if (cudaMemcpy(h, P.dflops, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
            for (int c = 0; c < 3; ++c) {
                P.tot.gemm_flops[c] += h[c];
                P.tot.operand_elems[c] += h[3 + c];
                P.tot.output_elems[c] += h[6 + c];
            }
            cudaMemsetAsync(P.dflops, 0, sizeof(h), ctx->stream);
            cudaStreamSynchronize(ctx->stream);
        }
        cudaGetLastError();
    }
    for (ProfMark& m : P.pending) {
        float ms = 0.f;
        if (m.cls >= 0 && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            if (m.cls <= PROF_GEMM_OTHER) {
                P.tot.gemm_calls[m.cls] += 1;
                P.tot.gemm_ms[m.cls] += ms;
                P.tot.gemm_flops[m.cls] += m.flops;
            } else if (m.cls == PROF_SLICE) {
                P.tot.slice_ms += ms;
            } else if (m.cls == PROF_EIG) {
                P.tot.eig_ms += ms;
            } else if (m.cls == PROF_STEP) {
                P.tot.step_ms += ms;
                P.tot.steps += 1;
            } else if (m.cls >= PROF_EIG_PART0 && m.cls < PROF_EIG_PART0 + 4) {
                P.tot.eig_part_ms[m.cls - PROF_EIG_PART0] += ms;
            }
        }
        cudaGetLastError();
        P.pool.push_back(m.a);
        P.pool.push_back(m.b);
    }
    P.pending.clear();
    return HOTRG_OK;
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

hotrg_status ws_reserve(hotrg_ctx* ctx, size_t bytes) {
    ctx->ws.used = 0;
    if (bytes <= ctx->ws.cap) return HOTRG_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (cs != cudaStreamCaptureStatusNone)
        return set_err(ctx, HOTRG_ENOMEM, "workspace too small and the stream is capturing");
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    ctx->ws.base = nullptr;
    ctx->ws.cap = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, HOTRG_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " workspace bytes failed");
    }
    ctx->ws.base = (char*)p;
    ctx->ws.cap = bytes;
    return HOTRG_OK;
}

void* ws_alloc(hotrg_ctx* ctx, size_t bytes) {
    const size_t b = a256(bytes);
    if (ctx->ws.used + b > ctx->ws.cap) return nullptr;
    void* r = ctx->ws.base + ctx->ws.used;
    ctx->ws.used += b;
    return r;
}

// ---------------------------------------------------------------------------
static int sym_of(const hotrg_params* p) {
    if (p->tkind == HOTRG_T_ISING) return SYM_Z2;
    if (p->h != 0.0) return SYM_NONE;
    if (p->h1 != 0.0) return SYM_Z2;
    return SYM_U1;
}

static hotrg_status check_params(hotrg_ctx* ctx, const hotrg_params* p) {
    if (!p) return set_err(ctx, HOTRG_EINVAL, "params is NULL");
    if (!(p->beta > 0.0) || !isfinite(p->beta)) return set_err(ctx, HOTRG_EINVAL, "beta must be > 0");
    if (!(p->delta >= 0.0 && p->delta <= 1.0)) return set_err(ctx, HOTRG_EINVAL, "Delta must lie in [0, 1]");
    if (!(p->h >= 0.0) || !(p->h1 >= 0.0) || !isfinite(p->h) || !isfinite(p->h1))
        return set_err(ctx, HOTRG_EINVAL, "fields h, h1 must be finite and >= 0");
    if (p->tkind != HOTRG_T_PURE && p->tkind != HOTRG_T_ISING)
        return set_err(ctx, HOTRG_EINVAL, "tkind must be HOTRG_T_PURE or HOTRG_T_ISING");
    if (p->n_max < 0 || p->n_max > 64) return set_err(ctx, HOTRG_EINVAL, "n_max must lie in [0, 64]");
    if (p->d_cut < 1 || p->d_cut > 128) return set_err(ctx, HOTRG_EINVAL, "d_cut must lie in [1, 128]");
    if (p->n_steps < 0 || p->n_steps > HOTRG_MAX_STEPS)
        return set_err(ctx, HOTRG_EINVAL, "n_steps must lie in [0, 64]");
    if (p->m_range < 0 || p->m_range > 200) return set_err(ctx, HOTRG_EINVAL, "m_range must lie in [0, 200]");
    if (p->prec < 0 || p->prec > 2) return set_err(ctx, HOTRG_EINVAL, "unknown precision form");
    if (p->env_policy < 0 || p->env_policy > 1) return set_err(ctx, HOTRG_EINVAL, "env_policy must be 0 or 1");
    if (p->prec != HOTRG_FP64 && !ctx->tc_ok)
        return set_err(ctx, HOTRG_ENOTSUP, "tensor-core forms need an sm_103 device");
    if (p->block_sparse < 0 || p->block_sparse > 1)
        return set_err(ctx, HOTRG_EINVAL, "block_sparse must be 0 or 1");
    if (p->eig_mode < 0 || p->eig_mode > 1) return set_err(ctx, HOTRG_EINVAL, "eig_mode must be 0 or 1");
    if (p->eig_fp64_iters < -1 || p->eig_fp64_iters > 8)
        return set_err(ctx, HOTRG_EINVAL, "eig_fp64_iters must lie in [-1, 8]");
    if (p->gxy_q < 0 || p->gxy_q > 4) return set_err(ctx, HOTRG_EINVAL, "gxy_q must lie in [0, 4] (0: q = 2)");
    return HOTRG_OK;
}

static int d0_of(const hotrg_params* p) { return p->tkind == HOTRG_T_ISING ? 2 : 2 * p->n_max + 1; }

// Whether an impurity run can take the block-sparse path: the impurity tensor must obey the
// pure tensor's symmetry.  With h = 0 and h1 != 0 (Z2: charge parity) the cos(2 theta)
// impurity of Eq. 3.21 changes the charge by an even amount, so it keeps the parity rule; the
// cos(theta) impurity (odd) and every impurity at h = h1 = 0 (U(1): charge changed by 1 or 2)
// do not.
static bool imp_blocks_ok(const hotrg_params* p, int imp_kind) {
    return p->tkind != HOTRG_T_ISING && imp_kind == HOTRG_T_IMP_M1 && sym_of(p) == SYM_Z2;
}

// Workspace bytes of one step with the given sizes (everything except T in/out).
static size_t step_bytes(const hotrg_params* p, int Dh, int Dv, bool imp, bool imp_blocks) {
    const size_t n = (size_t)Dh * Dh;
    const size_t Dp = std::min<size_t>(p->d_cut, n);
    const size_t d4 = (size_t)Dh * Dh * Dv * Dv;
    const size_t hv = (size_t)Dh * Dv;
    size_t b = 0;
    // environments
    b += a256(d4 * 8) * 2 + a256(hv * hv * 8) * 2 + a256(d4 * 8) * 2 + a256(n * n * 8) * 3;
    b += eig_workspace_bytes(Dh);
    b += a256(n * Dp * 8) * 3 + a256(Dp * 4);
    // coarse
    const size_t d5 = Dp * Dh * Dh * Dv * Dv;
    b += a256(d4 * 8) * 2 + a256(d5 * 8) * 2 + a256(Dp * Dp * Dv * Dv * 8) * (imp ? 2 : 1);
    b += a256(norm_partials() * 8) + a256(64) * 4;
    b += a256(hv * 4) + a256(n * 4);  // pair tables of the block-sparse intermediates
    const int64_t shapes[5][3] = {{(int64_t)hv, (int64_t)hv, (int64_t)hv},
                                  {(int64_t)n, (int64_t)n, (int64_t)Dv * Dv},
                                  {(int64_t)Dp * Dh, (int64_t)Dh * Dv * Dv, Dh},
                                  {(int64_t)Dp * Dh * Dv, (int64_t)hv, (int64_t)hv},
                                  {(int64_t)Dp * Dv * Dv, (int64_t)Dp, (int64_t)n}};
    size_t g = 0;
    // the dense engine is needed unless every product of the step runs per block (the same
    // condition as do_step's)
    const bool blocks = p->block_sparse && (!imp || imp_blocks) && sym_of(p) != SYM_NONE;
    if (!blocks)
        for (auto& sh : shapes) g = std::max(g, gemm_engine_workspace(p->prec, sh[0], sh[1], sh[2]));
    if (blocks) {
        // grouped products: (M, K, N) of s1, s2, s3 and of the environments' A, B and E
        const int64_t gs[5][3] = {{(int64_t)Dp * Dh, Dh, (int64_t)Dh * Dv * Dv},
                                  {(int64_t)Dp * Dh * Dv, (int64_t)hv, (int64_t)hv},
                                  {(int64_t)Dp * Dv * Dv, (int64_t)n, (int64_t)Dp},
                                  {(int64_t)hv, (int64_t)hv, (int64_t)hv},
                                  {(int64_t)n, (int64_t)Dv * Dv, (int64_t)n}};
        for (auto& sh : gs)
            g = std::max(g, bs_plan_bytes(sh[0], sh[1], sh[2]) +
                                (p->prec == HOTRG_FP64 ? 0 : umma_grouped_workspace(sh[0], sh[1], sh[2], sym_of(p))) +
                                4096);
    }
    b += g;
    return b;
}

// Sizes (Dh, Dv) of every step of a run from D0.
static void step_sizes(const hotrg_params* p, int D0, std::vector<int>& dh, std::vector<int>& dv) {
    int h = D0, v = D0;
    for (int k = 0; k < p->n_steps; ++k) {
        dh.push_back(h);
        dv.push_back(v);
        const int dp = (int)std::min<long>(p->d_cut, (long)h * h);
        h = v;
        v = dp;
    }
}

struct Perm {
    int nd;
    int64_t od[6], is[6];
};

static void permute(hotrg_ctx* ctx, const double* in, double* out, const Perm& pm) {
    launch_permute(in, out, pm.nd, pm.od, pm.is, ctx->stream);
}

// C = A B^T through the selected contraction engine.
static hotrg_status gemm(hotrg_ctx* ctx, int prec, int64_t M, int64_t N, int64_t K, const double* A,
                         const double* B, double* C, bool coarse) {
    return gemm_engine(ctx, prec, (int)M, (int)N, (int)K, A, K, B, K, C, N, coarse);
}

// E (n x n) for one side.  X1 rows (a, i) cols (b, c) gives A, X2 gives B.
static hotrg_status environment(hotrg_ctx* ctx, int prec, const double* T, int Dh, int Dv, bool right,
                                double* X1, double* X2, double* Am, double* Bm, double* A2, double* B2,
                                double* Ep, double* E) {
    const int64_t hv = (int64_t)Dh * Dv;
    const int64_t sL = (int64_t)Dh * Dv * Dv, sR = (int64_t)Dv * Dv, sU = Dv, sD = 1;
    const int64_t sa = right ? sR : sL, sb = right ? sL : sR;  // truncated leg, other horizontal leg
    // X1[a][d][b][u] -> A[(a,i),(a',j)] = sum_{b,u} T T  (i = down leg of the upper tensor)
    Perm p1{4, {Dh, Dv, Dh, Dv}, {sa, sD, sb, sU}};
    permute(ctx, T, X1, p1);
    // X2[a][u][b][d] -> B[(a,i),(a',j)] = sum_{b,d} T T  (i = up leg of the lower tensor)
    Perm p2{4, {Dh, Dv, Dh, Dv}, {sa, sU, sb, sD}};
    permute(ctx, T, X2, p2);
    hotrg_status s;
    if ((s = gemm(ctx, prec, hv, hv, hv, X1, X1, Am, false)) != HOTRG_OK) return s;
    if ((s = gemm(ctx, prec, hv, hv, hv, X2, X2, Bm, false)) != HOTRG_OK) return s;
    // A2[a][a'][i][j] = A[a][i][a'][j]
    Perm p3{4, {Dh, Dh, Dv, Dv}, {(int64_t)Dv * Dh * Dv, Dv, (int64_t)Dh * Dv, 1}};
    permute(ctx, Am, A2, p3);
    permute(ctx, Bm, B2, p3);
    const int64_t n = (int64_t)Dh * Dh;
    if ((s = gemm(ctx, prec, n, n, (int64_t)Dv * Dv, A2, B2, Ep, false)) != HOTRG_OK) return s;
    // E[a1][a2][a1'][a2'] = Ep[a1][a1'][a2][a2']
    Perm p4{4, {Dh, Dh, Dh, Dh}, {(int64_t)Dh * Dh * Dh, Dh, (int64_t)Dh * Dh, 1}};
    permute(ctx, Ep, E, p4);
    return HOTRG_OK;
}

// T_out[u][d][x][x'] = sum P[l1,l2,x] T_up[l1,r1,u,i] T_dn[l2,r2,i,d] P[r1,r2,x']
// Block-sparse environment (every precision form, U(1) or Z2 labels).  The same three
// products as environment(), read straight out of T and written straight into
// A2[a][a'][i][j], B2[a][a'][i][j] and E[a1][a2][a1'][a2'] through offset
// tables (no permutation).  a is the truncated horizontal leg, b the other
// one; the charge rule q_l + q_u = q_r + q_d gives the block values
//   left  (a = l):  A: (a,i) q_a - q_i | (b,u) q_b - q_u    B: (a,i) q_a + q_i | (b,d) q_b + q_d
//   right (a = r):  A: (a,i) q_a + q_i | (b,u) q_b + q_u    B: (a,i) q_a - q_i | (b,d) q_b - q_d
//   E: K = (i, j) with q_i - q_j; M = (a1, a1') and N = (a2, a2') with the
//      signs that make A[a1 i a1' j] and B[a2 i a2' j] nonzero.
// Only the sector-diagonal blocks of E are written; the eigensolver reads no
// other element.
static hotrg_status environment_blocks(hotrg_ctx* ctx, int prec, int sym, const double* T, const int32_t* qh,
                                       const int32_t* qv, int Dh, int Dv, bool right, double* A2, double* B2,
                                       double* E) {
    const int64_t h = Dh, v = Dv, vv = v * v;
    const int64_t sL = h * vv, sR = vv, sU = v, sD = 1;
    const int64_t sa = right ? sR : sL, sb = right ? sL : sR;
    const int ga = right ? +1 : -1;  // sign of the vertical leg of (a, i) in A's value
    auto run = [&](const BsSet& M, const BsSet& K, const BsSet& N, const double* X, const double* Y, double* C) {
        const size_t mark = ctx->ws.used;
        BsPlan pl;
        hotrg_status st = bs_plan(ctx, sym, M, K, N, PROF_GEMM_ENV, pl, prec == HOTRG_FP64 ? INT32_MAX : 0,
                                  prec == HOTRG_FP64 ? 128 : ctx->tile_n[0]);
        if (st == HOTRG_OK) st = grouped_engine(ctx, prec, pl, X, 0, Y, 0, C, 0, PROF_GEMM_ENV);
        ctx->ws.used = mark;
        return st;
    };
    hotrg_status s;
    // A[(a,i),(a',j)] = sum_{b,u} T(a, b, u, i = d) T(a', b, u, j = d)
    {
        BsSet M{2, {{qh, h, +1, sa, vv * h}, {qv, v, ga, sD, v}}, h * v};
        BsSet K{2, {{qh, h, +1, sb, sb}, {qv, v, ga, sU, sU}}, h * v};
        BsSet N{2, {{qh, h, +1, sa, vv}, {qv, v, ga, sD, 1}}, h * v};
        if ((s = run(M, K, N, T, T, A2)) != HOTRG_OK) return s;
    }
    // B[(a,i),(a',j)] = sum_{b,d} T(a, b, i = u, d) T(a', b, j = u, d)
    {
        BsSet M{2, {{qh, h, +1, sa, vv * h}, {qv, v, -ga, sU, v}}, h * v};
        BsSet K{2, {{qh, h, +1, sb, sb}, {qv, v, -ga, sD, sD}}, h * v};
        BsSet N{2, {{qh, h, +1, sa, vv}, {qv, v, -ga, sU, 1}}, h * v};
        if ((s = run(M, K, N, T, T, B2)) != HOTRG_OK) return s;
    }
    // E[a1][a2][a1'][a2'] = sum_{i,j} A2[a1][a1'][i][j] B2[a2][a2'][i][j]
    {
        const int sm = right ? -1 : +1;  // left: q_a1 - q_a1', q_a2' - q_a2; right: the negatives
        BsSet M{2, {{qh, h, sm, h * vv, h * h * h}, {qh, h, -sm, vv, h}}, h * h};
        BsSet K{2, {{qv, v, +1, v, v}, {qv, v, -1, 1, 1}}, vv};
        BsSet N{2, {{qh, h, -sm, h * vv, h * h}, {qh, h, sm, vv, 1}}, h * h};
        if ((s = run(M, K, N, A2, B2, E)) != HOTRG_OK) return s;
    }
    return HOTRG_OK;
}

static hotrg_status coarse(hotrg_ctx* ctx, int prec, const double* P, int Dh, int Dv, int Dp,
                           const double* T_up, const double* T_dn, double* Pt, double* Pt2, double* Tt,
                           double* Tb, double* W, double* W2, double* Tc, double* T_out) {
    const int64_t hh = (int64_t)Dh * Dh, vv = (int64_t)Dv * Dv;
    hotrg_status s;
    static int no_gather = -1;  // HOTRG_NO_GATHER=1: permuted copies instead of gather maps (diagnosis)
    if (no_gather < 0) {
        const char* v = getenv("HOTRG_NO_GATHER");
        no_gather = (v && v[0] == '1') ? 1 : 0;
    }
    if (prec != HOTRG_FP64 && !no_gather) {
        // split forms: every operand is sliced straight out of its tensor through a gather map
        // {rd1, rd2, rs0, rs1, rs2, kd, ks0, ks1}; no D^5 permutation is materialised.
        const int64_t BIG = 1 << 30;
        const int64_t h = Dh, v = Dv, p = Dp;
        // s1: W[(x,l2),(r1,u,i)] = sum_l1 P[l1][l2][x] T_up[l1][(r1,u,i)]
        const int64_t a1[8] = {1, h, 1, 0, p, BIG, 0, h * p};
        const int64_t b1[8] = {1, 1, 1, 0, 0, BIG, 0, h * vv};
        if ((s = umma_contract_gather(ctx, prec, (int)(p * h), (int)(h * vv), Dh, P, a1, T_up, b1, W, h * vv,
                                      true)) != HOTRG_OK)
            return s;
        // s2: Z'[(x,r1,u),(d,r2)] = sum_{(l2,i)} W[x][l2][r1][u][i] T_dn[l2][r2][i][d]
        const int64_t a2[8] = {h, v, hh * vv, vv, v, v, h * vv, 1};
        const int64_t b2[8] = {1, h, 1, 0, vv, v, h * vv, v};
        double* Z = W2;
        if ((s = umma_contract_gather(ctx, prec, (int)(p * h * v), (int)(v * h), (int)(h * v), W, a2, T_dn, b2, Z,
                                      v * h, true)) != HOTRG_OK)
            return s;
        // s3: Tc[(x,u,d),x'] = sum_{(r1,r2)} Z'[x][r1][u][d][r2] P[r1][r2][x']
        const int64_t a3[8] = {v, v, h * vv * h, v * h, h, h, vv * h, 1};
        const int64_t b3[8] = {1, 1, 1, 0, 0, BIG, 0, p};
        if ((s = umma_contract_gather(ctx, prec, (int)(p * vv), Dp, (int)hh, Z, a3, P, b3, Tc, p, true)) != HOTRG_OK)
            return s;
        Perm po{4, {Dv, Dv, Dp, Dp}, {(int64_t)Dv * Dp, Dp, vv * Dp, 1}};
        permute(ctx, Tc, T_out, po);
        return HOTRG_OK;
    }
    // s1: W[(x,l2),(r1,u,i)] = Pt[(x,l2),l1] . Tt[(r1,u,i),l1]
    Perm pp{3, {Dp, Dh, Dh}, {1, Dp, (int64_t)Dh * Dp}};
    permute(ctx, P, Pt, pp);
    Perm pt{4, {Dh, Dv, Dv, Dh}, {vv, Dv, 1, (int64_t)Dh * vv}};
    permute(ctx, T_up, Tt, pt);
    if ((s = gemm(ctx, prec, (int64_t)Dp * Dh, (int64_t)Dh * vv, Dh, Pt, Tt, W, true)) != HOTRG_OK) return s;
    // W2[x][r1][u][l2][i] = W[x][l2][r1][u][i]
    Perm pw{5, {Dp, Dh, Dv, Dh, Dv}, {hh * vv, vv, Dv, (int64_t)Dh * vv, 1}};
    permute(ctx, W, W2, pw);
    // s2: Z[(x,r1,u),(r2,d)] = W2[(x,r1,u),(l2,i)] . Tb[(r2,d),(l2,i)]
    Perm pb{4, {Dh, Dv, Dh, Dv}, {vv, 1, (int64_t)Dh * vv, Dv}};
    permute(ctx, T_dn, Tb, pb);
    double* Z = W;  // W is dead after the permutation
    if ((s = gemm(ctx, prec, (int64_t)Dp * Dh * Dv, (int64_t)Dh * Dv, (int64_t)Dh * Dv, W2, Tb, Z, true)) !=
        HOTRG_OK)
        return s;
    // Z2[x][u][d][r1][r2] = Z[x][r1][u][r2][d]
    double* Z2 = W2;
    Perm pz{5, {Dp, Dv, Dv, Dh, Dh}, {hh * vv, (int64_t)Dh * Dv, 1, (int64_t)Dv * Dh * Dv, Dv}};
    permute(ctx, Z, Z2, pz);
    // s3: Tc[(x,u,d),x'] = Z2[(x,u,d),(r1,r2)] . Pt2[x',(r1,r2)]
    Perm pp2{3, {Dp, Dh, Dh}, {1, (int64_t)Dh * Dp, Dp}};
    permute(ctx, P, Pt2, pp2);
    if ((s = gemm(ctx, prec, (int64_t)Dp * vv, Dp, hh, Z2, Pt2, Tc, true)) != HOTRG_OK) return s;
    // relabel for the other axis: T_out[u][d][x][x'] = Tc[x][u][d][x']
    Perm po{4, {Dv, Dv, Dp, Dp}, {(int64_t)Dv * Dp, Dp, vv * Dp, 1}};
    permute(ctx, Tc, T_out, po);
    return HOTRG_OK;
}

// One step; lnz_acc (device, may be null) += weight * ln c_k.
// Block-sparse coarse contraction (pure runs with U(1) or Z2 labels; every
// precision form).  Same s1 -> s2 -> s3 as coarse(), each contraction split into the
// charge blocks of its index sets (q: labels of the legs, qh horizontal, qv
// vertical, qn the new bond from the truncation):
//   s1  M = (x, l2): q_x - q_l2     K = l1: q_l1           N = (r1, u, i): q_r1 - q_u + q_i
//   s2  M = (x, r1, u): q_x - q_r1 + q_u   K = (l2, i): q_l2 + q_i   N = (d, r2): q_d + q_r2
//   s3  M = (x, u, d): q_x + q_u - q_d     K = (r1, r2): q_r1 + q_r2  N = x': q_x'
// These are the charge rules of P (q_x = q_a + q_b) and T (q_l + q_u = q_r + q_d)
// rewritten for each product, so every element a later product reads is
// written by the earlier one.  T_out is zeroed first: s3 writes only its blocks.
// Offsets: W and Z are laid out per the comment below; T and P as usual.
// piW, piZ: workspace for the two pair tables (Dh Dv and Dh Dh entries).
static hotrg_status coarse_blocks(hotrg_ctx* ctx, int prec, int sym, const double* P, const int32_t* qh,
                                  const int32_t* qv, const int32_t* qn, int Dh, int Dv, int Dp, const double* T_up,
                                  const double* T_dn, double* W, double* Z, double* T_out, int32_t* piW,
                                  int32_t* piZ) {
    const int64_t h = Dh, v = Dv, p = Dp, hh = h * h, vv = v * v;
    hotrg_status s;
    // In the split forms W and Z are written and read as exact FP32 pairs (8 bytes, the value
    // hi + lo): the tensor-core epilogue then needs no FP64 arithmetic for these two largest
    // outputs.  The FP64 form keeps them in FP64.
    const int wf = prec == HOTRG_FP64 ? 0 : 1;
    auto run = [&](const BsSet& M, const BsSet& K, const BsSet& N, const void* A, int af, const void* B,
                   void* C, int cf, const int32_t* pi_out) {
        const size_t mark = ctx->ws.used;
        BsPlan pl;
        hotrg_status st = bs_plan(ctx, sym, M, K, N, PROF_GEMM_COARSE, pl, prec == HOTRG_FP64 ? INT32_MAX : 0,
                                  prec == HOTRG_FP64 ? 128 : ctx->tile_n[1], pi_out);
        if (st == HOTRG_OK) st = grouped_engine(ctx, prec, pl, A, af, B, 0, C, cf, PROF_GEMM_COARSE);
        ctx->ws.used = mark;
        return st;
    };
    // The intermediates are stored so that each row of the next product's A
    // operand is one contiguous run: W[x][r1][u][piW(l2,i)] (s2 row (x,r1,u), K (l2,i))
    // and Z[x][u][d][piZ(r1,r2)] (s3 row (x,u,d), K (r1,r2)).  piW lists the h v pairs
    // (l2,i) by their s2 value q_l2 + q_i, piZ the h h pairs (r1,r2) by q_r1 + q_r2, so
    // the K elements of one block sit side by side in the order the planner lists
    // them: the slicer reads whole DRAM lines and the producing epilogue fills them,
    // instead of runs of one leg's equal labels (a few values) among structural zeros.
    if ((s = pair_table(ctx, sym, qh, Dh, qv, Dv, piW)) != HOTRG_OK) return s;
    if ((s = pair_table(ctx, sym, qh, Dh, qh, Dh, piZ)) != HOTRG_OK) return s;
    // s1: W[x][r1][u][piW(l2,i)] = sum_l1 P[l1][l2][x] T_up[l1][r1][u][i]
    {
        BsSet M{2, {{qn, p, +1, 1, hh * vv, 0}, {qh, h, -1, p, 0, v}}, p * h};
        BsSet K{1, {{qh, h, +1, h * p, h * vv}}, h};
        BsSet N{3, {{qh, h, +1, vv, v * h * v, 0}, {qv, v, -1, v, h * v, 0}, {qv, v, +1, 1, 0, 1}}, h * vv};
        if ((s = run(M, K, N, P, 0, T_up, W, wf, piW)) != HOTRG_OK) return s;
    }
    // s2: Z[x][u][d][piZ(r1,r2)] = sum_{l2,i} W[x][r1][u][piW(l2,i)] T_dn[l2][r2][i][d]
    {
        BsSet M{3,
                {{qn, p, +1, hh * vv, vv * hh, 0}, {qh, h, -1, v * h * v, 0, h}, {qv, v, +1, h * v, v * hh, 0}},
                p * h * v};
        BsSet K{2, {{qh, h, +1, v, h * vv}, {qv, v, +1, 1, v}}, h * v, piW};
        BsSet N{2, {{qv, v, +1, 1, hh, 0}, {qh, h, +1, vv, 0, 1}}, v * h};
        if ((s = run(M, K, N, W, wf, T_dn, Z, wf, piZ)) != HOTRG_OK) return s;
    }
    // s3, written straight into the next step's axis order (no relabelling pass):
    // T_out[u][d][x][x'] = sum_{r1,r2} Z[x][u][d][piZ(r1,r2)] P[r1][r2][x']
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(T_out, 0, (size_t)p * vv * p * 8, ctx->stream));
    {
        BsSet M{3, {{qn, p, +1, vv * hh, p}, {qv, v, +1, v * hh, v * p * p}, {qv, v, -1, hh, p * p}}, p * vv};
        BsSet K{2, {{qh, h, +1, h, h * p}, {qh, h, +1, 1, p}}, hh, piZ};
        BsSet N{1, {{qn, p, +1, 1, 1}}, p};
        if ((s = run(M, K, N, Z, wf, P, T_out, 0, nullptr)) != HOTRG_OK) return s;
    }
    return HOTRG_OK;
}

// imp_blocks: the impurity tensor keeps the pure tensor's block rule (imp_blocks_ok), so its
// co-update may run per charge block too.
static hotrg_status do_step(hotrg_ctx* ctx, const hotrg_params* p, const double* T_in, const int32_t* q_h,
                            const int32_t* q_v, int Dh, int Dv, double* T_out, int32_t* q_out, int* dprime,
                            hotrg_step_info* info, const double* Ti_in, double* Ti_out, double* lnz_acc,
                            double weight, bool imp_blocks) {
    (void)q_v;
    const int prec = p->prec;
    const int64_t n = (int64_t)Dh * Dh;
    const int Dp = (int)std::min<int64_t>(p->d_cut, n);
    *dprime = Dp;
    const int64_t d4 = (int64_t)Dh * Dh * Dv * Dv, hv = (int64_t)Dh * Dv;
    auto A = [&](size_t bytes) { return ws_alloc(ctx, bytes); };
    double* X1 = (double*)A(d4 * 8);
    double* X2 = (double*)A(d4 * 8);
    double* Am = (double*)A(hv * hv * 8);
    double* Bm = (double*)A(hv * hv * 8);
    double* A2 = (double*)A(d4 * 8);
    double* B2 = (double*)A(d4 * 8);
    double* Ep = (double*)A(n * n * 8);
    double* EL = (double*)A(n * n * 8);
    double* ER = (double*)A(n * n * 8);
    void* eigws = A(eig_workspace_bytes(Dh));
    double* P = (double*)A(n * Dp * 8);
    double* Pt = (double*)A(n * Dp * 8);
    double* Pt2 = (double*)A(n * Dp * 8);
    const int64_t d5 = (int64_t)Dp * Dh * Dh * Dv * Dv;
    double* Tt = (double*)A(d4 * 8);
    double* Tb = (double*)A(d4 * 8);
    double* W = (double*)A(d5 * 8);
    double* W2 = (double*)A(d5 * 8);
    const int64_t tn = (int64_t)Dp * Dp * Dv * Dv;
    double* Tc = (double*)A(tn * 8);
    double* Ti2 = Ti_in ? (double*)A(tn * 8) : nullptr;
    double* partial = (double*)A(norm_partials() * 8);
    double* norm = (double*)A(64);
    int32_t* piW = (int32_t*)A(hv * 4);
    int32_t* piZ = (int32_t*)A(n * 4);
    if (!X1 || !X2 || !Am || !Bm || !A2 || !B2 || !Ep || !EL || !ER || !eigws || !P || !Pt || !Pt2 || !Tt ||
        !Tb || !W || !W2 || !Tc || (Ti_in && !Ti2) || !partial || !norm || !piW || !piZ)
        return set_err(ctx, HOTRG_ENOMEM, "step workspace exhausted");
    hotrg_status s;
    const int h_step = prof_begin(ctx);
    const int sym = sym_of(p);
    const bool blocks = p->block_sparse && (!Ti_in || imp_blocks) && sym != SYM_NONE;
    if (blocks) {
        if ((s = environment_blocks(ctx, prec, sym, T_in, q_h, q_v, Dh, Dv, false, A2, B2, EL)) != HOTRG_OK)
            return s;
        if (p->env_policy == 0)
            if ((s = environment_blocks(ctx, prec, sym, T_in, q_h, q_v, Dh, Dv, true, A2, B2, ER)) != HOTRG_OK)
                return s;
    } else {
        if ((s = environment(ctx, prec, T_in, Dh, Dv, false, X1, X2, Am, Bm, A2, B2, Ep, EL)) != HOTRG_OK)
            return s;
        if (p->env_policy == 0)
            if ((s = environment(ctx, prec, T_in, Dh, Dv, true, X1, X2, Am, Bm, A2, B2, Ep, ER)) != HOTRG_OK)
                return s;
    }
    EigPlan plan;
    plan.n = (int)n;
    plan.Dh = Dh;
    plan.dprime = Dp;
    plan.sym = sym_of(p);
    plan.max_sweeps = p->eig_max_sweeps > 0 ? p->eig_max_sweeps : 40;
    plan.tol = p->eig_tol > 0 ? p->eig_tol : 1e-15;
    plan.tie_rtol = p->tie_rtol > 0 ? p->tie_rtol : 1e-9;
    plan.side_rtol = p->side_rtol > 0 ? p->side_rtol : 1e-6;
    plan.env_policy = p->env_policy;
    // the FP64 form lists the large U(1) blocks by subspace iteration refined in FP64 (U(1) blocks
    // list at least twice the states they keep, so the iteration converges fast); with Z2 or no
    // symmetry it solves every block by Jacobi; eig_mode = 1 asks for Jacobi everywhere
    plan.exact = p->eig_mode == 1 || (prec == HOTRG_FP64 && plan.sym != SYM_U1);
    plan.fp64_iters =
        p->eig_fp64_iters > 0 ? p->eig_fp64_iters : (p->eig_fp64_iters < 0 ? 0 : (prec == HOTRG_FP64 ? 6 : 0));
    const int h_eig = prof_begin(ctx);
    if ((s = eig_truncate(ctx, plan, EL, p->env_policy == 0 ? ER : nullptr, q_h, P, q_out, info, eigws)) !=
        HOTRG_OK)
        return s;
    prof_end(ctx, h_eig, PROF_EIG, 0.0);
    if (blocks) {
        if ((s = coarse_blocks(ctx, prec, sym, P, q_h, q_v, q_out, Dh, Dv, Dp, T_in, T_in, W, W2, T_out, piW,
                               piZ)) != HOTRG_OK)
            return s;
    } else if ((s = coarse(ctx, prec, P, Dh, Dv, Dp, T_in, T_in, Pt, Pt2, Tt, Tb, W, W2, Tc, T_out)) != HOTRG_OK) {
        return s;
    }
    launch_norm(T_out, tn, partial, norm, ctx->stream);
    if (Ti_in) {
        // T_imp' = [P^T (T_imp above T) P + P^T (T above T_imp) P] / (2 c_k)
        if (blocks) {
            if ((s = coarse_blocks(ctx, prec, sym, P, q_h, q_v, q_out, Dh, Dv, Dp, Ti_in, T_in, W, W2, Ti_out, piW,
                                   piZ)) != HOTRG_OK)
                return s;
            if ((s = coarse_blocks(ctx, prec, sym, P, q_h, q_v, q_out, Dh, Dv, Dp, T_in, Ti_in, W, W2, Ti2, piW,
                                   piZ)) != HOTRG_OK)
                return s;
        } else {
            if ((s = coarse(ctx, prec, P, Dh, Dv, Dp, Ti_in, T_in, Pt, Pt2, Tt, Tb, W, W2, Tc, Ti_out)) != HOTRG_OK)
                return s;
            if ((s = coarse(ctx, prec, P, Dh, Dv, Dp, T_in, Ti_in, Pt, Pt2, Tt, Tb, W, W2, Tc, Ti2)) != HOTRG_OK)
                return s;
        }
        launch_axpby(Ti_out, Ti2, 0.5, 0.5, tn, ctx->stream);
        launch_scale_inv(Ti_out, tn, norm, ctx->stream);
    }
    launch_scale_inv(T_out, tn, norm, ctx->stream);
    launch_step_scalars(norm, info, lnz_acc, weight, ctx->stream);
    HOTRG_LAUNCH_CHECK(ctx, "step");
    prof_end(ctx, h_step, PROF_STEP, 0.0);
    return HOTRG_OK;
}

// hotrg_step: an engine failure of the step (its status word) goes into the step's info
// unless the eigensolver already reported one; the word is cleared for the next step.
__global__ void fold_status_kernel(hotrg_step_info* info, int32_t* st) {
    if (threadIdx.x == 0) {
        const int32_t e = *st;
        if (e != 0 && info && info->status == 0) info->status = e;
        *st = 0;
    }
}

__global__ void log_kernel(double* dst, const double* src) {
    if (threadIdx.x == 0) *dst = log(*src);
}

__global__ void finish_kernel(double* lnz_acc, const double* tr, double weight, double* ln_tr, const double* tr_imp,
                              double* imp_ratio) {
    if (threadIdx.x == 0) {
        const double lt = log(*tr);
        *ln_tr = lt;
        *lnz_acc += weight * lt;
        if (tr_imp) *imp_ratio = *tr_imp / *tr;
    }
}

struct RunDev {
    double lnz, ln_c0, ln_tr, imp_ratio, tr, tr_imp, norm0;
    int32_t status, pad;  // the engine's status word while this point runs (zeroed with the block)
};

// While a point is enqueued (or captured) the engine reports into the point's own slot.
struct StatusSlot {
    hotrg_ctx* ctx;
    StatusSlot(hotrg_ctx* c, int32_t* slot) : ctx(c) { ctx->status_slot = slot; }
    ~StatusSlot() { ctx->status_slot = nullptr; }
};

// Buffers and sizes of one point; carved deterministically from the workspace
// base, so equal classes get equal addresses (a captured graph stays valid).
struct PointPlan {
    int D0 = 0;
    bool imp = false;
    std::vector<int> dh, dv;
    int qmax = 0;
    double *Ta = nullptr, *Tb = nullptr, *Ia = nullptr, *Ib = nullptr;
    int32_t *qa = nullptr, *qb = nullptr, *qspare = nullptr;
    double* scratch = nullptr;
    hotrg_step_info* infos = nullptr;
    RunDev* rd = nullptr;
    double* partial = nullptr;
    hotrg_params* dparams = nullptr;
    size_t step_base = 0;
    size_t bytes = 0;
};

static size_t point_bytes(const hotrg_params* p, int imp_kind, PointPlan& pl) {
    pl.D0 = d0_of(p);
    pl.imp = imp_kind == HOTRG_T_IMP_M || imp_kind == HOTRG_T_IMP_M1;
    pl.dh.clear();
    pl.dv.clear();
    step_sizes(p, pl.D0, pl.dh, pl.dv);
    size_t tmax = (size_t)pl.D0 * pl.D0 * pl.D0 * pl.D0, smax = 0;
    for (size_t k = 0; k < pl.dh.size(); ++k) {
        const size_t Dp = std::min<size_t>(p->d_cut, (size_t)pl.dh[k] * pl.dh[k]);
        tmax = std::max(tmax, Dp * Dp * pl.dv[k] * pl.dv[k]);
        smax = std::max(smax, step_bytes(p, pl.dh[k], pl.dv[k], pl.imp, imp_blocks_ok(p, imp_kind)));
    }
    pl.qmax = std::max(pl.D0, p->d_cut) + 1;
    const size_t fixed = a256(tmax * 8) * (pl.imp ? 4 : 2) + a256(pl.qmax * 4) * 3 + a256(16384) +
                         a256(sizeof(hotrg_step_info) * HOTRG_MAX_STEPS) + a256(sizeof(RunDev)) + a256(8192) +
                         a256(sizeof(hotrg_params));
    pl.bytes = fixed + smax;
    return tmax;
}

// Validate, reserve (may synchronise and grow the workspace; never while
// capturing) and carve the point's buffers.
static hotrg_status plan_point(hotrg_ctx* ctx, const hotrg_params* p, int imp_kind, PointPlan& pl,
                               size_t reserve_at_least) {
    hotrg_status s = check_params(ctx, p);
    if (s != HOTRG_OK) return s;
    const bool imp = imp_kind == HOTRG_T_IMP_M || imp_kind == HOTRG_T_IMP_M1;
    if (imp && p->tkind == HOTRG_T_ISING) return set_err(ctx, HOTRG_EINVAL, "no Ising impurity");
    const size_t tmax = point_bytes(p, imp_kind, pl);
    if ((s = ws_reserve(ctx, std::max(pl.bytes, reserve_at_least))) != HOTRG_OK) return s;
    pl.Ta = (double*)ws_alloc(ctx, tmax * 8);
    pl.Tb = (double*)ws_alloc(ctx, tmax * 8);
    pl.Ia = pl.imp ? (double*)ws_alloc(ctx, tmax * 8) : nullptr;
    pl.Ib = pl.imp ? (double*)ws_alloc(ctx, tmax * 8) : nullptr;
    pl.qa = (int32_t*)ws_alloc(ctx, pl.qmax * 4);
    pl.qb = (int32_t*)ws_alloc(ctx, pl.qmax * 4);
    pl.qspare = (int32_t*)ws_alloc(ctx, pl.qmax * 4);
    pl.scratch = (double*)ws_alloc(ctx, 16384);  // coefficient scratch: 2 x 1024 doubles
    pl.infos = (hotrg_step_info*)ws_alloc(ctx, sizeof(hotrg_step_info) * HOTRG_MAX_STEPS);
    pl.rd = (RunDev*)ws_alloc(ctx, sizeof(RunDev));
    pl.partial = (double*)ws_alloc(ctx, 4096 * 2);
    pl.dparams = (hotrg_params*)ws_alloc(ctx, sizeof(hotrg_params));
    if (!pl.Ta || !pl.Tb || (pl.imp && (!pl.Ia || !pl.Ib)) || !pl.qa || !pl.qb || !pl.qspare || !pl.dparams)
        return set_err(ctx, HOTRG_ENOMEM, "point workspace");
    pl.step_base = ctx->ws.used;
    return HOTRG_OK;
}

// Every device operation of one point, reading beta / Delta / h / h1 from
// pl.dparams: no host synchronisation and no allocation, so it can be captured.
static hotrg_status enqueue_point(hotrg_ctx* ctx, const hotrg_params* p, int imp_kind, PointPlan& pl) {
    cudaStream_t st = ctx->stream;
    StatusSlot slot(ctx, &pl.rd->status);
    const int D0 = pl.D0;
    const bool imp = pl.imp;
    const bool imp_blocks = imp && imp_blocks_ok(p, imp_kind);
    hotrg_status s;
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(pl.rd, 0, sizeof(RunDev), st));
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(pl.infos, 0, sizeof(hotrg_step_info) * HOTRG_MAX_STEPS, st));
    launch_init_tensor(p, pl.dparams, p->tkind, pl.Ta, pl.qa, pl.scratch, st);
    if (imp) launch_init_tensor(p, pl.dparams, imp_kind, pl.Ia, pl.qb, pl.scratch + 1024, st);
    HOTRG_LAUNCH_CHECK(ctx, "init tensor");
    // c_0 = ||T0||_F; T <- T / c_0 (impurity scaled by the same c_0)
    const int64_t n0 = (int64_t)D0 * D0 * D0 * D0;
    launch_norm(pl.Ta, n0, pl.partial, &pl.rd->norm0, st);
    launch_scale_inv(pl.Ta, n0, &pl.rd->norm0, st);
    if (imp) launch_scale_inv(pl.Ia, n0, &pl.rd->norm0, st);
    log_kernel<<<1, 32, 0, st>>>(&pl.rd->ln_c0, &pl.rd->norm0);
    log_kernel<<<1, 32, 0, st>>>(&pl.rd->lnz, &pl.rd->norm0);
    HOTRG_COUNT(2);
    // labels: both legs start with the same labels
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(pl.qb, pl.qa, D0 * 4, cudaMemcpyDeviceToDevice, st));
    int32_t* qh = pl.qa;
    int32_t* qv = pl.qb;
    int32_t* qspare = pl.qspare;
    double* Tcur = pl.Ta;
    double* Tnext = pl.Tb;
    double* Icur = pl.Ia;
    double* Inext = pl.Ib;
    for (int k = 0; k < p->n_steps; ++k) {
        ctx->ws.used = pl.step_base;
        int dp = 0;
        s = do_step(ctx, p, Tcur, qh, qv, pl.dh[k], pl.dv[k], Tnext, qspare, &dp, &pl.infos[k], Icur, Inext,
                    &pl.rd->lnz, ldexp(1.0, -(k + 1)), imp_blocks);
        if (s != HOTRG_OK) return s;
        // new horizontal labels = old vertical labels; new vertical = q_out
        int32_t* old_h = qh;
        qh = qv;
        qv = qspare;
        qspare = old_h;
        std::swap(Tcur, Tnext);
        std::swap(Icur, Inext);
    }
    const int Dx = p->n_steps == 0 ? D0 : (int)std::min<long>(p->d_cut, (long)pl.dh.back() * pl.dh.back());
    const int Dy = p->n_steps == 0 ? D0 : pl.dv.back();
    // the final tensor is [Dy][Dy][Dx][Dx] after relabelling (l,r legs = old vertical)
    launch_trace(Tcur, Dy, Dx, &pl.rd->tr, st);
    if (imp) launch_trace(Icur, Dy, Dx, &pl.rd->tr_imp, st);
    finish_kernel<<<1, 32, 0, st>>>(&pl.rd->lnz, &pl.rd->tr, ldexp(1.0, -p->n_steps), &pl.rd->ln_tr,
                                    imp ? &pl.rd->tr_imp : nullptr, &pl.rd->imp_ratio);
    HOTRG_COUNT(1);
    HOTRG_LAUNCH_CHECK(ctx, "finish");
    return HOTRG_OK;
}

// Unpack a finished point (host copies of its RunDev and step records).
static hotrg_status unpack_point(hotrg_ctx* ctx, const hotrg_params* p, const PointPlan& pl, const RunDev& h,
                                 hotrg_result* out) {
    out->lnz_per_site = h.lnz;
    out->ln_c0 = h.ln_c0;
    out->ln_trace = h.ln_tr;
    out->imp_ratio = pl.imp ? h.imp_ratio : 0.0;
    out->n_steps = p->n_steps;
    out->status = HOTRG_OK;
    if (h.status != 0) {
        out->status = h.status;
        return set_err(ctx, (hotrg_status)h.status,
                       h.status == HOTRG_ENOTSUP
                           ? "block planner: a product's label sums span more values than its table, or a charge "
                             "block is wider than the slice pitch"
                           : "tensor-core engine: a bounded wait ran out");
    }
    for (int k = 0; k < p->n_steps; ++k)
        if (out->step[k].status != HOTRG_OK) {
            out->status = out->step[k].status;
            return set_err(ctx, (hotrg_status)out->status,
                           "step " + std::to_string(k + 1) + ": eigensolver did not converge");
        }
    if (!(h.tr > 0.0) || !isfinite(h.lnz)) {
        out->status = HOTRG_ECUDA;
        return set_err(ctx, HOTRG_ECUDA, "non-positive or non-finite closing trace");
    }
    return HOTRG_OK;
}

static hotrg_status run_point(hotrg_ctx* ctx, const hotrg_params* p, int imp_kind, hotrg_result* out) {
    memset(out, 0, sizeof(*out));
    PointPlan pl;
    hotrg_status s = plan_point(ctx, p, imp_kind, pl, 0);
    if (s != HOTRG_OK) {
        out->status = s;
        return s;
    }
    cudaStream_t st = ctx->stream;
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(pl.dparams, p, sizeof(hotrg_params), cudaMemcpyHostToDevice, st));
    if ((s = enqueue_point(ctx, p, imp_kind, pl)) != HOTRG_OK) {
        out->status = s;
        return s;
    }
    RunDev h;
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, pl.rd, sizeof(RunDev), cudaMemcpyDeviceToHost, st));
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(out->step, pl.infos, sizeof(hotrg_step_info) * p->n_steps,
                                        cudaMemcpyDeviceToHost, st));
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    prof_fold(ctx);
    return unpack_point(ctx, p, pl, h, out);
}

// ---------------------------------------------------------------------------
// Batched points: LPT over worker streams, one CUDA graph per point class.
// ---------------------------------------------------------------------------
struct ClassKey {
    int n_max, d_cut, n_steps, prec, env_policy, tkind, m_range, eig_max_sweeps, imp_kind, hz, h1z, block_sparse, q,
        eig_mode, eig_fp64_iters;
    double tie_rtol, eig_tol;
    bool operator==(const ClassKey& o) const { return memcmp(this, &o, sizeof(ClassKey)) == 0; }
};

static ClassKey class_of(const hotrg_params* p, int imp_kind) {
    ClassKey k;
    memset(&k, 0, sizeof(k));
    k.n_max = p->n_max;
    k.d_cut = p->d_cut;
    k.n_steps = p->n_steps;
    k.prec = p->prec;
    k.env_policy = p->env_policy;
    k.tkind = p->tkind;
    k.m_range = p->m_range;
    k.eig_max_sweeps = p->eig_max_sweeps;
    k.imp_kind = imp_kind;
    k.hz = p->h == 0.0;
    k.h1z = p->h1 == 0.0;
    k.block_sparse = p->block_sparse;
    k.q = p->gxy_q == 0 ? 2 : p->gxy_q;
    k.eig_mode = p->eig_mode;
    k.eig_fp64_iters = p->eig_fp64_iters;
    k.tie_rtol = p->tie_rtol;
    k.eig_tol = p->eig_tol;
    return k;
}

static double point_cost(const hotrg_params* p) {
    std::vector<int> dh, dv;
    step_sizes(p, d0_of(p), dh, dv);
    double c = 0.0;
    for (size_t k = 0; k < dh.size(); ++k) {
        const double Dp = std::min<double>(p->d_cut, (double)dh[k] * dh[k]);
        c += Dp * std::pow((double)dh[k], 3) * std::pow((double)dv[k], 3) + 1e6;  // s2 flops + fixed cost
    }
    return c;
}

struct Worker {
    hotrg_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;  // joins the worker back into the context's stream
    struct Graph {
        ClassKey key;
        cudaGraphExec_t exec;
        PointPlan plan;
        long long launches;
    };
    std::vector<Graph> graphs;
};

struct Batch {
    std::vector<Worker> workers;
    cudaEvent_t fork = nullptr;  // workers start after the work already on the context's stream
    size_t reserve = 0;
};

static void profile_add(hotrg_profile& a, const hotrg_profile& b) {
    for (int c = 0; c < 3; ++c) {
        a.gemm_calls[c] += b.gemm_calls[c];
        a.gemm_ms[c] += b.gemm_ms[c];
        a.gemm_flops[c] += b.gemm_flops[c];
        a.operand_elems[c] += b.operand_elems[c];
        a.output_elems[c] += b.output_elems[c];
    }
    a.slice_ms += b.slice_ms;
    a.eig_ms += b.eig_ms;
    a.step_ms += b.step_ms;
    a.steps += b.steps;
    for (int c = 0; c < 4; ++c) a.eig_part_ms[c] += b.eig_part_ms[c];
}

static void batch_free(Batch* b) {
    if (!b) return;
    for (Worker& w : b->workers) {
        for (auto& g : w.graphs) cudaGraphExecDestroy(g.exec);
        if (w.ctx) {
            cudaStreamSynchronize(w.stream);
            if (w.ctx->ws.base) cudaFree(w.ctx->ws.base);
            for (cudaEvent_t e : w.ctx->prof.pool) cudaEventDestroy(e);
            if (w.ctx->prof.dflops) cudaFree(w.ctx->prof.dflops);
            if (w.ctx->status_dev) cudaFree(w.ctx->status_dev);
            delete w.ctx;
        }
        if (w.done) cudaEventDestroy(w.done);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // namespace hotrg

using namespace hotrg;


extern "C" {

hotrg_status hotrg_create(hotrg_ctx** out, size_t workspace_bytes, void* cuda_stream) {
    if (!out) return HOTRG_EINVAL;
    *out = nullptr;
    hotrg_ctx* ctx = new (std::nothrow) hotrg_ctx();
    if (!ctx) return HOTRG_ENOMEM;
    ctx->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return HOTRG_ECUDA;
    }
    ctx->device = dev;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return HOTRG_ECUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
    ctx->tc_ok = prop.major == 10 && prop.minor == 3;
    if (cudaMalloc(&ctx->status_dev, 64) != cudaSuccess || cudaMemset(ctx->status_dev, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->status_dev) cudaFree(ctx->status_dev);
        delete ctx;
        return HOTRG_ENOMEM;
    }
    if (workspace_bytes) {
        hotrg_status s = ws_reserve(ctx, workspace_bytes);
        if (s != HOTRG_OK) {
            cudaFree(ctx->status_dev);
            delete ctx;
            return s;
        }
    }
    *out = ctx;
    return HOTRG_OK;
}

void hotrg_destroy(hotrg_ctx* ctx) {
    if (!ctx) return;
    batch_free((Batch*)ctx->batch);
    cudaStreamSynchronize(ctx->stream);
    prof_fold(ctx);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->prof.dflops) cudaFree(ctx->prof.dflops);
    if (ctx->ws.base) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws.base);
    }
    if (ctx->status_dev) cudaFree(ctx->status_dev);
    delete ctx;
}

const char* hotrg_last_error(hotrg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

const char* hotrg_version(void) { return "libhotrg 0.1 (sm_103a)"; }

hotrg_status hotrg_profile_enable(hotrg_ctx* ctx, int32_t enable) {
    if (!ctx) return HOTRG_EINVAL;
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_fold(ctx);
    ctx->prof.on = enable != 0;
    if (ctx->prof.on) {
        hotrg_status s = prof_ensure_dflops(ctx);
        if (s != HOTRG_OK) return s;
        HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->prof.dflops, 0, 128, ctx->stream));
        HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    memset(&ctx->prof.tot, 0, sizeof(ctx->prof.tot));
    ctx->prof.launch_base = g_launches.load();
    return HOTRG_OK;
}

hotrg_status hotrg_profile_read(hotrg_ctx* ctx, hotrg_profile* out) {
    if (!ctx || !out) return HOTRG_EINVAL;
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_fold(ctx);
    *out = ctx->prof.tot;
    out->launches = g_launches.load() - ctx->prof.launch_base;
    return HOTRG_OK;
}

hotrg_status hotrg_init_tensor(hotrg_ctx* ctx, const hotrg_params* p, int32_t kind, double* T_dev,
                               int32_t* labels_dev) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!T_dev || !labels_dev) return set_err(ctx, HOTRG_EINVAL, "null output pointer");
    hotrg_params q = *p;
    if (kind == HOTRG_T_ISING) q.tkind = HOTRG_T_ISING;
    else q.tkind = HOTRG_T_PURE;
    q.prec = HOTRG_FP64;
    hotrg_status s = check_params(ctx, &q);
    if (s != HOTRG_OK) return s;
    if (kind < HOTRG_T_PURE || kind > HOTRG_T_ISING) return set_err(ctx, HOTRG_EINVAL, "unknown tensor kind");
    if ((s = ws_reserve(ctx, 16384)) != HOTRG_OK) return s;
    double* scratch = (double*)ws_alloc(ctx, 8192);
    hotrg_params* dq = (hotrg_params*)ws_alloc(ctx, sizeof(hotrg_params));
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(dq, &q, sizeof(hotrg_params), cudaMemcpyHostToDevice, ctx->stream));
    launch_init_tensor(&q, dq, kind, T_dev, labels_dev, scratch, ctx->stream);
    HOTRG_LAUNCH_CHECK(ctx, "init tensor");
    // the parameter slot is read by the kernels before the call returns to the workspace's next user
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return HOTRG_OK;
}

hotrg_status hotrg_step(hotrg_ctx* ctx, const hotrg_params* p, const double* T_in, const int32_t* q_h,
                        const int32_t* q_v, int32_t Dh, int32_t Dv, double* T_out, int32_t* q_out, int32_t* dprime,
                        hotrg_step_info* info_dev, const double* T_imp_in, double* T_imp_out) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    hotrg_status s = check_params(ctx, p);
    if (s != HOTRG_OK) return s;
    if (!T_in || !q_h || !q_v || !T_out || !q_out || !dprime)
        return set_err(ctx, HOTRG_EINVAL, "null pointer argument");
    if ((T_imp_in == nullptr) != (T_imp_out == nullptr))
        return set_err(ctx, HOTRG_EINVAL, "T_imp_in and T_imp_out must both be set or both be NULL");
    if (Dh < 1 || Dv < 1 || Dh > 128 || Dv > 128) return set_err(ctx, HOTRG_EINVAL, "Dh, Dv must lie in [1, 128]");
    if (T_out == T_in) return set_err(ctx, HOTRG_EINVAL, "T_out aliases T_in");
    const bool imp = T_imp_in != nullptr;
    if ((s = ws_reserve(ctx, step_bytes(p, Dh, Dv, imp, false) + 4096)) != HOTRG_OK) return s;
    int dp = 0;
    s = do_step(ctx, p, T_in, q_h, q_v, Dh, Dv, T_out, q_out, &dp, info_dev, T_imp_in, T_imp_out, nullptr, 0.0, false);
    *dprime = dp;
    if (s == HOTRG_OK) {
        fold_status_kernel<<<1, 32, 0, ctx->stream>>>(info_dev, ctx->status_dev);
        HOTRG_COUNT(1);
        HOTRG_LAUNCH_CHECK(ctx, "fold_status_kernel");
    }
    return s;
}

hotrg_status hotrg_contract(hotrg_ctx* ctx, int32_t prec, int32_t M, int32_t N, int32_t K, const double* A,
                            int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!A || !B || !C) return set_err(ctx, HOTRG_EINVAL, "null pointer argument");
    if (M < 1 || N < 1 || K < 1 || K > 16384 || lda < K || ldb < K || ldc < N)
        return set_err(ctx, HOTRG_EINVAL, "bad sizes or strides");
    if (prec < HOTRG_FP64 || prec > HOTRG_SPLIT_BF16_FAST) return set_err(ctx, HOTRG_EINVAL, "unknown precision form");
    if (prec != HOTRG_FP64 && !ctx->tc_ok) return set_err(ctx, HOTRG_ENOTSUP, "tensor-core forms need sm_103");
    hotrg_status s = ws_reserve(ctx, gemm_engine_workspace(prec, M, N, K) + 4096);
    if (s != HOTRG_OK) return s;
    if (prec == HOTRG_FP64) return gemm_engine(ctx, prec, M, N, K, A, lda, B, ldb, C, ldc, true);
    if ((s = umma_contract(ctx, prec, M, N, K, A, lda, B, ldb, C, ldc)) != HOTRG_OK) return s;
    return umma_check_status(ctx);
}

hotrg_status hotrg_run(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints, int32_t imp_kind,
                       hotrg_result* out) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!params || !out || npoints < 0) return set_err(ctx, HOTRG_EINVAL, "bad arguments");
    if (imp_kind != HOTRG_T_PURE && imp_kind != HOTRG_T_IMP_M && imp_kind != HOTRG_T_IMP_M1)
        return set_err(ctx, HOTRG_EINVAL, "imp_kind must be PURE, IMP_M or IMP_M1");
    hotrg_status first = HOTRG_OK;
    for (int i = 0; i < npoints; ++i) {
        hotrg_status s = run_point(ctx, &params[i], imp_kind, &out[i]);
        if (s != HOTRG_OK && first == HOTRG_OK) first = s;
    }
    return first;
}

hotrg_status hotrg_run_batch(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints, int32_t imp_kind,
                             int32_t nstreams, hotrg_result* out) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!params || !out || npoints < 0) return set_err(ctx, HOTRG_EINVAL, "bad arguments");
    if (nstreams == 0) nstreams = ctx->tuned_streams > 0 ? ctx->tuned_streams : 2;
    if (nstreams < 1 || nstreams > 16) return set_err(ctx, HOTRG_EINVAL, "nstreams must lie in [0, 16]");
    if (imp_kind != HOTRG_T_PURE && imp_kind != HOTRG_T_IMP_M && imp_kind != HOTRG_T_IMP_M1)
        return set_err(ctx, HOTRG_EINVAL, "imp_kind must be PURE, IMP_M or IMP_M1");
    hotrg_status first = HOTRG_OK;
    std::vector<int> valid;
    size_t need = 0;
    for (int i = 0; i < npoints; ++i) {
        memset(&out[i], 0, sizeof(hotrg_result));
        hotrg_status s = check_params(ctx, &params[i]);
        if (s == HOTRG_OK && (imp_kind != HOTRG_T_PURE) && params[i].tkind == HOTRG_T_ISING)
            s = set_err(ctx, HOTRG_EINVAL, "no Ising impurity");
        if (s != HOTRG_OK) {
            out[i].status = s;
            if (first == HOTRG_OK) first = s;
            continue;
        }
        PointPlan pl;
        point_bytes(&params[i], imp_kind, pl);
        need = std::max(need, pl.bytes + 4096);
        valid.push_back(i);
    }
    if (valid.empty()) return first;
    // workers: own non-blocking stream and workspace each
    Batch* B = (Batch*)ctx->batch;
    if (B && (int)B->workers.size() != nstreams) {
        batch_free(B);
        B = nullptr;
        ctx->batch = nullptr;
    }
    if (!B) {
        B = new Batch();
        ctx->batch = B;
        for (int w = 0; w < nstreams; ++w) {
            Worker wk;
            HOTRG_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&wk.stream, cudaStreamNonBlocking));
            wk.ctx = new hotrg_ctx();
            wk.ctx->stream = wk.stream;
            wk.ctx->device = ctx->device;
            wk.ctx->sm_count = ctx->sm_count;
            wk.ctx->smem_optin = ctx->smem_optin;
            wk.ctx->tc_ok = ctx->tc_ok;
            HOTRG_CUDA_TRY(ctx, cudaMalloc(&wk.ctx->status_dev, 64));
            HOTRG_CUDA_TRY(ctx, cudaMemset(wk.ctx->status_dev, 0, 64));
            HOTRG_CUDA_TRY(ctx, cudaEventCreateWithFlags(&wk.done, cudaEventDisableTiming));
            B->workers.push_back(wk);
        }
        HOTRG_CUDA_TRY(ctx, cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
    }
    // fork: every worker stream waits for the context stream's earlier work; with profiling on,
    // points run directly (no graph replay) so that every region is timed on its worker stream
    const bool profiling = ctx->prof.on;
    HOTRG_CUDA_TRY(ctx, cudaEventRecord(B->fork, ctx->stream));
    for (Worker& w : B->workers) {
        w.ctx->prof.on = profiling;
        if (profiling) {
            hotrg_status s = prof_ensure_dflops(w.ctx);
            if (s != HOTRG_OK) return set_err(ctx, s, w.ctx->last_error);
        }
        HOTRG_CUDA_TRY(ctx, cudaStreamWaitEvent(w.stream, B->fork, 0));
    }
    for (Worker& w : B->workers)
        if (w.ctx->tile_n[0] != ctx->tile_n[0] || w.ctx->tile_n[1] != ctx->tile_n[1]) {
            // the captured graphs hold the previous tile shapes' kernels
            for (auto& g : w.graphs) cudaGraphExecDestroy(g.exec);
            w.graphs.clear();
            w.ctx->tile_n[0] = ctx->tile_n[0];
            w.ctx->tile_n[1] = ctx->tile_n[1];
        }
    for (Worker& w : B->workers)
        if (w.ctx->ws.cap < need) {
            for (auto& g : w.graphs) cudaGraphExecDestroy(g.exec);  // their buffers move
            w.graphs.clear();
            hotrg_status s = ws_reserve(w.ctx, need);
            if (s != HOTRG_OK) return set_err(ctx, s, w.ctx->last_error);
        }
    // longest processing time first, each point to the least-loaded worker
    std::vector<double> cost(npoints, 0.0);
    for (int i : valid) cost[i] = point_cost(&params[i]);
    std::sort(valid.begin(), valid.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int>> queue(nstreams);
    std::vector<double> load(nstreams, 0.0);
    for (int i : valid) {
        int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        queue[w].push_back(i);
        load[w] += cost[i];
    }
    // pinned staging: parameters in, scalars out
    hotrg_params* hp = nullptr;
    RunDev* hr = nullptr;
    hotrg_step_info* hi = nullptr;
    HOTRG_CUDA_TRY(ctx, cudaHostAlloc((void**)&hp, sizeof(hotrg_params) * npoints, cudaHostAllocDefault));
    if (cudaHostAlloc((void**)&hr, sizeof(RunDev) * npoints, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&hi, sizeof(hotrg_step_info) * HOTRG_MAX_STEPS * npoints, cudaHostAllocDefault) !=
            cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(hp);
        if (hr) cudaFreeHost(hr);
        return set_err(ctx, HOTRG_ENOMEM, "pinned staging");
    }
    std::vector<PointPlan> plans(npoints);
    hotrg_status err = HOTRG_OK;
    size_t rounds = 0;
    for (auto& q : queue) rounds = std::max(rounds, q.size());
    for (size_t r = 0; r < rounds && err == HOTRG_OK; ++r) {
        for (int w = 0; w < nstreams && err == HOTRG_OK; ++w) {
            if (r >= queue[w].size()) continue;
            const int i = queue[w][r];
            const hotrg_params* p = &params[i];
            Worker& wk = B->workers[w];
            hotrg_ctx* wc = wk.ctx;
            hp[i] = *p;
            const ClassKey key = class_of(p, imp_kind);
            Worker::Graph* g = nullptr;
            for (auto& gg : wk.graphs)
                if (gg.key == key) g = &gg;
            PointPlan& pl = plans[i];
            hotrg_status s;
            if (profiling) {
                if ((s = plan_point(wc, p, imp_kind, pl, need)) != HOTRG_OK) {
                    err = set_err(ctx, s, wc->last_error);
                    break;
                }
                cudaMemcpyAsync(pl.dparams, &hp[i], sizeof(hotrg_params), cudaMemcpyHostToDevice, wk.stream);
                if ((s = enqueue_point(wc, p, imp_kind, pl)) != HOTRG_OK) {
                    err = set_err(ctx, s, wc->last_error);
                    break;
                }
            } else if (!g) {
                // first point of this class on this worker: run it directly, then capture the class's graph
                if ((s = plan_point(wc, p, imp_kind, pl, need)) != HOTRG_OK) {
                    err = set_err(ctx, s, wc->last_error);
                    break;
                }
                cudaMemcpyAsync(pl.dparams, &hp[i], sizeof(hotrg_params), cudaMemcpyHostToDevice, wk.stream);
                if ((s = enqueue_point(wc, p, imp_kind, pl)) != HOTRG_OK) {
                    err = set_err(ctx, s, wc->last_error);
                    break;
                }
                Worker::Graph ng;
                ng.key = key;
                ng.plan = pl;
                PointPlan cap;
                plan_point(wc, p, imp_kind, cap, need);  // same carving as pl
                const long long before = g_launches.load();
                cudaGraph_t graph;
                if (cudaStreamBeginCapture(wk.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    err = set_err(ctx, HOTRG_ECUDA, "cudaStreamBeginCapture failed");
                    break;
                }
                s = enqueue_point(wc, p, imp_kind, cap);
                const cudaError_t ce = cudaStreamEndCapture(wk.stream, &graph);
                if (s != HOTRG_OK || ce != cudaSuccess) {
                    cudaGetLastError();
                    err = set_err(ctx, HOTRG_ECUDA, "graph capture failed: " + wc->last_error);
                    break;
                }
                ng.launches = g_launches.load() - before;
                g_launches.fetch_sub(ng.launches);  // captured, not launched
                if (cudaGraphInstantiate(&ng.exec, graph, 0) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphDestroy(graph);
                    err = set_err(ctx, HOTRG_ECUDA, "cudaGraphInstantiate failed");
                    break;
                }
                cudaGraphDestroy(graph);
                wk.graphs.push_back(ng);
            } else {
                pl = g->plan;
                cudaMemcpyAsync(pl.dparams, &hp[i], sizeof(hotrg_params), cudaMemcpyHostToDevice, wk.stream);
                if (cudaGraphLaunch(g->exec, wk.stream) != cudaSuccess) {
                    cudaGetLastError();
                    err = set_err(ctx, HOTRG_ECUDA, "cudaGraphLaunch failed");
                    break;
                }
                HOTRG_COUNT(g->launches);
            }
            cudaMemcpyAsync(&hr[i], pl.rd, sizeof(RunDev), cudaMemcpyDeviceToHost, wk.stream);
            cudaMemcpyAsync(&hi[(size_t)i * HOTRG_MAX_STEPS], pl.infos, sizeof(hotrg_step_info) * p->n_steps,
                            cudaMemcpyDeviceToHost, wk.stream);
        }
    }
    // join: the context stream waits for every worker (CUDA events recorded on it bracket the batch)
    for (Worker& w : B->workers) {
        cudaEventRecord(w.done, w.stream);
        cudaStreamWaitEvent(ctx->stream, w.done, 0);
    }
    for (Worker& w : B->workers) cudaStreamSynchronize(w.stream);
    if (cudaGetLastError() != cudaSuccess && err == HOTRG_OK) err = set_err(ctx, HOTRG_ECUDA, "batch execution failed");
    if (profiling)
        for (Worker& w : B->workers) {
            prof_fold(w.ctx);
            profile_add(ctx->prof.tot, w.ctx->prof.tot);
            memset(&w.ctx->prof.tot, 0, sizeof(w.ctx->prof.tot));
        }
    for (int i : valid) {
        if (err != HOTRG_OK) {
            out[i].status = err;
            continue;
        }
        memcpy(out[i].step, &hi[(size_t)i * HOTRG_MAX_STEPS], sizeof(hotrg_step_info) * params[i].n_steps);
        hotrg_status s = unpack_point(ctx, &params[i], plans[i], hr[i], &out[i]);
        if (s != HOTRG_OK && first == HOTRG_OK) first = s;
    }
    cudaFreeHost(hp);
    cudaFreeHost(hr);
    cudaFreeHost(hi);
    return err != HOTRG_OK ? err : first;
}

hotrg_status hotrg_observables(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints, double hb,
                               double hbar, double dh, hotrg_obs* out) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!params || !out || npoints < 0 || !(hb > 0) || !(hbar >= 0) || !(dh > 0) || hbar - dh < 0)
        return set_err(ctx, HOTRG_EINVAL, "bad arguments (need hb > 0, dh > 0, hbar >= dh)");
    hotrg_status first = HOTRG_OK;
    for (int i = 0; i < npoints; ++i) {
        hotrg_obs& o = out[i];
        memset(&o, 0, sizeof(o));
        hotrg_params q = params[i];
        q.h = 0.0;
        q.h1 = 0.0;
        hotrg_result r0, rp, rm;
        hotrg_status s = HOTRG_OK;
        auto run1 = [&](hotrg_params pp, int kind, hotrg_result* r) {
            if (s == HOTRG_OK) s = run_point(ctx, &pp, kind, r);
        };
        hotrg_params a = q, b = q;
        a.beta = q.beta + hb;
        b.beta = q.beta - hb;
        run1(q, HOTRG_T_PURE, &r0);
        run1(a, HOTRG_T_PURE, &rp);
        run1(b, HOTRG_T_PURE, &rm);
        if (s == HOTRG_OK) {
            o.lnz = r0.lnz_per_site;
            o.f = -o.lnz / q.beta;
            o.cv = q.beta * q.beta * (rp.lnz_per_site - 2.0 * r0.lnz_per_site + rm.lnz_per_site) / (hb * hb);
        }
        hotrg_result m0, mp, mm;
        hotrg_params f0 = q, fp = q, fm = q;
        f0.h = hbar;
        fp.h = hbar + dh;
        fm.h = hbar - dh;
        run1(f0, HOTRG_T_IMP_M, &m0);
        run1(fp, HOTRG_T_IMP_M, &mp);
        run1(fm, HOTRG_T_IMP_M, &mm);
        if (s == HOTRG_OK) {
            o.m = m0.imp_ratio;
            o.chi = (mp.imp_ratio - mm.imp_ratio) / (2.0 * dh);
        }
        f0 = q;
        fp = q;
        fm = q;
        f0.h1 = hbar;
        fp.h1 = hbar + dh;
        fm.h1 = hbar - dh;
        run1(f0, HOTRG_T_IMP_M1, &m0);
        run1(fp, HOTRG_T_IMP_M1, &mp);
        run1(fm, HOTRG_T_IMP_M1, &mm);
        if (s == HOTRG_OK) {
            o.m1 = m0.imp_ratio;
            o.chi1 = (mp.imp_ratio - mm.imp_ratio) / (2.0 * dh);
        }
        o.status = s;
        if (s != HOTRG_OK && first == HOTRG_OK) first = s;
    }
    return first;
}


hotrg_status hotrg_observables_batch(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints, double hb,
                                     double hbar, double dh, int32_t nstreams, hotrg_obs* out) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!params || !out || npoints < 0 || !(hb > 0) || !(hbar >= 0) || !(dh > 0) || hbar - dh < 0)
        return set_err(ctx, HOTRG_EINVAL, "bad arguments (need hb > 0, dh > 0, hbar >= dh)");
    if (nstreams < 0 || nstreams > 16) return set_err(ctx, HOTRG_EINVAL, "nstreams must lie in [0, 16]");
    for (int i = 0; i < npoints; ++i) memset(&out[i], 0, sizeof(hotrg_obs));
    if (npoints == 0) return HOTRG_OK;
    // three families (beta +-hb pure; h = hbar +-dh with the M impurity; h1 = hbar +-dh with the M1
    // impurity), three runs per point each, in the order (centre, +, -) of hotrg_observables
    std::vector<hotrg_params> pp((size_t)3 * npoints);
    std::vector<hotrg_result> rr((size_t)3 * npoints);
    const int kinds[3] = {HOTRG_T_PURE, HOTRG_T_IMP_M, HOTRG_T_IMP_M1};
    hotrg_status fatal = HOTRG_OK;
    std::string fatal_msg;
    for (int f = 0; f < 3; ++f) {
        for (int i = 0; i < npoints; ++i) {
            hotrg_params q = params[i];
            q.h = 0.0;
            q.h1 = 0.0;
            for (int j = 0; j < 3; ++j) {
                hotrg_params a = q;
                if (f == 0) a.beta = j == 0 ? q.beta : (j == 1 ? q.beta + hb : q.beta - hb);
                if (f == 1) a.h = j == 0 ? hbar : (j == 1 ? hbar + dh : hbar - dh);
                if (f == 2) a.h1 = j == 0 ? hbar : (j == 1 ? hbar + dh : hbar - dh);
                pp[(size_t)3 * i + j] = a;
            }
        }
        const hotrg_status s = hotrg_run_batch(ctx, pp.data(), 3 * npoints, kinds[f], nstreams, rr.data());
        (void)s;  // per-run statuses are in rr
        for (int i = 0; i < npoints; ++i) {
            hotrg_obs& o = out[i];
            const hotrg_result* r = &rr[(size_t)3 * i];
            hotrg_status ps = HOTRG_OK;
            for (int j = 0; j < 3 && ps == HOTRG_OK; ++j) ps = (hotrg_status)r[j].status;
            if (ps != HOTRG_OK) {
                if (o.status == HOTRG_OK) o.status = ps;
                if (fatal == HOTRG_OK) {
                    fatal = ps;
                    fatal_msg = ctx->last_error;
                }
                continue;
            }
            if (o.status != HOTRG_OK) continue;
            if (f == 0) {
                o.lnz = r[0].lnz_per_site;
                o.f = -o.lnz / params[i].beta;
                o.cv = params[i].beta * params[i].beta *
                       (r[1].lnz_per_site - 2.0 * r[0].lnz_per_site + r[2].lnz_per_site) / (hb * hb);
            } else if (f == 1) {
                o.m = r[0].imp_ratio;
                o.chi = (r[1].imp_ratio - r[2].imp_ratio) / (2.0 * dh);
            } else {
                o.m1 = r[0].imp_ratio;
                o.chi1 = (r[1].imp_ratio - r[2].imp_ratio) / (2.0 * dh);
            }
        }
    }
    if (fatal != HOTRG_OK) ctx->last_error = fatal_msg;
    return fatal;
}


hotrg_status hotrg_autotune_batch(hotrg_ctx* ctx, const hotrg_params* sample, int32_t npoints, int32_t max_streams,
                                  int32_t* best, double* seconds) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!sample || npoints < 1 || max_streams < 1 || max_streams > 16)
        return set_err(ctx, HOTRG_EINVAL, "need npoints >= 1 and max_streams in [1, 16]");
    std::vector<hotrg_result> res((size_t)npoints);
    double tbest = 0.0;
    int kbest = 0;
    for (int k = 1; k <= max_streams; ++k) {
        // one untimed pass builds the workers' workspaces and graphs, the second is timed
        hotrg_status s = hotrg_run_batch(ctx, sample, npoints, HOTRG_T_PURE, k, res.data());
        if (s != HOTRG_OK) return s;
        const auto t0 = std::chrono::steady_clock::now();
        s = hotrg_run_batch(ctx, sample, npoints, HOTRG_T_PURE, k, res.data());
        if (s != HOTRG_OK) return s;
        const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (seconds) seconds[k - 1] = t;
        if (kbest == 0 || t < tbest) {
            tbest = t;
            kbest = k;
        }
    }
    ctx->tuned_streams = kbest;
    if (best) *best = kbest;
    return HOTRG_OK;
}

hotrg_status hotrg_set_tiles(hotrg_ctx* ctx, int32_t env_tile_n, int32_t coarse_tile_n) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if ((env_tile_n != 64 && env_tile_n != 128) || (coarse_tile_n != 64 && coarse_tile_n != 128))
        return set_err(ctx, HOTRG_EINVAL, "tile widths must be 64 or 128");
    ctx->tile_n[0] = env_tile_n;
    ctx->tile_n[1] = coarse_tile_n;
    return HOTRG_OK;
}

hotrg_status hotrg_autotune_tiles(hotrg_ctx* ctx, const hotrg_params* sample, int32_t npoints, int32_t nstreams,
                                  int32_t* env_tile_n, int32_t* coarse_tile_n, double* seconds) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    if (!sample || npoints < 1 || nstreams < 0 || nstreams > 16)
        return set_err(ctx, HOTRG_EINVAL, "need npoints >= 1 and nstreams in [0, 16]");
    const int widths[2] = {128, 64};
    std::vector<hotrg_result> res((size_t)npoints);
    double tbest = 0.0;
    int ebest = 128, cbest = 128, k = 0;
    for (int e : widths)
        for (int c : widths) {
            ctx->tile_n[0] = e;
            ctx->tile_n[1] = c;
            // untimed: the workers rebuild their graphs for the new shapes; then timed
            hotrg_status s = hotrg_run_batch(ctx, sample, npoints, HOTRG_T_PURE, nstreams, res.data());
            if (s != HOTRG_OK) return s;
            const auto t0 = std::chrono::steady_clock::now();
            s = hotrg_run_batch(ctx, sample, npoints, HOTRG_T_PURE, nstreams, res.data());
            if (s != HOTRG_OK) return s;
            const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (seconds) seconds[k] = t;
            ++k;
            if (k == 1 || t < tbest) {
                tbest = t;
                ebest = e;
                cbest = c;
            }
        }
    ctx->tile_n[0] = ebest;
    ctx->tile_n[1] = cbest;
    if (env_tile_n) *env_tile_n = ebest;
    if (coarse_tile_n) *coarse_tile_n = cbest;
    return HOTRG_OK;
}

}  // extern "C"
