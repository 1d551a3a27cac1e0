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
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace hotrg {

std::atomic<long long> g_launches{0};

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

hotrg_status prof_fold(hotrg_ctx* ctx) {
    Profiler& P = ctx->prof;
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
    return HOTRG_OK;
}

static int d0_of(const hotrg_params* p) { return p->tkind == HOTRG_T_ISING ? 2 : 2 * p->n_max + 1; }

// Workspace bytes of one step with the given sizes (everything except T in/out).
static size_t step_bytes(const hotrg_params* p, int Dh, int Dv, bool imp) {
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
    const int64_t shapes[5][3] = {{(int64_t)hv, (int64_t)hv, (int64_t)hv},
                                  {(int64_t)n, (int64_t)n, (int64_t)Dv * Dv},
                                  {(int64_t)Dp * Dh, (int64_t)Dh * Dv * Dv, Dh},
                                  {(int64_t)Dp * Dh * Dv, (int64_t)hv, (int64_t)hv},
                                  {(int64_t)Dp * Dv * Dv, (int64_t)Dp, (int64_t)n}};
    size_t g = 0;
    for (auto& sh : shapes) g = std::max(g, gemm_engine_workspace(p->prec, sh[0], sh[1], sh[2]));
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
static hotrg_status coarse(hotrg_ctx* ctx, int prec, const double* P, int Dh, int Dv, int Dp,
                           const double* T_up, const double* T_dn, double* Pt, double* Pt2, double* Tt,
                           double* Tb, double* W, double* W2, double* Tc, double* T_out) {
    const int64_t hh = (int64_t)Dh * Dh, vv = (int64_t)Dv * Dv;
    hotrg_status s;
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
static hotrg_status do_step(hotrg_ctx* ctx, const hotrg_params* p, const double* T_in, const int32_t* q_h,
                            const int32_t* q_v, int Dh, int Dv, double* T_out, int32_t* q_out, int* dprime,
                            hotrg_step_info* info, const double* Ti_in, double* Ti_out, double* lnz_acc,
                            double weight) {
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
    if (!X1 || !X2 || !Am || !Bm || !A2 || !B2 || !Ep || !EL || !ER || !eigws || !P || !Pt || !Pt2 || !Tt ||
        !Tb || !W || !W2 || !Tc || (Ti_in && !Ti2) || !partial || !norm)
        return set_err(ctx, HOTRG_ENOMEM, "step workspace exhausted");
    hotrg_status s;
    const int h_step = prof_begin(ctx);
    if ((s = environment(ctx, prec, T_in, Dh, Dv, false, X1, X2, Am, Bm, A2, B2, Ep, EL)) != HOTRG_OK) return s;
    if (p->env_policy == 0)
        if ((s = environment(ctx, prec, T_in, Dh, Dv, true, X1, X2, Am, Bm, A2, B2, Ep, ER)) != HOTRG_OK) return s;
    EigPlan plan;
    plan.n = (int)n;
    plan.Dh = Dh;
    plan.dprime = Dp;
    plan.sym = sym_of(p);
    plan.max_sweeps = p->eig_max_sweeps > 0 ? p->eig_max_sweeps : 40;
    plan.tol = p->eig_tol > 0 ? p->eig_tol : 1e-15;
    plan.tie_rtol = p->tie_rtol > 0 ? p->tie_rtol : 1e-12;
    plan.env_policy = p->env_policy;
    plan.exact = prec == HOTRG_FP64;
    const int h_eig = prof_begin(ctx);
    if ((s = eig_truncate(ctx, plan, EL, p->env_policy == 0 ? ER : nullptr, q_h, P, q_out, info, eigws)) !=
        HOTRG_OK)
        return s;
    prof_end(ctx, h_eig, PROF_EIG, 0.0);
    if ((s = coarse(ctx, prec, P, Dh, Dv, Dp, T_in, T_in, Pt, Pt2, Tt, Tb, W, W2, Tc, T_out)) != HOTRG_OK)
        return s;
    launch_norm(T_out, tn, partial, norm, ctx->stream);
    if (Ti_in) {
        // T_imp' = [P^T (T_imp above T) P + P^T (T above T_imp) P] / (2 c_k)
        if ((s = coarse(ctx, prec, P, Dh, Dv, Dp, Ti_in, T_in, Pt, Pt2, Tt, Tb, W, W2, Tc, Ti_out)) != HOTRG_OK)
            return s;
        if ((s = coarse(ctx, prec, P, Dh, Dv, Dp, T_in, Ti_in, Pt, Pt2, Tt, Tb, W, W2, Tc, Ti2)) != HOTRG_OK)
            return s;
        launch_axpby(Ti_out, Ti2, 0.5, 0.5, tn, ctx->stream);
        launch_scale_inv(Ti_out, tn, norm, ctx->stream);
    }
    launch_scale_inv(T_out, tn, norm, ctx->stream);
    launch_step_scalars(norm, info, lnz_acc, weight, ctx->stream);
    HOTRG_LAUNCH_CHECK(ctx, "step");
    prof_end(ctx, h_step, PROF_STEP, 0.0);
    return HOTRG_OK;
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
};

static hotrg_status run_point(hotrg_ctx* ctx, const hotrg_params* p, int imp_kind, hotrg_result* out) {
    memset(out, 0, sizeof(*out));
    hotrg_status s = check_params(ctx, p);
    if (s != HOTRG_OK) { out->status = s; return (hotrg_status)out->status; }
    const int D0 = d0_of(p);
    const bool imp = imp_kind == HOTRG_T_IMP_M || imp_kind == HOTRG_T_IMP_M1;
    if (imp && p->tkind == HOTRG_T_ISING) { out->status = set_err(ctx, HOTRG_EINVAL, "no Ising impurity"); return (hotrg_status)out->status; }
    std::vector<int> dh, dv;
    step_sizes(p, D0, dh, dv);
    size_t tmax = (size_t)D0 * D0 * D0 * D0, smax = 0;
    for (size_t k = 0; k < dh.size(); ++k) {
        const size_t Dp = std::min<size_t>(p->d_cut, (size_t)dh[k] * dh[k]);
        tmax = std::max(tmax, Dp * Dp * dv[k] * dv[k]);
        smax = std::max(smax, step_bytes(p, dh[k], dv[k], imp));
    }
    const int qmax = std::max(D0, p->d_cut) + 1;
    const size_t fixed = a256(tmax * 8) * (imp ? 4 : 2) + a256(qmax * 4) * 3 + a256(16384) +
                         a256(sizeof(hotrg_step_info) * HOTRG_MAX_STEPS) + a256(sizeof(RunDev)) + a256(8192);
    if ((s = ws_reserve(ctx, fixed + smax)) != HOTRG_OK) { out->status = s; return (hotrg_status)out->status; }
    double* Ta = (double*)ws_alloc(ctx, tmax * 8);
    double* Tb = (double*)ws_alloc(ctx, tmax * 8);
    double* Ia = imp ? (double*)ws_alloc(ctx, tmax * 8) : nullptr;
    double* Ib = imp ? (double*)ws_alloc(ctx, tmax * 8) : nullptr;
    int32_t* qa = (int32_t*)ws_alloc(ctx, qmax * 4);
    int32_t* qb = (int32_t*)ws_alloc(ctx, qmax * 4);
    double* scratch = (double*)ws_alloc(ctx, 16384);  // coefficient scratch: 2 x 1024 doubles
    hotrg_step_info* infos = (hotrg_step_info*)ws_alloc(ctx, sizeof(hotrg_step_info) * HOTRG_MAX_STEPS);
    RunDev* rd = (RunDev*)ws_alloc(ctx, sizeof(RunDev));
    double* partial = (double*)ws_alloc(ctx, 4096 * 2);
    const size_t step_base = ctx->ws.used;
    cudaStream_t st = ctx->stream;
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(rd, 0, sizeof(RunDev), st));
    HOTRG_CUDA_TRY(ctx, cudaMemsetAsync(infos, 0, sizeof(hotrg_step_info) * HOTRG_MAX_STEPS, st));
    launch_init_tensor(p, p->tkind, Ta, qa, scratch, st);
    if (imp) {
        int32_t* qdummy = qb;
        launch_init_tensor(p, imp_kind, Ia, qdummy, scratch + 1024, st);
    }
    HOTRG_LAUNCH_CHECK(ctx, "init tensor");
    // c_0 = ||T0||_F; T <- T / c_0 (impurity scaled by the same c_0)
    const int64_t n0 = (int64_t)D0 * D0 * D0 * D0;
    launch_norm(Ta, n0, partial, &rd->norm0, st);
    launch_scale_inv(Ta, n0, &rd->norm0, st);
    if (imp) launch_scale_inv(Ia, n0, &rd->norm0, st);
    log_kernel<<<1, 32, 0, st>>>(&rd->ln_c0, &rd->norm0);
    log_kernel<<<1, 32, 0, st>>>(&rd->lnz, &rd->norm0);
    HOTRG_COUNT(2);
    // labels: both legs start with the same labels
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(qb, qa, D0 * 4, cudaMemcpyDeviceToDevice, st));
    int32_t* qh = qa;
    int32_t* qv = qb;
    int32_t* qspare = (int32_t*)ws_alloc(ctx, qmax * 4);
    if (!qspare) { out->status = set_err(ctx, HOTRG_ENOMEM, "label buffer"); return (hotrg_status)out->status; }
    const size_t step_base2 = ctx->ws.used;
    (void)step_base;
    double* Tcur = Ta;
    double* Tnext = Tb;
    double* Icur = Ia;
    double* Inext = Ib;
    for (int k = 0; k < p->n_steps; ++k) {
        ctx->ws.used = step_base2;
        int dp = 0;
        s = do_step(ctx, p, Tcur, qh, qv, dh[k], dv[k], Tnext, qspare, &dp, &infos[k], Icur, Inext, &rd->lnz,
                    ldexp(1.0, -(k + 1)));
        if (s != HOTRG_OK) { out->status = s; return (hotrg_status)out->status; }
        // new horizontal labels = old vertical labels; new vertical = q_out
        int32_t* old_h = qh;
        qh = qv;
        qv = qspare;
        qspare = old_h;
        std::swap(Tcur, Tnext);
        std::swap(Icur, Inext);
    }
    const int Dx = p->n_steps == 0 ? D0 : (int)std::min<long>(p->d_cut, (long)dh.back() * dh.back());
    const int Dy = p->n_steps == 0 ? D0 : dv.back();
    // the final tensor is [Dy][Dy][Dx][Dx] after relabelling (l,r legs = old vertical)
    launch_trace(Tcur, Dy, Dx, &rd->tr, st);
    if (imp) launch_trace(Icur, Dy, Dx, &rd->tr_imp, st);
    finish_kernel<<<1, 32, 0, st>>>(&rd->lnz, &rd->tr, ldexp(1.0, -p->n_steps), &rd->ln_tr,
                                    imp ? &rd->tr_imp : nullptr, &rd->imp_ratio);
    HOTRG_COUNT(1);
    HOTRG_LAUNCH_CHECK(ctx, "finish");
    RunDev h;
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, rd, sizeof(RunDev), cudaMemcpyDeviceToHost, st));
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(out->step, infos, sizeof(hotrg_step_info) * p->n_steps,
                                        cudaMemcpyDeviceToHost, st));
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    prof_fold(ctx);
    if (p->prec != HOTRG_FP64)
        if ((s = umma_check_status(ctx)) != HOTRG_OK) { out->status = s; return s; }
    out->lnz_per_site = h.lnz;
    out->ln_c0 = h.ln_c0;
    out->ln_trace = h.ln_tr;
    out->imp_ratio = imp ? h.imp_ratio : 0.0;
    out->n_steps = p->n_steps;
    out->status = HOTRG_OK;
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
    if (workspace_bytes) {
        hotrg_status s = ws_reserve(ctx, workspace_bytes);
        if (s != HOTRG_OK) {
            delete ctx;
            return s;
        }
    }
    *out = ctx;
    return HOTRG_OK;
}

void hotrg_destroy(hotrg_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    prof_fold(ctx);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->ws.base) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws.base);
    }
    delete ctx;
}

const char* hotrg_last_error(hotrg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

const char* hotrg_version(void) { return "libhotrg 0.1 (sm_103a)"; }

hotrg_status hotrg_profile_enable(hotrg_ctx* ctx, int32_t enable) {
    if (!ctx) return HOTRG_EINVAL;
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_fold(ctx);
    ctx->prof.on = enable != 0;
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
    launch_init_tensor(&q, kind, T_dev, labels_dev, scratch, ctx->stream);
    HOTRG_LAUNCH_CHECK(ctx, "init tensor");
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
    if ((s = ws_reserve(ctx, step_bytes(p, Dh, Dv, imp) + 4096)) != HOTRG_OK) return s;
    int dp = 0;
    s = do_step(ctx, p, T_in, q_h, q_v, Dh, Dv, T_out, q_out, &dp, info_dev, T_imp_in, T_imp_out, nullptr, 0.0);
    *dprime = dp;
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

}  // extern "C"
