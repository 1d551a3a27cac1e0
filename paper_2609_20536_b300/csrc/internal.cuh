// Internal declarations of libhotrg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hotrg.h"

namespace hotrg {

// kernels launched by the library (all contexts)
extern std::atomic<long long> g_launches;
#define HOTRG_COUNT(n) (::hotrg::g_launches.fetch_add((n), std::memory_order_relaxed))

// profiling classes
enum ProfClass : int { PROF_GEMM_ENV = 0, PROF_GEMM_COARSE = 1, PROF_GEMM_OTHER = 2, PROF_SLICE = 3, PROF_EIG = 4,
                       PROF_STEP = 5, PROF_EIG_PART0 = 6 /* .. 9 */ };

struct ProfMark {
    cudaEvent_t a, b;
    int cls;
    double flops;
};

struct Profiler {
    bool on = false;
    // device, 16 doubles: per GEMM class c the block planner adds the algorithmic flops at [c],
    // the operand elements at [3 + c] and the output elements at [6 + c]
    double* dflops = nullptr;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfMark> pending;
    hotrg_profile tot{};
    long long launch_base = 0;
};

// Symmetry of the fused-leg labels: U(1) charge, Z2 parity, or none.
enum SymMode : int { SYM_U1 = 0, SYM_Z2 = 1, SYM_NONE = 2 };

struct Workspace {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    bool owned_growth_ok = true;
};

}  // namespace hotrg

struct hotrg_ctx {
    cudaStream_t stream = nullptr;
    hotrg::Workspace ws;
    std::string last_error;
    int device = 0;
    int sm_count = 148;
    int smem_optin = 0;
    bool tc_ok = false;  // sm_103a tensor-core path usable on this device
    hotrg::Profiler prof;
    void* batch = nullptr;  // worker streams and graph cache of hotrg_run_batch
    int tuned_streams = 0;  // hotrg_autotune_batch's choice (0: not tuned, batch calls default to 2)
    // Engine status words (bounded waits that ran out, planner overflow): status_dev is this
    // context's own (64 bytes on ctx->device, made with the context); while a point is enqueued
    // status_slot points at that point's slot in its device result block, so that a failure is
    // reported for that point alone (also inside captured graphs).
    int32_t* status_dev = nullptr;
    int32_t* status_slot = nullptr;
    // tile width (output columns per tile, 128 or 64) of the split forms' grouped products,
    // [0] environments, [1] coarse contraction; set by hotrg_set_tiles / hotrg_autotune_tiles
    int tile_n[2] = {128, 128};
};

namespace hotrg {

// ---- error helpers -------------------------------------------------------
hotrg_status set_err(hotrg_ctx* ctx, hotrg_status st, const std::string& msg);

// Kernel attributes (cudaFuncSetAttribute) belong to one device: true the first time
// a (kernel, device) pair is seen, so that the caller sets them once per device.
bool attr_once(const void* kernel, int device);

#define HOTRG_CUDA_TRY(ctx, call)                                                           \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess)                                                              \
            return ::hotrg::set_err((ctx), HOTRG_ECUDA,                                     \
                                    std::string(#call) + ": " + cudaGetErrorString(_e));    \
    } while (0)

#define HOTRG_LAUNCH_CHECK(ctx, what)                                                       \
    do {                                                                                    \
        cudaError_t _e = cudaGetLastError();                                                \
        if (_e != cudaSuccess)                                                              \
            return ::hotrg::set_err((ctx), HOTRG_ECUDA,                                     \
                                    std::string("launch ") + (what) + ": " +                \
                                        cudaGetErrorString(_e));                            \
    } while (0)

// ---- profiling: bracket a region with prof_begin / prof_end on ctx->stream --
int prof_begin(hotrg_ctx* ctx);  // returns a handle (-1 when profiling is off)
void prof_end(hotrg_ctx* ctx, int handle, int cls, double flops);
hotrg_status prof_fold(hotrg_ctx* ctx);  // after a stream sync: accumulate finished marks

// ---- workspace (bump allocator, 256-byte aligned) -------------------------
hotrg_status ws_reserve(hotrg_ctx* ctx, size_t bytes);
void* ws_alloc(hotrg_ctx* ctx, size_t bytes);  // returns nullptr when over capacity

// ---- kernels: elementwise / tensor plumbing (hotrg_kernels.cu) ------------
// Output-ordered permutation: out is contiguous with dims od[0..nd) (od[nd-1]
// fastest); element (o_0..o_{nd-1}) is read from in[sum o_k * is[k]].
void launch_permute(const double* in, double* out, int nd, const int64_t* od, const int64_t* is,
                    cudaStream_t st);
// C[b](M x N, ldc) = A[b](M x K, lda) * B[b](N x K, ldb)^T in FP64 (SIMT DFMA).
void launch_gemm_tn_f64(int M, int N, int K, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double* C, int64_t ldc, int batch, int64_t sA, int64_t sB,
                        int64_t sC, cudaStream_t st);
// Frobenius norm of x[0..n) into *norm (two-pass, deterministic); partial is a
// scratch array of at least norm_partials() doubles.
int norm_partials();
void launch_norm(const double* x, int64_t n, double* partial, double* norm, cudaStream_t st);
// x[i] *= 1 / *c  (c on the device)
void launch_scale_inv(double* x, int64_t n, const double* c, cudaStream_t st);
// *tr = sum_{x,y} T[x][x][y][y] for T [Dx][Dx][Dy][Dy]
void launch_trace(const double* T, int Dx, int Dy, double* tr, cudaStream_t st);
// Initial tensor (Eq. 3.4, 3.15, 3.20, 3.21) or the Ising tensor.  Sizes and the
// symmetry come from the host copy p; beta, Delta, h, h1 are read on the
// device from dp (so a captured graph can be replayed with new values).
void launch_init_tensor(const hotrg_params* p, const hotrg_params* dp, int kind, double* T, int32_t* labels,
                        double* scratch, cudaStream_t st);
// Step bookkeeping: info->ln_c = log(*norm), lnz accumulation etc.
void launch_step_scalars(const double* norm, hotrg_step_info* info, double* lnz_acc, double weight,
                         cudaStream_t st);
void launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st);

// ---- eigensolver + truncation (hotrg_eig.cu) -------------------------------
struct EigPlan {
    int n;        // Dh^2 states
    int Dh;
    int dprime;
    int sym;      // SymMode
    int max_sweeps;
    double tol;
    double tie_rtol;
    double side_rtol;
    int env_policy;
    bool exact;      // FP64 Jacobi on every block
    int fp64_iters;  // FP64 subspace iterations after the first Rayleigh-Ritz step (subspace path)
};
size_t eig_workspace_bytes(int Dh);
// E[0] = E_L, E[1] = E_R (E[1] may be null when env_policy == 1).  Writes P
// ((Dh^2) x D' row-major), q_out (D'), and info->{eps_left, eps_right, side,
// sweeps, status}.
hotrg_status eig_truncate(hotrg_ctx* ctx, const EigPlan& plan, const double* EL, const double* ER,
                          const int32_t* q_h, double* P, int32_t* q_out, hotrg_step_info* info,
                          void* ws);

// ---- contraction engines (FP64 SIMT; tensor-core split forms) -------------
// C (M x N, ldc) = A (M x K, lda) * B (N x K, ldb)^T with FP64 in/out.
hotrg_status gemm_engine(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda,
                         const double* B, int64_t ldb, double* C, int64_t ldc, bool coarse);
size_t gemm_engine_workspace(int prec, int64_t M, int64_t N, int64_t K);
hotrg_status umma_contract(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda,
                           const double* B, int64_t ldb, double* C, int64_t ldc);
hotrg_status umma_check_status(hotrg_ctx* ctx);
// Split-form contraction reading A and B through gather maps
// {rd1, rd2, rs0, rs1, rs2, kd, ks0, ks1}: element (r, k) sits at
// (r/(rd1 rd2)) rs0 + ((r/rd2) % rd1) rs1 + (r % rd2) rs2 + (k/kd) ks0 + (k % kd) ks1.
hotrg_status umma_contract_gather(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, const int64_t* am,
                                  const double* B, const int64_t* bm, double* C, int64_t ldc, bool coarse);
int32_t* umma_status_word(hotrg_ctx* ctx);

// ---- block-sparse contractions (hotrg_blocks.cu, hotrg_umma.cu) -----------
constexpr int BS_V = 128;       // charge values tracked per index set
constexpr int BS_VOFF = 64;     // value v is stored at slot v - centre + BS_VOFF (centre: bs_centre_kernel)
constexpr int BS_CHUNK = 256;   // elements per warp in the counting passes

// One leg of an index set: its label array, extent, sign in the set's value,
// and its element strides in the two tensors that use the set; st2 is the leg's
// stride in the index of a pair table (the output's value-sorted pair layout).
struct BsFactor {
    const int32_t* lab;
    int64_t ext;
    int sgn;
    int64_t st0, st1;
    int64_t st2;
};
// An index set of up to three legs, factor 0 the most significant digit.  With
// pi0 set, the first offset is a pair table entry: o0 = pi0[sum_f i_f st0_f].
struct BsSet {
    int nf;
    BsFactor f[3];
    int64_t size;
    const int32_t* pi0;
};
struct BsGroup {  // one charge block of a grouped contraction
    int64_t mbase, kbase, nbase;  // first positions in the sorted M / K / N lists
    int64_t mpad, npad;           // first padded slice rows of the group's A / B rows
    int32_t M, K, N, Kp;
    int32_t tiles_n, tile_base;
};
struct BsHeader {
    int32_t G, total_tiles;
    int64_t mpad_total, npad_total;
    double flops;  // sum over groups of 2 M K N
};
struct BsPlan {  // device pointers (workspace) plus the host-known set sizes
    BsGroup* groups;
    BsHeader* hdr;
    int64_t *offM0, *offM1;  // M set: offsets in A, in C
    int64_t *offK0, *offK1;  // K set: offsets in A, in B
    int64_t *offN0, *offN1;  // N set: offsets in B, in C
    // Output in a pair layout (pi_out set): element (m, n) goes to
    // C[offM1[m] + offN1[n] + pi_out[offM2[m] + offN2[n]]].
    const int32_t* pi_out;
    int32_t *offM2, *offN2;
    // The K set reads A through a pair table: each group's A-side K offsets are then
    // consecutive (the table ranks the pairs of one value in the order the planner
    // lists them), so a row's elements are one contiguous run.
    int32_t kA_contig;
    int64_t nM, nK, nN;
    int32_t kp_cap;  // slice row pitch (>= every block's padded K; checked on the device)
    int32_t tile_n;  // output columns per tile of the tile table (128, or 64 for the split forms)
};
size_t bs_plan_bytes(int64_t nM, int64_t nK, int64_t nN);
// Enqueues the planner for C = A B^T over index sets (M, K, N) with the given
// symmetry; the value table (BS_V slots) is centred on the product's range of
// label sums, and a product whose sums span BS_V or more values records
// HOTRG_ENOTSUP in the engine's status word.
// kp_cap_override > 0 replaces the slice pitch limit (the FP64 engine slices nothing).
// tile_n: output columns per tile of the tile table (rows are always 128).
// pi_out: the output's pair table (null: the output offset is offM1 + offN1).
hotrg_status bs_plan(hotrg_ctx* ctx, int sym, const BsSet& M, const BsSet& K, const BsSet& N, int prof_class,
                     BsPlan& out, int32_t kp_cap_override = 0, int tile_n = 128, const int32_t* pi_out = nullptr);
// Pair table of two legs a (labels qa, extent na) and b (qb, nb): pi[a nb + b] = the rank of
// the pair (a, b) in the order of (value, a, b), value = qa[a] + qb[b] (its parity for Z2).
// Pairs of one value then occupy one contiguous range, in the order the planner lists them.
hotrg_status pair_table(hotrg_ctx* ctx, int sym, const int32_t* qa, int na, const int32_t* qb, int nb, int32_t* pi);
// Slice row pitch of a grouped product: the whole K set rounded to 32 for small sets and
// Z2; half of it (at least 4096) for larger U(1) sets (bs_plan checks every block on the device).
int32_t bs_pitch(int64_t nK, int sym);
size_t umma_grouped_workspace(int64_t nM, int64_t nK, int64_t nN, int sym);
// Operand / output formats: 0 = FP64, 1 = exact FP32 pairs (hi, lo) with value hi + lo.
hotrg_status umma_grouped(hotrg_ctx* ctx, int prec, const BsPlan& pl, const void* A, int afmt, const void* B,
                          int bfmt, void* C, int cfmt, int prof_class);
// The same grouped product in plain FP64 (SIMT FMA; FP64 operands and output only).
hotrg_status dgemm_grouped(hotrg_ctx* ctx, const BsPlan& pl, const void* A, int afmt, const void* B, int bfmt,
                           void* C, int cfmt, int prof_class);
// Grouped product through the engine of the precision form.
hotrg_status grouped_engine(hotrg_ctx* ctx, int prec, const BsPlan& pl, const void* A, int afmt, const void* B,
                            int bfmt, void* C, int cfmt, int prof_class);

}  // namespace hotrg
