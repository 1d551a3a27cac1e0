/*
 * hotrg.h -- C ABI of libhotrg: HOTRG coarse-graining of the 2D generalized
 * XY model (q = 2) on one NVIDIA B300 (sm_103a).
 *
 * The method is the higher-order tensor renormalization group of the thesis
 * "Numerical Investigations of Phase Transitions in Lattice Field Theories",
 * §2.4.1 (Eq. 2.11 fuse, Eq. 2.12 HOSVD, the eps_1/eps_2 rule and Eq. 2.15
 * projector, Eq. 2.16 coarse tensor), applied to the character-expanded
 * generalized XY tensor of §3.2-§3.3 (Eq. 3.4 coefficients a_n, Eq. 3.6 /
 * 3.15 site tensor) with the impurity tensors of §3.4 (Eq. 3.20, 3.21).
 *
 * Conventions common to every entry point
 *   - Every call returns a hotrg_status and never aborts, traps or throws.
 *     On a status other than HOTRG_OK the outputs are undefined and
 *     hotrg_last_error(ctx) returns a one-line description.
 *   - Tensors are row-major FP64 with legs [l][r][u][d] (left, right, up,
 *     down; d fastest).  Bond-state labels are int32: the U(1) charge
 *     n = i - n_max at zero field, the charge parity with h1 only (h = 0),
 *     0 when h != 0 (no block structure).
 *   - Pointers documented as "device" are caller-owned device memory
 *     (cudaMalloc or a framework allocator); "host" pointers are ordinary
 *     host memory.  The library owns only the workspace inside hotrg_ctx.
 *   - All device work is enqueued on the stream given to hotrg_create.
 *     hotrg_init_tensor and hotrg_step are asynchronous with respect to the
 *     host except for the error checks noted; hotrg_run and
 *     hotrg_observables return after their host outputs are written.
 *   - One hotrg_ctx per host thread; a context is not thread-safe.
 *   - Precision forms: HOTRG_FP64 computes every contraction with FP64
 *     fused multiply-adds.  HOTRG_SPLIT_BF16 computes the environment and
 *     coarse contractions on the tensor cores from fixed-point BF16 slices
 *     of the FP64 operands: per-row power-of-two scaling, balanced 8-bit
 *     digits, 5 slices (39 bits, 15 slice products) for the coarse
 *     contraction and 4 slices (31 bits, 10 products) for the environments.
 *     Slice products accumulate exactly in FP32 over chunks of 512 and are
 *     carried across chunks in double-float registers.  The environment
 *     eigensolve (FP32 subspace iteration refined by an FP64 Rayleigh-Ritz
 *     step on large blocks, FP64 Jacobi on small ones), normalisation and
 *     ln Z stay FP64.  HOTRG_SPLIT_BF16_FAST uses 3 slices everywhere (23
 *     bits, the FP32 accuracy class of a 3xTF32 split).
 */
#ifndef HOTRG_H
#define HOTRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HOTRG_MAX_STEPS 64

typedef struct hotrg_ctx hotrg_ctx; /* opaque; owns device workspace */

typedef enum {
    HOTRG_OK = 0,
    HOTRG_EINVAL = -1,   /* invalid argument (sizes, parameters, null pointer) */
    HOTRG_ENOMEM = -2,   /* device or host allocation failed */
    HOTRG_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    HOTRG_ENOCONV = -4,  /* eigensolver (sweep cap) or zero-field fit did not converge */
    HOTRG_ETIMEOUT = -5, /* a bounded device wait ran out */
    HOTRG_ENOTSUP = -6   /* form not available in this build / on this device, or block labels too wide */
} hotrg_status;

typedef enum { HOTRG_FP64 = 0, HOTRG_SPLIT_BF16 = 1, HOTRG_SPLIT_BF16_FAST = 2 } hotrg_prec;

typedef enum {
    HOTRG_T_PURE = 0,   /* Eq. 3.15: sqrt(a_l a_r a_u a_d) * sum_j I_{Q+2j}(bh) I_j(bh1) */
    HOTRG_T_IMP_M = 1,  /* Eq. 3.20: cos(theta) impurity */
    HOTRG_T_IMP_M1 = 2, /* Eq. 3.21: cos(2 theta) impurity */
    HOTRG_T_ISING = 3   /* 2D Ising tensor (bond dimension 2), a test model */
} hotrg_tkind;

/* Parameters of one (beta, Delta) point. */
typedef struct {
    double beta;         /* inverse temperature, > 0 */
    double delta;        /* Delta in [0, 1]: J = Delta, J1 = 1 - Delta (Eq. 3.1) */
    double h;            /* field on cos(theta), >= 0 (Eq. 3.7) */
    double h1;           /* field on cos(2 theta), >= 0 (Eq. 3.7) */
    int32_t n_max;       /* Fourier cutoff: D0 = 2 n_max + 1, 0 <= n_max <= 64 */
    int32_t d_cut;       /* bond-dimension cap D_cut, 1 <= d_cut <= 128 */
    int32_t n_steps;     /* coarse-graining steps, one axis each: N = 2^n_steps sites */
    int32_t prec;        /* hotrg_prec */
    int32_t env_policy;  /* 0: compare eps_1 and eps_2 (§2.4.1); 1: left side only */
    int32_t m_range;     /* Bessel-sum range m in [-m_range, m_range]; the thesis uses 50 */
    int32_t eig_max_sweeps; /* Jacobi sweep cap (default 40 when <= 0) */
    int32_t tkind;       /* hotrg_tkind of the pure tensor: HOTRG_T_PURE or HOTRG_T_ISING */
    double tie_rtol;     /* cut-cluster width relative to lambda_max (default 1e-9 when <= 0): wide
                            enough that exactly degenerate charge-conjugate pairs stay tied under the
                            split forms' ~1e-10 relative error */
    double eig_tol;      /* Jacobi stop: off-diagonal Frobenius <= eig_tol * ||E_q||_F (1e-15 when <= 0) */
    double side_rtol;    /* eps_2 wins only if eps_2 < eps_1 (1 - side_rtol) (default 1e-6 when <= 0):
                            mirror-image environments give eps_1 = eps_2, which must not be decided by
                            the rounding of the eigenvalue sums */
    int32_t block_sparse; /* 1: the environments (A, B, E) and the coarse contraction (s1, s2, s3)
                             run per charge block (the U(1) or Z2 structure of the block-sparse remark
                             of §2.3.1), in every precision form (HOTRG_FP64: FP64 FMA per block).
                             It has no effect with h != 0 (no conserved label), nor on impurity runs
                             except the cos(2 theta) impurity (Eq. 3.21) at h = 0, h1 != 0, which keeps
                             the pure tensor's charge parity and so runs in the Z2 block form.  The
                             result equals the dense form's up to the rounding of the form (the FP64
                             form sums each block's products in the same K order as the dense one, but
                             over the block's elements only).  The planner's value table follows each
                             product's label range (kept charge windows may drift far from 0); a
                             product whose signed label sums span 128 or more values stops that point
                             with HOTRG_ENOTSUP. */
    int32_t gxy_q;       /* order q of the second coupling (1 - Delta) cos(q theta): 0 or 2 = the
                            thesis's q = 2 model; 1, 3, 4 the generalisations it names as future
                            work, a_n = sum_m I_{n - q m}(beta Delta) I_m(beta (1 - Delta)).  The
                            tensor, its charge rule and every kernel are otherwise the same. */
    int32_t eig_mode;    /* eigensolver of the truncation.  0: the form's default -- blocks of at most b
                            states (the listed width) by FP64 Jacobi; larger blocks list b eigenpairs by
                            block subspace iteration: FP32 iterations, then an FP64 Rayleigh-Ritz step,
                            then eig_fp64_iters FP64 subspace iterations each with its Rayleigh-Ritz step
                            (the FP64 form uses this path for U(1) labels and Jacobi on every block for
                            Z2 or no symmetry).  1: FP64 Jacobi on every block (all eigenpairs). */
    int32_t eig_fp64_iters; /* FP64 subspace iterations after the first Rayleigh-Ritz step: 0 = the
                               form's default (6 for HOTRG_FP64, none for the split forms), 1..8 that
                               many, -1 none */
} hotrg_params;

/* Per-step scalars (device- or host-resident, see each entry point). */
typedef struct {
    double ln_c;       /* ln of the Frobenius norm c_k of the coarse tensor */
    double eps_left;   /* discarded eigenvalue weight of E_L (eps_1) */
    double eps_right;  /* same for E_R (eps_2); NaN when env_policy = 1 */
    int32_t side;      /* 0: projector from E_L; 1: from E_R */
    int32_t dprime;    /* D' = min(D_cut, D_h^2) */
    int32_t sweeps;    /* largest Jacobi sweep count over the sectors */
    int32_t status;    /* hotrg_status of the device part of the step: the eigensolver's, else a
                          contraction engine failure (HOTRG_ETIMEOUT, HOTRG_ENOTSUP) */
} hotrg_step_info;

/* Result of one point. */
typedef struct {
    double lnz_per_site;   /* ln Z / N, N = 2^n_steps */
    double ln_c0;          /* ln ||T0||_F */
    double ln_trace;       /* ln sum_{x,y} T[x,x,y,y] of the final tensor */
    double imp_ratio;      /* tTr(T_imp)/tTr(T) when an impurity ran, else 0 */
    hotrg_step_info step[HOTRG_MAX_STEPS];
    int32_t n_steps;
    int32_t status;
} hotrg_result;

/* Observables of one point (§3.4). */
typedef struct {
    double lnz;   /* ln Z / N at (beta, Delta, h = h1 = 0) */
    double f;     /* -lnz / beta */
    double cv;    /* Eq. 3.17 by central difference in beta */
    double m;     /* <cos theta> at h = hbar (impurity, Eq. 3.20) */
    double m1;    /* <cos 2 theta> at h1 = hbar (impurity, Eq. 3.21) */
    double chi;   /* dm/dh at hbar by central difference (Eq. 3.18) */
    double chi1;  /* dm1/dh1 at hbar by central difference */
    int32_t status;
    int32_t pad;
} hotrg_obs;

/* Create a context whose device work goes to cuda_stream (a cudaStream_t,
 * NULL for the legacy default stream).  workspace_bytes reserves device
 * memory up front (0: grow on demand; growth never happens during stream
 * capture -- a run that needs more than the reservation returns
 * HOTRG_ENOMEM while capturing).  Errors: HOTRG_EINVAL (ctx NULL),
 * HOTRG_ENOMEM, HOTRG_ECUDA. */
hotrg_status hotrg_create(hotrg_ctx** ctx, size_t workspace_bytes, void* cuda_stream);

/* Release the context and its workspace.  NULL is a no-op. */
void hotrg_destroy(hotrg_ctx* ctx);

/* Build the initial site tensor (synchronous: returns once the tensor is
 * written) (Eq. 3.4 coefficients with the own Bessel
 * series on the device; Eq. 3.15 / 3.20 / 3.21 field and impurity factors)
 * into T_dev (device, D0^4 FP64, [l][r][u][d], D0 = 2 n_max + 1; for
 * HOTRG_T_ISING D0 = 2) and the D0 bond labels into labels_dev (device,
 * int32).  The tensor is NOT normalised.  Errors: HOTRG_EINVAL for
 * beta <= 0, Delta outside [0,1], negative fields, n_max outside [0, 64],
 * m_range outside [1, 200], null pointers; HOTRG_ECUDA on launch failure. */
hotrg_status hotrg_init_tensor(hotrg_ctx* ctx, const hotrg_params* p, int32_t kind,
                               double* T_dev, int32_t* labels_dev);

/* One coarse-graining step (§2.4.1) of the normalised tensor T_in (device,
 * [Dh][Dh][Dv][Dv] FP64) with horizontal labels q_h (device, Dh int32) and
 * vertical labels q_v (device, Dv int32).  Writes the normalised coarse
 * tensor, already relabelled for the other axis, to T_out (device,
 * [Dv][Dv][D'][D'], D' = min(d_cut, Dh^2)); its new vertical labels to
 * q_out (device, D' int32; the new horizontal labels are q_v); D' to
 * *dprime (host).  info_dev (device, may be NULL) receives the step's
 * scalars.  T_imp_in / T_imp_out (device, may both be NULL) co-update an
 * impurity tensor with the pure tensor's projector and norm:
 * T_imp' = [P^T(T_imp above T)P + P^T(T above T_imp)P] / (2 c_k).
 * T_out must not alias T_in.  Errors: HOTRG_EINVAL (sizes < 1, Dh > 128,
 * Dv > 128, null pointers), HOTRG_ENOMEM (workspace), HOTRG_ECUDA. */
hotrg_status hotrg_step(hotrg_ctx* ctx, const hotrg_params* p,
                        const double* T_in, const int32_t* q_h, const int32_t* q_v,
                        int32_t Dh, int32_t Dv,
                        double* T_out, int32_t* q_out, int32_t* dprime,
                        hotrg_step_info* info_dev,
                        const double* T_imp_in, double* T_imp_out);

/* Run npoints independent points params[0..npoints) (host array) from the
 * initial tensor to ln Z / N, writing out[0..npoints) (host).  With
 * imp_kind = HOTRG_T_IMP_M or HOTRG_T_IMP_M1 each point also carries that
 * impurity tensor and reports imp_ratio; HOTRG_T_PURE runs the pure tensor
 * only.  Returns the first non-OK point status (each out[i].status holds
 * its own: a device-side failure -- a bounded wait that ran out, a block
 * plan that overflowed -- is recorded in a status slot of that point's own
 * device result block and fails that point alone).  Synchronous. */
hotrg_status hotrg_run(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints,
                       int32_t imp_kind, hotrg_result* out);

/* Batched points: the same results as hotrg_run, computed concurrently on
 * nstreams worker streams (1..16, created by the context, each with its own
 * workspace).  Points are sorted by cost (longest first, the s2 work of
 * every step) and each goes to the least-loaded worker.  The first point of
 * a class (every parameter except beta, Delta and the values -- not the
 * zero pattern -- of h, h1) on a worker runs directly; its sequence of
 * kernels is then captured once into a CUDA graph that later points of the
 * class replay, with beta, Delta, h, h1 fed through a device parameter slot.
 * The workers start after the work already enqueued on the context's stream
 * and the context's stream waits for all of them at the end, so CUDA events
 * recorded on it bracket the batch.  With profiling on (hotrg_profile_enable)
 * no graph is replayed: every point runs directly, its regions are timed on
 * its worker's stream and added to the context's counters.
 * nstreams = 0 takes the count chosen by hotrg_autotune_batch (2 if untuned).
 * params, out: host arrays of npoints.  Synchronous.  Returns the first
 * non-OK status (each out[i].status holds its own).  A point that fails on
 * the host (invalid parameters) or on the device (its own status slot, as in
 * hotrg_run, also inside a replayed graph) fails alone; the other points'
 * results are unaffected.  Only a failure of the batch machinery itself
 * (stream, graph or pinned-memory calls) fails every point. */
hotrg_status hotrg_run_batch(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints,
                             int32_t imp_kind, int32_t nstreams, hotrg_result* out);

/* Autotuner of the batch runner (no counterpart in the thesis): runs the
 * sample points (host array, pure tensors) through hotrg_run_batch with 1,
 * 2, ..., max_streams (<= 16) worker streams, each once untimed (workspaces,
 * graphs) and once timed on the host clock, and keeps the fastest count in
 * the context; hotrg_run_batch and hotrg_observables_batch with nstreams = 0
 * use it (2 when never tuned).  best (may be NULL) receives the choice,
 * seconds (may be NULL, max_streams entries) the timed runs.  Synchronous. */
hotrg_status hotrg_autotune_batch(hotrg_ctx* ctx, const hotrg_params* sample, int32_t npoints,
                                  int32_t max_streams, int32_t* best, double* seconds);

/* Tile shape of the split forms' block-sparse tensor-core products (no
 * counterpart in the thesis): every output tile has 128 rows and
 * env_tile_n (environment products) or coarse_tile_n (s1, s2, s3) columns,
 * 128 or 64.  The 64-column tile wastes less of a thin charge block's padding
 * and keeps two TMEM accumulator sets, so the next tile's products run while
 * the previous tile is written out; the 128-column tile issues half as many
 * B loads per row of A.  The results of the two shapes agree to the split
 * form's rounding.  The FP64 form always uses 128 x 128 tiles.  Default:
 * 128 and 128.  Errors: HOTRG_EINVAL for other widths. */
hotrg_status hotrg_set_tiles(hotrg_ctx* ctx, int32_t env_tile_n, int32_t coarse_tile_n);

/* Autotuner of the tile shapes: runs the sample points (host array, pure
 * tensors) through hotrg_run_batch with nstreams worker streams (0: the
 * tuned count) for each of the four (env, coarse) width pairs in the order
 * (128,128), (128,64), (64,128), (64,64) -- each once untimed (graphs of
 * the new shapes) and once timed on the host clock -- and keeps the fastest
 * pair in the context.  env_tile_n, coarse_tile_n (may be NULL) receive it,
 * seconds (may be NULL, 4 entries) the timed runs.  Synchronous. */
hotrg_status hotrg_autotune_tiles(hotrg_ctx* ctx, const hotrg_params* sample, int32_t npoints, int32_t nstreams,
                                  int32_t* env_tile_n, int32_t* coarse_tile_n, double* seconds);

/* Observables of npoints points (§3.4): ln Z/N and f at zero field;
 * C_V = beta^2 [l(beta+hb) - 2 l(beta) + l(beta-hb)] / hb^2 (Eq. 3.17);
 * m = <cos theta> at h = hbar and m1 = <cos 2theta> at h1 = hbar from the
 * impurity tensors (Eq. 3.19-3.21); chi, chi1 by central differences of m,
 * m1 with step dh (Eq. 3.18).  The fields in params are ignored.
 * Synchronous. */
hotrg_status hotrg_observables(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints,
                               double hb, double hbar, double dh, hotrg_obs* out);

/* hotrg_observables for many points at once: the nine runs of every point
 * (beta, beta +- hb; h = hbar, hbar +- dh with the M impurity; h1 = hbar,
 * hbar +- dh with the M1 impurity) go through hotrg_run_batch on nstreams
 * worker streams (1..16; 0: the autotuned count), so the outputs equal hotrg_observables' bit for
 * bit.  Synchronous.  Returns the first failing run's status (each out[i]
 * holds its own); HOTRG_EINVAL for bad arguments. */
hotrg_status hotrg_observables_batch(hotrg_ctx* ctx, const hotrg_params* params, int32_t npoints,
                                     double hb, double hbar, double dh, int32_t nstreams,
                                     hotrg_obs* out);

/* Verification entry point for the contraction engine of a precision
 * form: C = A B^T with A (device, M x K FP64, row stride lda), B (device,
 * N x K FP64, row stride ldb), C (device, M x N FP64, row stride ldc).
 * Every contraction of hotrg_step goes through this engine (the split forms
 * with their coarse-contraction slice count).  Asynchronous.  Errors:
 * HOTRG_EINVAL (sizes < 1, K > 16384, strides < K or < N, null pointers),
 * HOTRG_ENOTSUP (split form without sm_103), HOTRG_ENOMEM, HOTRG_ECUDA. */
hotrg_status hotrg_contract(hotrg_ctx* ctx, int32_t prec, int32_t M, int32_t N, int32_t K,
                            const double* A, int64_t lda, const double* B, int64_t ldb,
                            double* C, int64_t ldc);

/* Allocation-free variant of hotrg_contract for the split forms (the thesis
 * has no counterpart; this is a library convenience).  It is meant for
 * callers that cannot allocate device memory: code running while another
 * allocator owns the whole device memory budget, or code that must not risk
 * the implicit device-wide synchronisation of cudaMalloc.  It needs no
 * hotrg_ctx and calls no cudaMalloc, cudaFree or allocating library routine:
 * its scratch (BF16 operand slices, row exponents and a status word) is one
 * static 32 MiB device array that every GPU loading the library holds until
 * the process exits.
 *   C = A B^T, A (device, M x K FP64, row stride lda), B (device, N x K FP64,
 *   row stride ldb), C (device, M x N FP64, row stride ldc), prec
 *   HOTRG_SPLIT_BF16 or HOTRG_SPLIT_BF16_FAST, work on cuda_stream (a
 *   cudaStream_t, NULL for the legacy default stream).  The call returns
 *   after C is written (it synchronises the stream to read the status word).
 * NS is the slice count of the form's coarse contraction, as in
 * hotrg_contract: 5 for HOTRG_SPLIT_BF16 (the environment variable
 * HOTRG_SPLIT_SLICES="e,c", read once per process, sets it to c in 3..5, which
 * changes both the accuracy and the size limit below) and 3 for _FAST.
 * Size limit: with Kp = K rounded up to 32, Mp and Np = M and N rounded up to
 * 128, the call needs
 * NS (Mp + Np) Kp 2 + 4 (Mp + Np) bytes (each term rounded up to 256) plus
 * 256; above 32 MiB it returns HOTRG_EINVAL without launching anything.
 * The first call on each device looks up the device address of the static
 * array (cudaGetSymbolAddress) and sets kernel attributes with that device
 * current; make that first call before any stream capture.  All calls on a
 * device share the array, so calls that overlap on the GPU (other streams,
 * other host threads) race; each call clears the status word and rewrites
 * the slices and exponents it reads.  Errors: HOTRG_EINVAL (null pointers,
 * sizes < 1, K > 16384, strides < K or < N, other prec, too large),
 * HOTRG_ENOTSUP (not sm_103), HOTRG_ETIMEOUT, HOTRG_ECUDA. */
hotrg_status hotrg_contract_noalloc(int32_t prec, int32_t M, int32_t N, int32_t K,
                                    const double* A, int64_t lda, const double* B, int64_t ldb,
                                    double* C, int64_t ldc, void* cuda_stream);

/* Surrogate network (no counterpart in the thesis): an ensemble of MLPs
 * 2 -> 128 -> 128 -> 128 -> 4 (tanh hidden layers, linear output) mapping
 * standardised (beta, Delta) to standardised (f, C_V, chi, chi1).  Weights
 * are used in BF16 by every product, which accumulates in FP32; Adam keeps
 * FP32 master weights.  Parameters are laid out flat per member as
 * [W_0 b_0 W_1 b_1 W_2 b_2 W_3 b_3] with W_l row-major [in][out]
 * (hotrg_mlp_num_params() floats).  All buffers named X, T, mean, spread,
 * flat are host arrays (X: n x 2, T / mean / spread: n x 4, row-major). */
typedef struct hotrg_mlp hotrg_mlp;

/* ensemble in [1, 16]; seed fixes the initialisation (Glorot uniform, zero
 * biases) and the minibatch order. */
hotrg_status hotrg_mlp_create(hotrg_mlp** m, int32_t ensemble, uint64_t seed, void* cuda_stream);
void hotrg_mlp_destroy(hotrg_mlp* m);
int64_t hotrg_mlp_num_params(void);
hotrg_status hotrg_mlp_set_params(hotrg_mlp* m, int32_t member, const float* flat);
hotrg_status hotrg_mlp_get_params(hotrg_mlp* m, int32_t member, float* flat);
/* Loss (mean squared error) and its gradient for one member on n <= 4096
 * samples (gradient written to grad_flat when not NULL). */
hotrg_status hotrg_mlp_gradients(hotrg_mlp* m, int32_t member, const float* X, const float* T, int32_t n,
                                 float* loss, float* grad_flat);
/* epochs of Adam (learning rate lr) over minibatches of batch <= 4096 for
 * every member; final_loss: the members' mean loss on the last minibatch. */
hotrg_status hotrg_mlp_train(hotrg_mlp* m, const float* X, const float* T, int32_t n, int32_t epochs,
                             int32_t batch, float lr, float* final_loss);
/* Ensemble mean and spread (standard deviation over members) per output. */
hotrg_status hotrg_mlp_predict(hotrg_mlp* m, const float* X, int32_t n, float* mean, float* spread);

/* Surrogate driver (no counterpart in the thesis).  The surrogate maps
 * (beta, Delta) to (f, C_V, chi, chi1) = (f, cv, chi, chi1) of hotrg_obs,
 * through the MLP ensemble above on standardised inputs and outputs.  X
 * arrays are host n x 2 (beta, Delta) and Y arrays host n x 4, row-major,
 * FP64, in physical units. */
typedef struct {
    double x_mean[2], x_std[2];   /* input standardisation, x' = (x - mean) / std */
    double y_mean[4], y_std[4];   /* output standardisation */
} hotrg_scaling;

/* Mean and population standard deviation of every column (a zero standard
 * deviation is replaced by 1).  Host only.  Errors: HOTRG_EINVAL. */
hotrg_status hotrg_scaling_fit(const double* X, const double* Y, int32_t n, hotrg_scaling* s);

/* Fit the scaling to (X, Y) and train every member of m on the
 * standardised data (hotrg_mlp_train).  Synchronous. */
hotrg_status hotrg_surrogate_fit(hotrg_mlp* m, const double* X, const double* Y, int32_t n, int32_t epochs,
                                 int32_t batch, float lr, hotrg_scaling* s, float* final_loss);

/* Ensemble prediction in physical units (y, n x 4) and the ensemble spread
 * in standardised units (spread, n x 4; may be NULL).  Synchronous. */
hotrg_status hotrg_surrogate_predict(hotrg_mlp* m, const hotrg_scaling* s, const double* X, int32_t n,
                                     double* y, double* spread);

/* Refinement points near the transition: for each of n_delta values of
 * Delta, the surrogate's C_V and chi are evaluated on n_beta points evenly
 * spaced over [beta_lo, beta_hi]; around each of the two maxima, per_peak
 * points evenly spaced over [beta* - width, beta* + width] (clipped to the
 * range) are written to X_out (n_delta * 2 * per_peak rows: Delta-major,
 * C_V window first).  peaks_out (n_delta x 2, may be NULL) receives the
 * beta of the C_V and chi maxima.  Synchronous. */
hotrg_status hotrg_surrogate_peaks(hotrg_mlp* m, const hotrg_scaling* s, const double* deltas, int32_t n_delta,
                                   double beta_lo, double beta_hi, int32_t n_beta, int32_t per_peak,
                                   double width, double* X_out, double* peaks_out);

/* Predict at n points; every point whose largest standardised spread
 * exceeds threshold is re-solved by hotrg_observables_batch with params
 * base (beta and Delta replaced; nstreams worker streams) and its y row
 * replaced by the HOTRG values.  solved[i] = 1 for re-solved points, else
 * 0; *n_solved (may be NULL) counts them.  spread (may be NULL) keeps the
 * ensemble's spread for every point.  Synchronous. */
hotrg_status hotrg_surrogate_refine(hotrg_ctx* ctx, hotrg_mlp* m, const hotrg_scaling* s,
                                    const hotrg_params* base, const double* X, int32_t n, double threshold,
                                    double hb, double hbar, double dh, int32_t nstreams, double* y,
                                    double* spread, int32_t* solved, int32_t* n_solved);

/* Phase-boundary extraction (§3.4 results, Table 3.1).
 *
 * The thesis locates the transitions from temperature scans at fixed Delta:
 * the peaks of C_V(T) at zero field, and the peak of chi(T) (Eq. 3.18) at a
 * small central field hbar, extrapolated to hbar -> 0.  The extrapolation is
 * read as the least-squares fit T_p(hbar) = a + b hbar^c: the thesis prints
 * a, b, c for Delta = 0.32 (a being the zero-field T_c of Table 3.1 there)
 * and cites the form without printing it.
 *
 * hotrg_find_peaks and hotrg_fit_tc are host only (no context, no device
 * work); hotrg_phase_scan runs its HOTRG points through hotrg_run_batch. */

/* Peaks of y sampled on a strictly ascending grid x (n host points).  A
 * peak is an interior local maximum: a run y[i] = ... = y[j] (1 <= i <= j <=
 * n - 2) with y[i-1] < y[i] and y[j] > y[j+1], taken at k = (i + j) / 2
 * (integer division).  Its prominence is y[k] minus the higher of the two
 * smallest values met walking left and right from k up to the first
 * strictly higher value or the end.  Peaks with prominence >= min_prominence
 * count and *n_found receives their number; of these the cap most prominent
 * (ties: smaller k) are written in ascending x: x_peak / y_peak the vertex
 * of the parabola through the samples k-1, k, k+1 (the sample k itself when
 * the three values are equal), prominence (may be NULL) the prominences.
 * Errors: HOTRG_EINVAL (NULL x, y or n_found; NULL x_peak / y_peak with
 * cap > 0; n < 0; cap < 0; x not strictly ascending; a non-finite x, y or
 * min_prominence). */
hotrg_status hotrg_find_peaks(const double* x, const double* y, int32_t n, double min_prominence, int32_t cap,
                              double* x_peak, double* y_peak, double* prominence, int32_t* n_found);

typedef struct {
    double a, b, c;             /* T_p(hbar) = a + b hbar^c; a = T_c in the limit hbar -> 0 */
    double a_err, b_err, c_err; /* sqrt(diag(s^2 (J^T J)^-1)), s^2 = rss / (n - 3), J = d model / d(a, b, c);
                                   0 when n = 3 */
    double rss;                 /* residual sum of squares at (a, b, c) */
    int32_t n;                  /* points fitted (0: no fit was made) */
    int32_t at_bound;           /* 1 when c sits on c_lo or c_hi (always when c_lo = c_hi) */
} hotrg_tc_fit;

/* Least-squares fit of T_p(hbar) = a + b hbar^c over n host points, with
 * c in [c_lo, c_hi] (c_lo = c_hi fixes c; c_lo <= 0 and c_hi <= 0 together
 * select the bracket [0.05, 2]).  For each c the best (a, b) is linear; the
 * profile residual is scanned on 2001 evenly spaced c and its stationary
 * point around the best one solved to full precision; a minimum on a bound
 * stays on it.  Errors: HOTRG_EINVAL (NULL pointers; fewer than 3 distinct
 * hbar; hbar <= 0; a non-finite value; 0 < c_lo <= c_hi violated),
 * HOTRG_ENOCONV (no stationary point found in the bracket). */
hotrg_status hotrg_fit_tc(const double* hbar, const double* t_peak, int32_t n, double c_lo, double c_hi,
                          hotrg_tc_fit* out);

typedef struct {
    int32_t field;         /* HOTRG_T_IMP_M: chi = dm/dh in the field h; HOTRG_T_IMP_M1: chi1 = dm1/dh1 in h1;
                              0: the thesis's choice, h for Delta > 0.36 and h1 for Delta <= 0.36 */
    int32_t nstreams;      /* worker streams of hotrg_run_batch, 0..16 (0: the tuned count) */
    double dh;             /* field step of chi's central difference, > 0 and <= every hbar */
    double hb;             /* beta step of C_V's central difference, > 0 */
    double min_prominence; /* of a chi peak (hotrg_find_peaks), finite */
    double c_lo, c_hi;     /* exponent bracket of the fit (hotrg_fit_tc) */
} hotrg_phase_opts;

/* Temperature scans at one Delta.  base fixes the gXY model and the run
 * (delta, n_max, d_cut, n_steps, prec, block_sparse, ...; tkind must be
 * HOTRG_T_PURE); its beta, h and h1 are ignored.  temps: n_t >= 3 strictly
 * ascending positive temperatures (host), beta_j = 1 / temps[j].
 *   chi[k * n_t + j] = [m(hbar[k] + dh) - m(hbar[k] - dh)] / (2 dh) at beta_j,
 *     m the impurity ratio of the selected field (the other field 0): the
 *     runs and arithmetic of hotrg_observables' chi / chi1 at hbar = hbar[k],
 *     so the values equal its bit for bit (n_h >= 0 rows);
 *   cv[j] (cv may be NULL: no pure runs) = beta_j^2 [lnZ(beta_j + hb)
 *     - 2 lnZ(beta_j) + lnZ(beta_j - hb)] / hb^2 at h = h1 = 0, hotrg_obs.cv
 *     bit for bit;
 *   t_peak[k] (may be NULL) = x_peak of the most prominent peak of row k
 *     (hotrg_find_peaks with opts->min_prominence), NaN when the row has none;
 *   *fit (may be NULL) = hotrg_fit_tc over the rows with a peak, or n = 0 and
 *     NaN parameters when fewer than three rows have one;
 *   *field_used (may be NULL) = the field applied (HOTRG_T_IMP_M or _M1).
 * 2 n_h n_t impurity runs and 3 n_t pure runs go through hotrg_run_batch.
 * Synchronous; host outputs.  Errors: HOTRG_EINVAL (arguments); a run's
 * status (the tables are then undefined); HOTRG_ENOCONV from the fit (the
 * tables and t_peak are valid). */
hotrg_status hotrg_phase_scan(hotrg_ctx* ctx, const hotrg_params* base, const double* temps, int32_t n_t,
                              const double* hbar, int32_t n_h, const hotrg_phase_opts* opts, double* cv,
                              double* chi, double* t_peak, hotrg_tc_fit* fit, int32_t* field_used);

/* Per-kernel-class timing recorded with CUDA events on the context's stream
 * (the stream every library kernel runs on).  Classes of the contraction
 * engine: 0 environment products, 1 coarse contraction (s1, s2, s3), 2 other.
 * gemm_ms / gemm_flops cover only the GEMM kernel launches themselves (FP64
 * SIMT or tensor-core), gemm_flops being the algorithmic 2 M N K of each
 * launch; slice_ms covers the operand-slicing kernels of the split forms;
 * eig_ms the truncation (eigensolve, selection, projector); step_ms whole
 * steps.  launches counts every kernel the library launched. */
typedef struct {
    int64_t launches;
    int64_t gemm_calls[3];
    double gemm_ms[3];
    double gemm_flops[3];
    double slice_ms;
    double eig_ms;
    double step_ms;
    int64_t steps;
    double eig_part_ms[4]; /* block discovery + Jacobi; FP32 subspace; FP64 Rayleigh-Ritz; selection + projector */
    /* Block-sparse products only (counted on the device by the block planner), per class:
     * operand_elems = sum over blocks of (M_g + N_g) K_g, the operand elements a product reads
     * once (what the slicers of the split forms read as 8 bytes and write as NS BF16 slices);
     * output_elems = sum over blocks of M_g N_g, the elements it writes. */
    double operand_elems[3];
    double output_elems[3];
} hotrg_profile;

/* Turn event timing on (enable != 0) or off, and reset the counters.
 * Errors: HOTRG_EINVAL (ctx NULL), HOTRG_ECUDA. */
hotrg_status hotrg_profile_enable(hotrg_ctx* ctx, int32_t enable);

/* Synchronise the context's stream, fold the pending events into the
 * totals and copy them to *out (host).  Errors: HOTRG_EINVAL, HOTRG_ECUDA. */
hotrg_status hotrg_profile_read(hotrg_ctx* ctx, hotrg_profile* out);

/* Text of the last error on this context ("" when none).  Valid until the
 * next call on the same context. */
const char* hotrg_last_error(hotrg_ctx* ctx);

/* Library version string. */
const char* hotrg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HOTRG_H */
