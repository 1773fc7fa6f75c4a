/*
 * psms.h -- C ABI of the GB300 (sm_103a) library for the hot path of the
 * Partially Stochastic Multi-Step (PSMS) filter for N_f = 2 Wilson fermions
 * (J. Finkenrath, F. Knechtli, B. Leder, "Fermions as Global Correction: the
 * QCD Case", arXiv:1204.1306).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Lattice extents dims[4] = (L0, L1, L2, L3); mu = 0 is time.  Quark fields
 *    are antiperiodic in time and periodic in space (Sec. 6); gauge fields are
 *    periodic.  Domain blocks have extents block[4]; every block extent must be
 *    a power of two >= 2 dividing the lattice extent (Sec. 3, Fig. 1).
 *  - Canonical layouts (used by *_set / *_get / *_import / *_export):
 *      links  : complex<double> U[x0][x1][x2][x3][mu][3][3]   (x3 fastest)
 *      spinor : complex<double> psi[x0][x1][x2][x3][spin][colour]
 *    complex numbers are interleaved (re, im) doubles.  U[x][mu] is the link
 *    from x to x + mu-hat.  gamma matrices: chiral basis,
 *      gamma_mu = [[0, e_mu], [e_mu^dagger, 0]], e_0 = -1, e_k = -i sigma_k,
 *    gamma_5 = diag(1, 1, -1, -1).
 *  - D always denotes D_w + m0 of Eq. (Dw) with m0 = 1/(2 kappa) - 4:
 *      D psi(x) = (4 + m0) psi(x) - 1/2 sum_mu { U(x,mu)(1 - gamma_mu) psi(x+mu)
 *                                   + U(x-mu,mu)^dagger (1 + gamma_mu) psi(x-mu) }.
 *  - "native" spinor buffers hold one full-lattice quark field in the
 *    library's device layout for the given precision (even-odd, block-major,
 *    structure of arrays); their size is psms_spinor_bytes().  Convert with
 *    psms_spinor_import / psms_spinor_export.
 *  - All pointers named *_dev are device pointers owned by the caller; the
 *    library never frees them.  Host result arrays are caller-allocated.  The
 *    context owns its gauge fields, scratch buffers and CUDA events.
 *  - Every entry point returns a psms_status and never throws or aborts; on
 *    error psms_last_error() describes the failure.  Work is queued on the
 *    stream given to psms_set_stream (default: the legacy default stream);
 *    entry points that return host values synchronise that stream.
 *  - Random numbers: Philox-4x64-10 (Salmon et al., SC'11), key = (seed, tag),
 *    counters as stated at each entry point; a uniform is
 *    ((w >> 12) + 1/2) * 2^-52 of a 64-bit output word w, so identical
 *    (seed, counter) give identical draws on every device.
 */
#ifndef PSMS_H
#define PSMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSMS_OK = 0,
    PSMS_EINVAL = 1,     /* bad argument or unsupported geometry            */
    PSMS_ENOMEM = 2,     /* device allocation failed                        */
    PSMS_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed     */
    PSMS_ENOCONV = 4,    /* a Krylov solve missed its tolerance at maxit    */
    PSMS_ETIMEOUT = 5,   /* a device-side bounded wait ran out              */
    PSMS_ESPECTRUM = 6,  /* non-finite estimate (NaN / Inf)                 */
    PSMS_EHEATBATH = 7   /* an SU(2) draw hit its attempt limit             */
} psms_status;

typedef enum {
    PSMS_PREC_F64 = 0,   /* FP64 links, FP64 spinors, FP64 arithmetic       */
    PSMS_PREC_F32 = 1,   /* FP32 links, FP32 spinors, FP32 arithmetic       */
    PSMS_PREC_BF16 = 2   /* FP32 links, BF16 spinor storage, FP32 arithmetic*/
} psms_prec;

/* Operator selector for psms_dw_apply / psms_solve. */
enum {
    PSMS_OP_FULL = -1,   /* D on the whole lattice (Eq. (Dw))               */
    PSMS_OP_BLOCKS = -2  /* D_bb + D_ww: every Dirichlet block at once      */
    /* a value b >= 0 selects the single block D_b with lexicographic block
       index b = ((B0*nb1 + B1)*nb2 + B2)*nb3 + B3, B_mu = x_mu / block[mu];
       the output is zero outside block b. */
};

/* Active-link sets of psms_gauge_sweep. */
enum {
    PSMS_ACTIVE_BLOCKS = 0, /* links of a block with <= 1 endpoint on its boundary
                               (Sec. 3); every intra-block link if an extent <= 2 */
    PSMS_ACTIVE_ALL = 1     /* every link (pure-gauge thermalisation)          */
};

/* Estimator levels / modes of psms_logdet_ratio.  PSMS_LEVEL_GLOBAL always
 * means the global Schur complement of the context's blocks;
 * PSMS_LEVEL_SUB and PSMS_LEVEL_OUTER_GLOBAL need outer blocks
 * (psms_set_outer_blocks). */
enum { PSMS_LEVEL_BLOCK = 1, PSMS_LEVEL_GLOBAL = 2, PSMS_LEVEL_SUB = 4, PSMS_LEVEL_OUTER_GLOBAL = 6 };
enum { PSMS_EST_INTERP = 0, PSMS_EST_INDEPENDENT = 1 };

typedef struct psms_ctx psms_ctx;

typedef struct {
    int dims[4];       /* lattice extents L0..L3 (each even)                 */
    int block[4];      /* block extents l0..l3 (powers of two >= 2)          */
    double kappa;      /* hopping parameter, kappa = 1/(2 m0 + 8)            */
    int n_fields;      /* number of gauge-field slots owned by the context   */
} psms_lattice_desc;

typedef struct {
    int outer_iters;       /* FP64 defect-correction steps                     */
    long long inner_iters; /* Krylov iterations summed over systems            */
    double true_residual;  /* max over systems of |b - D x| / |b| (FP64)       */
    int n_systems;
} psms_solve_info;

/* Relative gauge fixing (Sec. 4.2 and App. B): steepest descent of the
 * distance of Eq. (sprodgf) between U^{g_1} and U'^{g_2}, the
 * transformations living on the block interiors (sites whose eight
 * neighbours lie in the same block).  Per step and interior point:
 * Delta = sum_mu [U'(x,mu) U(x,mu)^dag + U'(x-mu,mu)^dag U(x-mu,mu)] on the
 * current pair, Y = Delta - Delta^dag - Tr(Delta - Delta^dag)/3,
 * theta = sum |Y_ij|^2, and the pair takes U -> U^h, U' -> U'^{h^{-1}} with
 * h = exp(alpha/4 Y) (relative rotation exp(alpha/2 Y), Eq. (ming)).  A block
 * stops when the mean theta over its interior drops below theta_tol; after
 * max_iter steps without that it restarts with alpha - dalpha, down to
 * alpha_min, and keeps its last state after that.  Each block iterates on
 * its pair in a canonical order, so exchanging U and U' exchanges the
 * results exactly (the symmetry detailed balance needs). */
typedef struct {
    double alpha0;     /* first step size (App. B: 0.15)                     */
    double alpha_min;  /* smallest step size (0.10)                          */
    double dalpha;     /* step-size decrement (0.01)                         */
    double theta_tol;  /* convergence threshold on the block mean of theta   */
    int max_iter;      /* steps per step size, 0 .. 10^6                     */
    int prec;          /* PSMS_PREC_F64 or PSMS_PREC_F32 iteration arithmetic */
} psms_relgf_params;

typedef struct {
    /* level 0: proposal (Sec. 6): n_iter x (HB + n_or OR + n_or OR + HB)    */
    double beta0;
    int n_iter;
    int n_or;
    /* level 1: block det ratios, N = n_block interpolation steps (Eq. (staccN)) */
    int n_block;
    double beta_block;     /* coefficient of dS_w,b at level 1 (App. C; dS_w,b as
                              in psms_block_action_change)                     */
    /* level 2: global Schur-complement det ratio                              */
    int n_global;
    double beta_global;    /* coefficient of dS_w at level 2 (App. C)          */
    int global_level;      /* 0: stop after level 1                            */
    double tol;            /* relative true residual of every solve            */
    int inner_prec;        /* psms_prec of the inner Krylov iterations         */
    uint64_t seed;
    uint64_t step;         /* filter step counter (RNG counter base)           */
    int learned;           /* 1: insert the learned level before level 1       */
    int gauge_fix;         /* 1: interpolate between relatively gauge-fixed
                              endpoints (Sec. 4.2) at levels 1 and 2          */
    psms_relgf_params relgf;
    int proposal_field;    /* -1: level 0 is the domain sweep; else the slot
                              holding an external proposal, which must differ
                              from the field on active links only and be
                              drawn by a symmetric proposal (detailed-balance
                              tests); the slot is left unchanged             */
    int translate;         /* 1: random translation after the global level */
    /* parametrised HYP level (App. C; the first filter of Tables 1 and 2):
       with hyp_level = 1 a level before the learned and block levels accepts
       block b with min{1, exp(-Delta_b)}, Delta_b = hyp_beta[0] dS_w,b +
       hyp_beta[1] dS_HYP,b (psms_block_action_change,
       psms_hyp_block_action with the default smearing), decision counter
       (step, 5, b), or one decision on the sum (counter (step, 5, 0)) for
       block extents <= 2; blocks it rejects keep their links and skip the
       later block levels.  beta_block_hyp and beta_global_hyp add the HYP
       action's change to the block and global levels.                    */
    int hyp_level;
    double hyp_beta[2];
    double beta_block_hyp;
    double beta_global_hyp;
    /* recursive decomposition (psms_set_outer_blocks): stage 2 with n_sub
       interpolation steps (0: off) and the coefficient of dS_w           */
    int n_sub;
    double beta_sub;
    /* exact block level (Sec. 3: LU of the small blocks; Tables 1 and 2):
       with exact_block = 1 the block level uses beta_block_det times the
       exact change of S_b = -2 ln|det D_b| (psms_block_logdet) instead of
       the stochastic estimate; beta_global_blockdet adds that action's
       change on the accepted blocks to the global level (App. C allows
       coefficients on exactly evaluated actions only).  Not combined with
       the recursive decomposition. */
    int exact_block;
    double beta_block_det;
    double beta_global_blockdet;
} psms_filter_params;

typedef struct {
    int n_blocks;
    int n_accept_blocks;
    int accept_global;
    int shift[4];
    double delta_global;
    double delta_block_sum;
    long long solver_iters;
    int hb_failed;
    int n_accept_learned;  /* blocks passing the learned level (-1: no level)  */
    long long gf_steps;    /* gauge-fixing steps summed over blocks            */
    int n_accept_hyp;      /* blocks passing the HYP level (-1: no level)      */
    int n_accept_sub;      /* outer blocks accepted at stage 2 (-1: no stage)  */
} psms_filter_result;

typedef struct {
    int epochs;
    int batch;             /* minibatch size                                   */
    double lr;             /* AdamW step size                                  */
    double beta1, beta2, eps;
    double weight_decay;
    int normalise;         /* 1: set the input mean / scale and the output scale ys
                              (spread of the labels about their mean) from the data */
    uint64_t seed;         /* minibatch shuffling                              */
} psms_train_params;

/* ---- context ------------------------------------------------------------ */

/* Create a context for one lattice geometry (Sec. 3).  Allocates n_fields
 * FP64 gauge fields (set to the unit field).  Fails with PSMS_EINVAL for
 * extents that are odd, not divisible by the block, or blocks that are not
 * powers of two; PSMS_ENOMEM / PSMS_ECUDA otherwise. */
psms_status psms_create(const psms_lattice_desc *desc, psms_ctx **out);
psms_status psms_destroy(psms_ctx *ctx);
/* Static description of the last error on ctx (never NULL). */
const char *psms_last_error(const psms_ctx *ctx);
/* Queue subsequent work on this cudaStream_t (pass NULL for the default). */
psms_status psms_set_stream(psms_ctx *ctx, void *cuda_stream);
/* Lattice facts: n_blocks, dim(P) of Eq. (dimproj) (0 without a black/white
 * colouring), active links per lattice. */
psms_status psms_geometry_info(const psms_ctx *ctx, long long *n_blocks, long long *dim_P,
                               long long *n_active_links);

/* ---- gauge fields --------------------------------------------------------- */

/* Synthetic field U = exp(i eps H), H = sum_a omega_a lambda_a / 2, omega_a ~
 * N(0,1) from Philox (key (seed, 1), counter (4*site+mu, j, 0, 0), j = 0,1,
 * Box-Muller), then reunitarised (Gram-Schmidt rows 0,1; row 2 = conj(r0 x r1)). */
psms_status psms_gauge_init(psms_ctx *ctx, int field, double eps, uint64_t seed);
/* Copy a canonical-layout FP64 field in / out of slot `field`. */
/* psms_gauge_set rejects a field holding NaN or infinite values with
 * PSMS_EINVAL before writing the slot; psms_spinor_import and psms_solve
 * do the same for their input spinor. */
psms_status psms_gauge_set(psms_ctx *ctx, int field, const double *links_dev);
psms_status psms_gauge_get(psms_ctx *ctx, int field, double *links_dev);
psms_status psms_gauge_copy(psms_ctx *ctx, int dst, int src);
/* Mean plaquette <ReTr U_p>/3 and S_w of Eq. (Sw) (without beta), FP64,
 * deterministic reduction.  Host outputs (either may be NULL). */
psms_status psms_plaquette(psms_ctx *ctx, int field, double *mean_plaq, double *s_w);
/* Pure-gauge proposal (Sec. 6) on slot `field`: n_iter iterations of
 * HB + n_or OR sweeps (checkerboard subsets (mu, parity) in forward order)
 * and n_or OR + HB sweeps in reversed order, Cabibbo-Marinari SU(2)
 * subgroups in random order per link, at coupling beta, then FP64
 * reunitarisation of the updated links.  Sweep ids start at sweep0.
 * *failed_out (may be NULL) counts SU(2) draws that hit 1000 attempts. */
psms_status psms_gauge_sweep(psms_ctx *ctx, int field, int active_set, int n_iter, int n_or,
                             double beta, uint64_t seed, uint64_t sweep0, int *failed_out);
/* Random translation U'(x) = U(x - s) of slot `field` (Sec. 3). */
psms_status psms_gauge_translate(psms_ctx *ctx, int field, const int shift[4]);

/* ---- quark fields ----------------------------------------------------------- */

size_t psms_spinor_bytes(const psms_ctx *ctx, int prec);
psms_status psms_spinor_import(psms_ctx *ctx, const double *canonical_dev, void *native_dev, int prec);
psms_status psms_spinor_export(psms_ctx *ctx, const void *native_dev, double *canonical_dev, int prec);

/* out = op(U_field) in, Eq. (Dw); op is PSMS_OP_FULL, PSMS_OP_BLOCKS or a
 * block index (Eq. (domdec), Dirichlet blocks).  in / out are native
 * buffers of precision prec and must not alias. */
psms_status psms_dw_apply(psms_ctx *ctx, int field, int op, const void *in_dev, void *out_dev, int prec);

/* Solve op(U_field) x = b to |b - op x| <= tol |b| in FP64 (true residual),
 * with inner Krylov iterations on the even-odd operator in inner_prec inside
 * FP64 defect correction: BiCGStab (whole lattice, default) or CGNR (blocks,
 * default), see psms_full_solver / psms_block_krylov.  b, x: native FP64
 * buffers.  PSMS_ENOCONV if maxit inner iterations do not reach tol;
 * PSMS_EINVAL for a non-finite b. */
psms_status psms_solve(psms_ctx *ctx, int field, int op, const void *b_dev, void *x_dev, double tol,
                       int maxit, int inner_prec, psms_solve_info *info);

/* Stochastic estimate of ln det ratios between slots field_old (U) and
 * field_new (U'), Eqs. (stacc), (staccN), (gfparam):
 *   mode PSMS_EST_INTERP: n factors M_i = op(U_{i+1})^-1 op(U_i),
 *     U_i = ((n-i)/n) U + (i/n) U', one noise xi_i each;
 *   mode PSMS_EST_INDEPENDENT: n independent noises with M = op(U')^-1 op(U).
 * level PSMS_LEVEL_BLOCK: op = D_b for every block b; delta_out[b*n + i] =
 *   |M_{b,i} xi_i|^2 - |xi_i|^2 restricted to block b.
 * level PSMS_LEVEL_GLOBAL: op = 1 - PQ (Sec. 4.4), noise on range(P),
 *   (1 - PQ)^-1 = 1 - P D^-1 D_wb; delta_out[i].
 * Noise: key (seed, 2), counter (counter, (level << 32) | i, site, j).
 * delta_out: host array. */
psms_status psms_logdet_ratio(psms_ctx *ctx, int level, int field_old, int field_new, int n, int mode,
                              uint64_t seed, uint64_t counter, double tol, int inner_prec,
                              double *delta_out);

/* One step of the 3-level hierarchical filter (Eq. (hierarchy), Sec. 3):
 * proposal sweep of `field`, per-block stochastic det-ratio accept/reject
 * (one decision on the sum for blocks with an extent <= 2), global Schur
 * accept/reject, random translation.  Decisions: accept iff Delta <= 0 or
 * u < exp(-Delta), u from key (seed, 4), counter (step, level, block, 0).
 * delta_block_out / accept_block_out: host arrays of n_blocks (may be NULL). */
psms_status psms_filter_step(psms_ctx *ctx, int field, const psms_filter_params *prm,
                             psms_filter_result *res, double *delta_block_out, int *accept_block_out);

/* Per-block records of the last psms_filter_step on ctx, for callers that
 * check or log what a level decided on.  what selects the record and n the
 * capacity of out (host):
 *   PSMS_REC_H          n_blocks: the learned level's h_b as the step used it
 *                       (0 where the level is off);
 *   PSMS_REC_DELTA_HYP  n_blocks: Delta_b of the HYP level (0 when off);
 *   PSMS_REC_ACCEPT_BLOCK n_blocks: level-1 decisions (1 / 0) before stage 2;
 *   PSMS_REC_DELTA_SUB  n_outer: Delta_b of stage 2 per outer block (0 for
 *                       outer blocks that were not estimated);
 *   PSMS_REC_ACCEPT_SUB n_outer: stage-2 decisions per outer block (1 / 0).
 * Blocks in lexicographic order.  Returns the record's length in *n_out.
 * PSMS_EINVAL for an unknown record, n too small, or no step with that
 * record yet. */
enum { PSMS_REC_H = 0, PSMS_REC_DELTA_HYP = 1, PSMS_REC_ACCEPT_BLOCK = 2, PSMS_REC_DELTA_SUB = 3,
       PSMS_REC_ACCEPT_SUB = 4 };
psms_status psms_filter_record(psms_ctx *ctx, int what, double *out, int n, int *n_out);

/* ---- batched block solves over several lattices ---------------------------
 * All Dirichlet blocks x all right-hand sides of several lattices (each its
 * own context, possibly of different sizes; same device) solved by one
 * persistent launch (Sec. 3: the block levels are independent per block):
 * CTAs take (lattice, block, system) items from an atomic counter; every
 * item runs the even-odd CGNR with its FP64 defect correction on the device.
 * psms_block_plan_create allocates the scratch, autotunes the schedule
 * (persistent grid of 1..4 CTAs per SM x three work orders, each timed once
 * on the given inputs; the results do not depend on the schedule) and
 * captures the tuned launch sequence in a CUDA graph.  psms_block_plan_run
 * replays the graph on `stream` (refreshing FP32 link copies first) and
 * returns the summed inner iterations and the worst relative residual.
 * Problem i: b_dev / x_dev hold n_rhs native FP64 fields back to back; the
 * pointers and fields are fixed at plan creation. */
typedef struct {
    psms_ctx *ctx;
    int field;
    int n_rhs;
    const void *b_dev;
    void *x_dev;
} psms_block_problem;
typedef struct psms_block_plan psms_block_plan;
psms_status psms_block_plan_create(const psms_block_problem *probs, int n_probs, double tol, int maxit,
                                   int inner_prec, psms_block_plan **out);
psms_status psms_block_plan_run(psms_block_plan *plan, void *cuda_stream, psms_solve_info *info);
/* The tuned schedule: persistent CTAs, work order (0 lattice-major,
 * 1 system-major, 2 round-robin over lattices), its tuning time in ms. */
psms_status psms_block_plan_schedule(const psms_block_plan *plan, int *ctas, int *order, double *tuned_ms);
psms_status psms_block_plan_destroy(psms_block_plan *plan);

/* ---- learned delayed-acceptance level ------------------------------------
 * The paper has no learned level; it is inserted through the mechanism of
 * App. C (an auxiliary action whose coefficients sum to zero over the later
 * levels): a deterministic antisymmetric surrogate h_b(U, U') of the block
 * log det ratio is accepted with min{1, exp(-h_b)} per block (u from key
 * (seed, 4), counter (step, 3, block, 0)), and level 1 then uses
 * Delta_b - h_b, so the chain stays exact whatever the network predicts.
 *
 * Features (32 per block, float, out[b * 32 + k], b lexicographic): mean and
 * population variance of ReTr U_p / 3 over the plaquettes inside the block
 * per plane (mu,nu) = (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) (k = 0..5, 6..11),
 * mean Tr F_{mu nu}^2 of the clover field strength over sites whose four
 * leaves lie inside the block (k = 12..17), zeros (k = 18..31). */
psms_status psms_domain_features(psms_ctx *ctx, int field, float *out_dev);
/* Network input rows of a proposal field_old -> field_new, out[b * 64 + k]:
 * k < 32 features of the old field, k >= 32 of the new one, and in slots 18
 * and 50 (both halves) the distance of Sec. 4.2, Eq. (sprodgf), restricted
 * to the block: sum over the block's links of ReTr(1 - U^dagger U') / (12 *
 * number of links).  This is the input the filter step's learned level uses. */
psms_status psms_domain_features_pair(psms_ctx *ctx, int field_old, int field_new, float *out_dev);
/* MLP 64 -> 256 -> 256 -> 1 (ReLU), BF16 tensor-core GEMMs with FP32
 * accumulation, FP32 master parameters.  Input z = [f(U_b), f(U'_b)],
 * standardised by per-column mean / scale (both halves share them);
 * h = ys * (n(z) - n(swap z)) / 2.  Parameters: He-normal from Philox
 * key (seed, 6). */
psms_status psms_mlp_init(psms_ctx *ctx, uint64_t seed);
/* Number of floats of the parameter block: W1[256][64], b1[256],
 * W2[256][256], b2[256], w3[256], b3, mu[64], sigma[64], ys. */
size_t psms_mlp_param_count(void);
/* Copy the parameter block to (set = 0) or from (set = 1) host memory. */
psms_status psms_mlp_params(psms_ctx *ctx, float *host, int set);
/* h for n rows of 64 features (device in / out). */
psms_status psms_mlp_predict(psms_ctx *ctx, const float *feats_dev, int n, float *h_dev);
/* Mean squared error of h against labels and its gradient (the first
 * W1..b3 entries of the parameter block) into grad_host (may be NULL). */
psms_status psms_mlp_grad(psms_ctx *ctx, const float *feats_dev, const double *labels_dev, int n, float *grad_host,
                          double *loss);
/* AdamW training on (feats, labels) for tp->epochs epochs of shuffled
 * minibatches; loss_per_epoch[e] (host, may be NULL) = mean minibatch MSE. */
psms_status psms_mlp_train(psms_ctx *ctx, const float *feats_dev, const double *labels_dev, int n,
                           const psms_train_params *tp, double *loss_per_epoch);

/* Profiling: when enabled, the context records CUDA events on its stream
 * around every full-operator Wilson hop launch (enable = 1), or only those of
 * storage precision p (enable = 10 + p); psms_profile_read returns the launch
 * count, the summed milliseconds and the summed algorithmic bytes (spinors in
 * and out, 4 links per output site of a both-parity launch, 8 of a
 * single-parity launch). */
psms_status psms_profile_enable(psms_ctx *ctx, int enable);
psms_status psms_profile_read(psms_ctx *ctx, long long *launches, double *total_ms,
                              double *bytes_per_launch_sum);
/* The same for the block-solver launches while profiling is enabled: count,
 * summed milliseconds and algorithmic bytes (per block-CG iteration and
 * half-block site: 4416 B with FP32 inner iterations, 8832 B with FP64). */
psms_status psms_profile_read_block(psms_ctx *ctx, long long *launches, double *total_ms, double *bytes);
/* Per block-solver launch since profiling was enabled (the first 4096, in
 * launch order): CUDA-event milliseconds and algorithmic bytes.  Writes
 * min(n_max, recorded) entries to the host arrays ms, bytes (each may be
 * NULL) and their number to *n_out. */
psms_status psms_profile_block_launches(psms_ctx *ctx, int n_max, int *n_out, double *ms, double *bytes);

/* Dirichlet block solve that allocates no memory.  The paper has no
 * counterpart: this is a deployment variant of psms_solve for op =
 * PSMS_OP_BLOCKS or a single block index, with FP64 inner iterations.
 *
 * For callers that must not allocate while they run (a fixed memory pool,
 * a host that reserved all device memory up front, or code that cannot let
 * cudaMalloc / cudaFree synchronise the device): its scratch is one static
 * device array of 32 MiB inside the library, held by every GPU that loads
 * the library until the process exits.  The call makes no cudaMalloc,
 * cudaFree or other allocating call; b_dev / x_dev are caller-owned native
 * FP64 buffers, x outside the selected blocks is set to zero.
 *  - Lattices needing more scratch than the array holds (about 26,000 sites)
 *    are rejected with PSMS_EINVAL and a message giving both sizes.
 *  - The first call on a device looks up the array's device address with
 *    that device current (cudaGetSymbolAddress) and caches it; make that
 *    first call outside any stream capture.
 *  - Every call shares the one array and the kernel initialises all of it
 *    that it reads, so nothing carries over between calls; but calls whose
 *    work overlaps on the GPU (other streams, other threads, other contexts
 *    on the same device) race on the array and must be serialised.
 * iters_out: total inner iterations over the blocks; resid_out: largest
 * relative true residual (both host, may be NULL).  PSMS_ENOCONV if a block
 * misses tol within maxit iterations. */
psms_status psms_block_solve_noalloc(psms_ctx *ctx, int field, int op, const void *b_dev, void *x_dev, double tol,
                                     int maxit, long long *iters_out, double *resid_out);

/* ---- relative gauge fixing --------------------------------------------------
 * Gauge-fixes the pair (field_old, field_new) (Sec. 4.2, App. B; parameters
 * and iteration above psms_filter_params) and writes the interpolation
 * endpoints U^{g_1} to slot out_old and U'^{g_2} to slot out_new (FP64).
 * out_old may equal field_old and out_new field_new; out_old != field_new,
 * out_new != field_old, out_old != out_new (else PSMS_EINVAL).  Host arrays
 * of n_blocks entries in lexicographic block order, each may be NULL: steps
 * taken at the final step size, that step size, the final block mean theta,
 * and whether the block iterated on (U', U).  g_dev (device, may be NULL):
 * g_1 then g_2 in the canonical layout [2][V][3][3] complex<double>. */
psms_status psms_relative_gauge_fix(psms_ctx *ctx, int field_old, int field_new, int out_old, int out_new,
                                    const psms_relgf_params *prm, int *steps, double *alpha, double *theta,
                                    int *swapped, void *g_dev);

/* ---- implementation controls -------------------------------------------------
 * The calls below choose how the library computes, not what: the paper has
 * no counterpart for them (it does not fix the Krylov solver), and every
 * choice reaches the same tolerances. */

/* Inner Krylov method of the whole-lattice solves (psms_solve with
 * PSMS_OP_FULL and the global level): BiCGStab on Dhat (default; 16 % faster
 * on the 16^4 global level) or even-odd CGNR on Dhat^dag Dhat; both run
 * inside the same FP64 defect correction to the same true residual.
 * PSMS_EINVAL for another kind. */
enum { PSMS_SOLVER_CGNR = 0, PSMS_SOLVER_BICGSTAB = 1 };
psms_status psms_full_solver(psms_ctx *ctx, int kind);
/* Relative residual reduction that the FP32 / BF16 inner Krylov solve of one
 * defect-correction step of a whole-lattice solve aims for (delta in
 * [1e-8, 0.5]); 0 restores the defaults (BiCGStab 1e-6, CGNR 2e-6 in FP32,
 * 5e-3 in BF16).  A smaller delta means fewer outer steps (each one FP64
 * application of D) and longer inner solves; the FP64 true-residual target
 * is unchanged.  PSMS_EINVAL outside the range. */
psms_status psms_inner_reduction(psms_ctx *ctx, double delta);
/* Links of the FP32 / BF16 inner iterations of the estimators' batched
 * whole-lattice solves (global level, domain levels): on = 1 (default)
 * forms system k's links in the hop as a_k U + b_k U' from FP32 copies of
 * the two endpoint fields of Eq. (gfparam), with the systems of a launch
 * walked side by side so that every endpoint link leaves HBM about once per
 * launch; on = 0 reads one materialised FP32 field per interpolation step.
 * The FP64 true residuals use the FP64 interpolated fields either way, so
 * both reach the same tolerance.  PSMS_EINVAL for another value. */
psms_status psms_shared_links(psms_ctx *ctx, int on);
/* Inner Krylov method of the Dirichlet block solves (default CGNR; the
 * autotuner then chooses among that method's variants only, so every tuned
 * choice gives identical results).  PSMS_EINVAL for another kind. */
psms_status psms_block_krylov(psms_ctx *ctx, int kind);

/* Largest number of interpolation steps (systems) batched into one launch
 * by the estimators; 0 (default) sizes the batches from a device-memory
 * estimate.  Any value gives the same estimates.  PSMS_EINVAL for n < 0. */
psms_status psms_max_chunk(psms_ctx *ctx, int n);

/* Force the Wilson-hop kernel variant (register cap and, for the whole
 * lattice, the branch-free specialisation, the form with two threads per
 * output site, and on blocks of 2 x 128 sites (4^4) the variants that stage
 * each block's input of the other parity in shared memory by per-thread or
 * bulk (TMA) copies; for FP32 links in the whole-lattice mode 14 variants on
 * such blocks, 10 on others, 15 with shared-endpoint links, 4 otherwise; for
 * FP64 links 4 in the whole-lattice mode, 1 otherwise; used modulo their
 * count) instead of the autotuned one; -1 returns to autotuning.  All
 * variants compute the same operator.  *n_variants (may be NULL) receives
 * 15.  PSMS_EINVAL outside -1..14. */
psms_status psms_hop_variant(psms_ctx *ctx, int variant, int *n_variants);

/* ---- checkpoint / resume ----------------------------------------------------
 * The chain state: the FP64 gauge field of slot `field` (canonical layout),
 * the caller's filter-step counter and seed, and the learned level's
 * parameters if present.  All random numbers are counter-based (Philox keyed
 * by seed, counters from the step), so a chain resumed from a checkpoint
 * continues bit-identically.  Loading checks the lattice, blocks and kappa
 * (PSMS_EINVAL on mismatch or a damaged file). */
psms_status psms_checkpoint_save(psms_ctx *ctx, int field, const char *path, uint64_t step, uint64_t seed);
psms_status psms_checkpoint_load(psms_ctx *ctx, int field, const char *path, uint64_t *step, uint64_t *seed);

/* Autotuning of launch variants (on by default; an implementation control).
 * The hop kernel's register cap and branch-free specialisation and the
 * block solver's (cluster size, register cap, hop form) are timed on their
 * first use per shape and the fastest kept.  block_variant >= 0 forces block-solver variant
 * (cluster size, min CTAs per SM) = (1,1),(1,4),(2,1),(2,4),(4,1),(4,4),
 * (8,1),(8,4) for index 0..7, (1,1),(1,4) with one out-of-line copy of
 * the hop for 8, 9, and (1,1),(1,4),(4,4),(8,4) with the branch-free hop
 * (every direction computed, those leaving the block multiplied by zero) for
 * 10..13, (1,4) with the branch-free hop out of line for 14, and with
 * BiCGStab on Dhat instead of CGNR: (1,4) branch-free for 15, (1,4) out of
 * line for 16, (8,4) branch-free for 17 (falling back to 0 when the block is
 * too small for the cluster), and with the block's FP32 links staged once
 * into shared memory (FP32 inner iterations, blocks whose links take at
 * most 100 KB, e.g. 4^4): (1,3) inlined for 18, branch-free for 19, out of
 * line for 20 (falling back to 0 otherwise); -1 restores the tuned choice.
 * Clears the tuning cache.  PSMS_EINVAL outside -1..20.  Variants of one Krylov method
 * give identical results; the two methods agree to the solve tolerance. */
psms_status psms_autotune(psms_ctx *ctx, int enable, int block_variant);

/* Per-block change of the plaquette action, dS_w,b = S_w,b(new) - S_w,b(old)
 * (Eq. (Sw) without beta), for every block (lexicographic block index) into
 * ds_host[n_blocks].  A plaquette whose links changed belongs to the block
 * of the starting site of its first changed link in the order (x,mu),
 * (x+mu,nu), (x+nu,mu), (x,nu) (a link changed when any of its numbers
 * differs); the sum over blocks is the change of S_w.  It is the term
 * psms_filter_params.beta_block multiplies.  FP64, deterministic;
 * synchronises the context's stream. */
psms_status psms_block_action_change(psms_ctx *ctx, int field_old, int field_new, double *ds_host);

/* Exact ln|det D_b(U_field)| of every Dirichlet block (Sec. 3: the paper
 * takes small-block determinants by LU), lexicographic block index, into
 * out_host[n_blocks]: det D_b = A^{n_e} det(Dhat_b) with A = 4 + m0 and
 * Dhat_b = A - D_oe D_eo / A the even-odd reduced block operator (n x n
 * complex, n = 6 x block volume), factorised by batched FP64 LU with
 * partial pivoting on the device.  Cost about (8/3) n^3 FP64 flop per block
 * (1e10 for a 4^4 block); device memory n^2 x 16 B per block of a batch
 * (batches sized from the free memory, psms_max_chunk caps them).
 * PSMS_ESPECTRUM if a block operator is singular (non-finite result);
 * PSMS_EINVAL for blocks of more than 1024 sites.  Synchronises the
 * context's stream. */
psms_status psms_block_logdet(psms_ctx *ctx, int field, double *out_host);

/* ---- recursive domain decomposition (Eq. (ddrec), the 5-step filter) --------
 * psms_set_outer_blocks: outer blocks of extents outer[4] tiled by the
 * context's blocks (outer = NULL or outer[0] = 0: off).  Each outer extent
 * must be an even multiple of the block extent and divide the lattice
 * extent an even number of times (PSMS_EINVAL otherwise).  With outer
 * blocks set:
 *  - psms_logdet_ratio(level = PSMS_LEVEL_SUB) estimates, for every outer
 *    block b, ln |det D-hat_b(U) / det D-hat_b(U')|^2 with D-hat_b the Schur
 *    complement of b's black and white blocks (Dirichlet on b's faces):
 *    Eq. (staccN) with M_i = (1 - P_b Q_b(U_{i+1}))^-1 (1 - P_b Q_b(U_i)) on
 *    range(P_b), P_b the projector onto the faces of black blocks that lie
 *    inside b; noise stream level 4; delta_out[b*n + i], b the lexicographic
 *    outer block index;
 *  - psms_logdet_ratio(level = PSMS_LEVEL_OUTER_GLOBAL) estimates the
 *    global Schur complement of the outer decomposition (Eq. (ddfactor)
 *    with the outer blocks as the blocks; noise stream and decision
 *    counter of PSMS_LEVEL_GLOBAL), delta_out[i];
 *  - psms_filter_step with n_sub >= 1 runs the filter with one level of
 *    recursion (Eq. (4step)): after the block level, every outer block with
 *    an accepted block is accepted with min{1, exp(-Delta_b)},
 *    Delta_b = beta_sub sum dS_w (its accepted blocks) + the SUB estimate
 *    between U and the field after the block level (counter (step, 4, b);
 *    one decision on the sum for block extents <= 2); an outer block none
 *    of whose accepted blocks changed a link has Delta_b = 0 and is not
 *    estimated (its det D-hat_b is unchanged, Eq. (ddrec)); a rejected
 *    outer block restores all its blocks; the global level then uses the
 *    outer blocks (PSMS_LEVEL_OUTER_GLOBAL).  With the learned level the
 *    inner blocks pass it first; with relative gauge fixing stage 2 and the
 *    global level interpolate between the stage-1 endpoints merged on the
 *    accepted inner blocks.  Not combined with the HYP options or the exact
 *    block level (PSMS_EINVAL). */
psms_status psms_set_outer_blocks(psms_ctx *ctx, const int *outer);

/* ---- HYP-smeared links and the block HYP plaquette action (App. C, Sec. 5) ----
 * One level of HYP smearing of gauge slot `field`: three steps, each a
 * weighted sum of a link and its staples projected onto SU(3), confined to
 * the hypercubes attached to the link, with parameters alpha = (a1, a2, a3)
 * (NULL: (0.75, 0.6, 0.3), the HYP construction's; each must lie in
 * [0, 1], else PSMS_EINVAL).  The projection is the unitary polar factor
 * with the determinant's phase removed by the principal cube root.  FP64.
 *
 * psms_hyp_smear writes the fat links to links_dev (canonical layout,
 * 4V x 9 complex doubles, caller-owned device memory).
 *
 * psms_hyp_block_action writes S_HYP,b for every block (lexicographic
 * block index) to s_host[n_blocks]: Eq. (Sw) without beta on the fat links,
 * restricted to the plaquettes whose four corners lie in block b.  With
 * blocks of extent >= 3 it depends only on the block's active links and on
 * links that are never active, so its change factorises over blocks.
 * PSMS_ESPECTRUM if a smearing sum was singular (non-finite result).
 * Synchronises the context's stream. */
psms_status psms_hyp_smear(psms_ctx *ctx, int field, const double *alpha, double *links_dev);
psms_status psms_hyp_block_action(psms_ctx *ctx, int field, const double *alpha, double *s_host);

/* ---- coefficients of the parametrised levels (App. C) ------------------------
 * Host functions: no context, no device memory, no kernel; callable without
 * a GPU.  They return a status only (psms_last_error needs a context).
 *
 * psms_level_covariance: C^(jk) of Eq. (sigmaDeltaSiparams) from n_samples
 * rows of n_actions action changes (Delta S^(0), ..., Delta S^(i)), samples
 * row-major [n_samples][n_actions]; cov receives the n_actions x n_actions
 * matrix (row-major), normalised by n_samples.  PSMS_EINVAL for null
 * pointers, n_samples < 2, n_actions outside 1..64 or a non-finite sample.
 *
 * psms_level_coefficients: the coefficients beta_i^(j) of Eq. (Si) for
 * levels i = 0..n_levels (level 0 is the pure-gauge proposal), written to
 * beta as a row-major (n_levels+1)^2 lower-triangular matrix, row i =
 * level, column j = action.  covs packs the covariance of level i = 1..n
 * ((i+1) x (i+1), actions 0..i, row-major) one after the other; targets[j]
 * is beta^(j), the value every action's coefficients must sum to (the
 * plaquette's beta, 0 for an auxiliary action, 1 for a determinant);
 * stochastic (optional, n_levels+1 flags) marks actions estimated
 * stochastically, which take no coefficient at later levels.  From the last
 * level down the level's own coefficient follows from its target and the
 * free ones minimise the level's variance beta^T C_i beta, i.e. solve
 * sum_k C^(jk) beta_i^(k) = -C^(ji) beta_i^(i) (Eq. (paramsi) read as the
 * stationarity condition of Eq. (sigmaDeltaSiparams)); beta_0^(0) closes the
 * plaquette constraint.  PSMS_EINVAL for null pointers, n_levels outside
 * 1..63, a non-finite input or a singular system of free actions. */
psms_status psms_level_covariance(const double *samples, long long n_samples, int n_actions, double *cov);
psms_status psms_level_coefficients(int n_levels, const double *covs, const double *targets,
                                    const int *stochastic, double *beta);

/* Device memory the context holds in scratch buffers (bytes, host output);
 * it grows when a call needs more and is freed with the context. */
psms_status psms_scratch_bytes(const psms_ctx *ctx, size_t *bytes);

/* Number of CUDA kernels the library has launched in this process. */
long long psms_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* PSMS_H */
