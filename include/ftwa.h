/*
 * ftwa.h -- C ABI of the GB300 (sm_103a) fTWA library.
 *
 * The library integrates many independent phase-space samples of the
 * fermionic truncated Wigner approximation (fTWA) for the Fermi-Hubbard
 * model of Rousse, Eriksson and Ogren (arXiv:2212.04352):
 *
 *   H = - sum_{ij s} j_ij c+_is c_js + U sum_i n_i,up n_i,dn         (Eq. 1)
 *
 * with nearest-neighbour hoppings j_ij = t_b on the bonds of a lattice of
 * degree <= 3 and on-site U.  A sample is one complex one-body matrix
 * rho_ij,s per spin s, drawn from the Gaussian Wigner distribution of a
 * diagonal initial state (Eq. 7) and advanced by the fTWA equation of
 * motion (Eq. 6)
 *
 *   d/dt rho_s = i (rho_s J - J rho_s) + i U (D_sbar rho_s - rho_s D_sbar),
 *   D_sbar = diag(Re rho_kk,sbar + 1/2),
 *
 * with classical RK4 (the paper names no integrator).  Occupations and
 * density-density correlators are sample means (Eqs. 5 and 10).
 *
 * Conventions (all entry points):
 *  - Every call returns an int status: FTWA_OK (0) or a negative FTWA_ERR_*
 *    code.  No call aborts or throws.
 *  - Pointers named *_dev are device pointers; every other pointer is host
 *    memory.  The caller owns every state, snapshot and output buffer; the
 *    plan owns only its constant tables and its internal workspace.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued asynchronously on it; host-side
 *    argument errors are reported synchronously before anything is enqueued.
 *  - Errors raised inside a kernel (a bounded wait that timed out, a
 *    non-finite value) are recorded in the plan's device status word and
 *    returned by ftwa_status().
 *  - State layout at the ABI ("rho_dev"): [M][2][N][N] complex, row-major,
 *    interleaved (re, im), in the plan's precision (double for FTWA_FP64,
 *    float for FTWA_FP32).  Index s = 0 is spin up, s = 1 spin down.  Only the
 *    upper triangle i <= j is read on input (the state is Hermitian); the
 *    full Hermitian matrix is written on output.
 *  - Snapshot layout ("snap_dev"): [n_out][M][2N] real, plan precision,
 *    X[t][m][s*N + i] = Re rho_ii,s of sample m after t*out_every steps,
 *    n_out = n_steps / out_every + 1 (row 0 is the initial state).
 */
#ifndef FTWA_H
#define FTWA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FTWA_OK                     0
#define FTWA_ERR_INVALID_ARGUMENT  -1  /* null pointer, bad size, bad value   */
#define FTWA_ERR_UNSUPPORTED       -2  /* degree > 3, N above the limit, ...  */
#define FTWA_ERR_OUT_OF_MEMORY     -3  /* device allocation failed            */
#define FTWA_ERR_CUDA              -4  /* a CUDA runtime call failed          */
#define FTWA_ERR_DEVICE_TIMEOUT    -5  /* a bounded in-kernel wait gave up    */
#define FTWA_ERR_NONFINITE         -6  /* a kernel produced NaN/Inf           */

/* ---- precision and Gram modes ------------------------------------------ */
#define FTWA_FP64          0   /* state and arithmetic in double             */
#define FTWA_FP32          1   /* state and arithmetic in float              */
#define FTWA_GRAM_FP64     0   /* connected Gram in double (CUDA cores)      */
#define FTWA_GRAM_BF16X3   1   /* hi/lo bf16 split products on tcgen05 MMA   */

/* Largest lattice a plan accepts (sites). */
#define FTWA_MAX_SITES   256

typedef struct ftwa_plan ftwa_plan_t;

/* Lattice of Eq. 1: n_sites sites and n_bonds bonds (i, j), 0 <= i < j <
 * n_sites, unique; every site has at most 3 bonds.  t_bond (nullable) gives
 * j_ij per bond; when NULL every bond has hopping `t` (argument of
 * ftwa_plan).  Arrays are read during ftwa_plan only. */
typedef struct {
    int32_t n_sites;
    int32_t n_bonds;
    const int32_t *bonds;    /* host, [n_bonds][2] */
    const double *t_bond;    /* host, [n_bonds] or NULL */
} ftwa_lattice;

/* Diagonal initial state of Eq. 7: occupations n_i,s in [0, 1] (Fock
 * states use 0/1; fractional values describe a thermal diagonal state). */
typedef struct {
    const double *n_up;      /* host, [n_sites] */
    const double *n_dn;      /* host, [n_sites] */
} ftwa_init_state;

/* Options (zero-initialised = defaults: FP64, dt 0.01, out_every 10,
 * automatic launch shape). */
typedef struct {
    int32_t precision;        /* FTWA_FP64 or FTWA_FP32                       */
    double dt;                /* RK4 step in units of hbar/t (> 0)            */
    int32_t out_every;        /* snapshot cadence in steps (>= 1)             */
    int32_t cluster_override; /* CTAs per sample (1..8), 0 = automatic         */
    int32_t threads_override; /* threads per CTA: 0 (automatic: 512 for the
                                 tiled stepper, else 768) or 768; the tiled
                                 stepper (variant 3) also takes 512           */
    int32_t autotune;         /* 1 = time candidate shapes on first evolve     */
    uint64_t timeout_us;      /* limit of every bounded in-kernel wait in
                                 microseconds, 0 = default (5 s)             */
    int32_t variant;          /* stepper: 0 automatic, 1 banded (rows keep a
                                 mirror band of width = lattice bandwidth),
                                 2 general packed triangle, 3 tiled (FP32,
                                 on-site U: the banded layout in 32-column
                                 blocks at a fixed row stride)               */
} ftwa_options;

/* Launch shape chosen by the plan (for reporting and tests). */
typedef struct {
    int32_t n_sites, n_bonds, precision;
    int32_t cluster;          /* CTAs per sample                              */
    int32_t threads;          /* threads per CTA                              */
    int32_t samples_per_cta;  /* samples resident in one CTA (cluster == 1)   */
    int32_t smem_bytes;       /* dynamic shared memory per CTA                */
    int32_t tmem_cols;        /* tensor-memory columns per CTA                */
    int32_t grid_clusters;    /* persistent clusters launched                 */
    int32_t units_per_warp;   /* 32-lane work units per warp and sample slot  */
    int32_t variant;          /* stepper chosen: 1 banded, 2 general, 3 tiled */
} ftwa_plan_info;

/* Create a plan: validates the lattice and initial state, builds the
 * neighbour tables (degree <= 3, per-bond hopping) and uploads them to the
 * current device.  U is the on-site interaction of Eq. 1.  `filling`, when
 * > 0, must equal sum_i (n_up + n_dn) / (2 N) within 1e-9 (a consistency
 * check); when init is NULL a Neel state is built from the lattice's
 * two-colouring (sublattice of site 0 spin up) and `filling` must be 0.5.
 * On success *out receives a plan to be released with ftwa_destroy.
 * Errors: FTWA_ERR_INVALID_ARGUMENT (null out/lattice, bad bonds, n outside
 * [0,1], dt <= 0, filling mismatch, non-bipartite lattice without init),
 * FTWA_ERR_UNSUPPORTED (degree > 3, n_sites > FTWA_MAX_SITES or < 2),
 * FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
int ftwa_plan(const ftwa_lattice *lattice, double U, double t, double filling,
              const ftwa_init_state *init, const ftwa_options *opts, ftwa_plan_t **out);

/* Release a plan and its device tables (NULL is accepted). */
void ftwa_destroy(ftwa_plan_t *plan);

/* Report the plan's launch shape. */
int ftwa_get_info(const ftwa_plan_t *plan, ftwa_plan_info *info);

/* Eq. 7 (ic_fTWA): write M initial samples m = first_sample ..
 * first_sample + M - 1 into rho_dev ([M][2][N][N] complex, plan precision):
 * rho_ii,s = n_i,s - 1/2 and, for i < j, rho_ij,s = xi_ij,s sqrt((n_i,s +
 * n_j,s - 2 n_i,s n_j,s)/2), rho_ji,s = conj(rho_ij,s), xi standard complex
 * normal (E|xi|^2 = 1, the covariance of App. A.3).  xi comes from
 * Philox4x32-10 (Salmon et al., SC'11) with key (seed_lo, seed_hi) and
 * counter (m_lo, m_hi, s, p), p = i N - i(i+1)/2 + j - i - 1, followed by
 * Box-Muller on two 53-bit uniforms; sample m is a pure function of
 * (seed, m).  Errors: FTWA_ERR_INVALID_ARGUMENT (null plan/rho_dev with
 * M > 0, M < 0, first_sample < 0), FTWA_ERR_CUDA. */
int ftwa_sample(ftwa_plan_t *plan, uint64_t seed, int64_t first_sample, int64_t M,
                void *rho_dev, void *stream);

/* General (non-diagonal) initial state, App. A (the covariance of the
 * Gaussian Wigner density) with Eq. 7 applied in a diagonalising basis: the
 * one-body density matrix of spin s is n_s = V_s diag(lambda_s) V_s^dagger
 * with n_s,ij = <c^dagger_i c_j>.  Host arrays: lambda[2][N] eigen-occupations
 * in [0, 1]; v_re, v_im [2][N][N] row-major, column k of V_s the eigenvector
 * of lambda_s,k (v_im may be NULL for a real basis).  After this call
 * ftwa_sample draws rho~ by Eq. 7 with lambda (same Philox counters) and
 * writes rho = V rho~ V^dagger (mean n - 1/2); the rotation runs on the
 * device in the plan's precision and keeps a workspace of at most 256 MB.
 * lambda == NULL returns the plan to its diagonal initial state.  The plan
 * copies the arrays.  ftwa_adjoint is not available while a basis is set.
 * Errors: FTWA_ERR_INVALID_ARGUMENT (null plan or v_re, lambda outside
 * [0, 1], non-finite entries, V not unitary to 1e-10), FTWA_ERR_CUDA,
 * FTWA_ERR_OUT_OF_MEMORY. */
int ftwa_set_initial_basis(ftwa_plan_t *plan, const double *lambda, const double *v_re, const double *v_im);

/* Raw Philox4x32-10 words for counters (m_lo, m_hi, spin, p0 + q),
 * q = 0 .. count-1, key (seed_lo, seed_hi): out_dev[q][4] uint32.  Exposes
 * the integer stage of ftwa_sample for bit-exact checks. */
int ftwa_philox(uint64_t seed, int64_t m, int32_t spin, int64_t p0, int64_t count,
                uint32_t *out_dev, void *stream);

/* Eq. 6 (drho) with classical RK4: advance the M samples in rho_dev
 * (in place, [M][2][N][N] complex, plan precision) by n_steps steps of
 * size dt.  When snap_dev is not NULL, X[t][m][s*N+i] = Re rho_ii,s after
 * t*out_every steps is written for t = 0 .. n_steps/out_every ([n_out][M][2N],
 * plan precision).  Samples are processed by a persistent kernel; one
 * sample's state stays on chip (shared memory, split across a thread-block
 * cluster for large N; RK4 registers in tensor memory) for all n_steps.
 * Errors: FTWA_ERR_INVALID_ARGUMENT (null plan/rho_dev with M > 0, M < 0,
 * n_steps < 0), FTWA_ERR_UNSUPPORTED (no launch shape fits on chip),
 * FTWA_ERR_CUDA; in-kernel timeouts via ftwa_status. */
int ftwa_evolve(ftwa_plan_t *plan, void *rho_dev, int64_t M, int64_t n_steps,
                void *snap_dev, void *stream);

/* Time-dependent on-site drive (the time-dependent Hamiltonians that Sec. III
 * admits; e.g. a pulsed site potential): h_ii,s(t) += v_i,s(t) with
 * v_i,s(t) = amp[s][i] f(t), f(t) = exp(-(t - t0)^2 / (2 sigma^2))
 * cos(omega (t - t0) + phase) (sigma <= 0: no envelope).  Eq. 6 gains
 * i (v_i,s - v_j,s) rho_ij,s, evaluated at the RK4 stage times.  amp: host
 * [2][N] (copied); amp == NULL removes the drive.  While a drive is set,
 * ftwa_evolve / ftwa_evolve_at run the banded stepper (FTWA_ERR_UNSUPPORTED if
 * its shape does not fit), and ftwa_adjoint and ftwa_batch_create return
 * FTWA_ERR_UNSUPPORTED.  Errors: FTWA_ERR_INVALID_ARGUMENT (null plan,
 * non-finite values), FTWA_ERR_CUDA, FTWA_ERR_OUT_OF_MEMORY. */
int ftwa_set_drive(ftwa_plan_t *plan, const double *amp, double t0, double sigma, double omega, double phase);

/* Time-dependent hopping (a second form of the time-dependent Hamiltonians
 * that Sec. III admits): every j_ij of Eq. 1 is scaled by
 * m(t) = 1 + eps g(t), g(t) = exp(-(t - t0)^2 / (2 sigma^2))
 * cos(omega (t - t0) + phase) (sigma <= 0: no envelope), evaluated at the RK4
 * stage times; eps = 0 removes it.  Start times as in ftwa_evolve_at; the
 * same restrictions as ftwa_set_drive (banded stepper; no adjoint, no graph
 * batch).  Errors: FTWA_ERR_INVALID_ARGUMENT (null plan, non-finite values). */
int ftwa_set_hopping_drive(ftwa_plan_t *plan, double eps, double t0, double sigma, double omega, double phase);

/* Long-range interaction (Eq. 1 with a general u_ij; Eq. 6 with its sum over
 * k): u is a host [N][N] symmetric matrix (copied; u_ii is the on-site term
 * and replaces the plan's U).  Eq. 6 then uses the diagonal field
 * h_ii,s = sum_k u_ik (rho_kk,sbar + 1/2), a dense mat-vec per stage computed
 * on the device.  u == NULL returns to the on-site U.  While set,
 * ftwa_evolve runs the banded stepper (FTWA_ERR_UNSUPPORTED if its shape
 * does not fit) and ftwa_adjoint / ftwa_batch_create return
 * FTWA_ERR_UNSUPPORTED.  Errors: FTWA_ERR_INVALID_ARGUMENT (null plan,
 * non-finite or non-symmetric u), FTWA_ERR_CUDA, FTWA_ERR_OUT_OF_MEMORY. */
int ftwa_set_interaction(ftwa_plan_t *plan, const double *u);

/* ftwa_evolve from time t_start (the time of the state in rho_dev; only the
 * drive depends on it): stage times t_start + (step + c) dt, c = 0, 1/2,
 * 1/2, 1.  ftwa_evolve is ftwa_evolve_at with t_start = 0.  With a drive the
 * plan keeps a device table of 4 n_steps pulse values (grown on demand).
 * Errors: as ftwa_evolve, and FTWA_ERR_INVALID_ARGUMENT for a non-finite
 * t_start. */
int ftwa_evolve_at(ftwa_plan_t *plan, void *rho_dev, int64_t M, int64_t n_steps, double t_start, void *snap_dev,
                   void *stream);

/* Eqs. 5 and 10 (fTWA_moments, g2_fTWA) from snapshots snap_dev
 * ([n_times][M][2N], plan precision), accumulated in double:
 *   occ_dev[t][k]     = <n_k>(t) = mean_m X[t][m][k] + 1/2,   k = s*N + i
 *   conn_dev[t][k][l] = (1/M) sum_m (X_k - mu_k)(X_l - mu_l)  (connected
 *                       <n_k n_l> - <n_k><n_l> for k != l; the diagonal is
 *                       the sample variance of X_k)
 *   g2_dev[t][k][l]   = mean((X_k + 1/2)(X_l + 1/2)) / (<n_k><n_l>)  (Eq. 10;
 *                       nullable; the k == l entries are not a g2)
 * gram_mode FTWA_GRAM_FP64 forms the Gram in double; FTWA_GRAM_BF16X3 forms
 * it on the tensor cores from centred data split as x = hi + lo (bf16) with
 * products hi*hi + hi*lo + lo*hi in fp32, reduced across sample blocks in
 * double (FP32 plans only).  All outputs are device double arrays.  The
 * plan keeps a workspace for the means and the per-split partial tiles
 * (grown on demand).  Errors: FTWA_ERR_INVALID_ARGUMENT (null pointers,
 * M < 1, n_times < 1, bad mode), FTWA_ERR_UNSUPPORTED (BF16X3 on an FP64
 * plan), FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
int ftwa_moments(ftwa_plan_t *plan, const void *snap_dev, int64_t M, int32_t n_times,
                 double *occ_dev, double *conn_dev, double *g2_dev, int32_t gram_mode,
                 void *stream);

/* Discrete adjoint of the RK4 integration of Eq. 6.  The loss is given
 * through its gradient with respect to the occupations: the caller supplies
 * dL_docc_dev[t][k] = dL/d<n_k>(t) for the output rows t = 0 .. T (T =
 * n_steps/out_every, [T+1][2N] device doubles, k = s*N + i); for a loss
 * L(<n>) this is exact at the point where it was evaluated.  Samples
 * m = 0 .. M-1 of `seed` are regenerated exactly as ftwa_sample draws them
 * (Eq. 7), integrated forward with a checkpoint every ckpt_every steps, and
 * swept backward stage by stage (each segment replayed from its checkpoint).
 * Outputs (device doubles, overwritten; any may be NULL): grad_U_dev[1] =
 * dL/dU, grad_t_dev[n_bonds] = dL/dt_b in the lattice's bond order,
 * grad_n0_dev[2][N] = dL/dn_i,s through rho_ii(0) = n - 1/2 and through the
 * noise scale s_ij(n) of Eq. 7; pairs with s_ij = 0 (e.g. two filled or two
 * empty sites of a Fock state) are skipped, since n -> s_ij is not
 * differentiable there.  ckpt_every must divide n_steps and be a multiple of
 * out_every.  The plan keeps a per-CTA workspace (checkpoints, one replayed
 * segment, stage states; grown on demand).  Errors:
 * FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_UNSUPPORTED (lattice too large for
 * the per-sample tables, or a general initial basis is set),
 * FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
int ftwa_adjoint(ftwa_plan_t *plan, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every,
                 const double *dL_docc_dev, double *grad_U_dev, double *grad_t_dev,
                 double *grad_n0_dev, void *stream);

/* Discrete adjoint for losses of the occupations and of the connected
 * correlator of Eq. 5 (fTWA_moments): the caller supplies dL_docc_dev as for
 * ftwa_adjoint (or NULL) and dL_dconn_dev[t][k][l] = dL/dC_kl(t) ([T+1][2N][2N]
 * device doubles, any matrix, or NULL; not both NULL), with occ_dev[t][k] the
 * forward occupations <n_k>(t) of the same M samples (ftwa_moments' occ
 * output; required with dL_dconn_dev).  C_kl = (1/M) sum_m x_mk x_ml -
 * mu_k mu_l with x_mk = Re rho^m_kk and mu = occ - 1/2, so sample m's
 * diagonal entry j receives (1/M) sum_l (G_jl + G_lj)(x_ml - mu_l) at every
 * output row; a loss of <n_k n_l> or g2 (Eq. 10) reaches the library
 * through its chain rule onto occ and conn.  Everything else (samples,
 * checkpoints, outputs, errors) as for ftwa_adjoint; the plan also keeps a
 * workspace of (T+1)(2N)^2 doubles for the symmetrised G.  Errors:
 * FTWA_ERR_INVALID_ARGUMENT (both cotangents NULL, dL_dconn_dev without
 * occ_dev, or the conditions of ftwa_adjoint), FTWA_ERR_UNSUPPORTED,
 * FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
int ftwa_adjoint_corr(ftwa_plan_t *plan, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every,
                      const double *dL_docc_dev, const double *dL_dconn_dev, const double *occ_dev,
                      double *grad_U_dev, double *grad_t_dev, double *grad_n0_dev, void *stream);

/* Allocation-free variant of ftwa_moments with gram_mode FTWA_GRAM_FP64.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, such as applications whose device memory is owned
 * by another allocator (a framework's caching allocator, a pool sized at
 * start-up) and latency-critical loops that cannot accept cudaMalloc's
 * implicit device synchronisation.  It needs no plan and allocates nothing:
 * the caller passes the snapshots (snap_dev, [n_times][M][2 n_sites] of
 * `precision`) and the outputs, with the same layout and meaning as for
 * ftwa_moments (occ_dev [n_times][2N], conn_dev and the nullable g2_dev
 * [n_times][2N][2N], device doubles).  The only scratch, the per-time sample
 * means, is a static device array of FTWA_MOMENTS_NOALLOC_MAX_TK doubles
 * (1 MiB, held by every device that loads the library until the process
 * exits); n_times * 2 n_sites beyond that limit is rejected with
 * FTWA_ERR_UNSUPPORTED, and so is n_times > 65535.  Each call on a stream
 * that is not capturing looks up the array's device address
 * (cudaGetSymbolAddress) with the calling device current, so a device reset
 * or another current context between calls is followed; a call on a
 * capturing stream reuses the address of the last non-capturing call on the
 * device (FTWA_ERR_UNSUPPORTED if there was none), so make a first call
 * before any stream capture and do not reset the device between that call
 * and a capture.  Every call shares the array and overwrites the entries it
 * uses before reading them, so nothing needs clearing; calls whose work
 * overlaps on the GPU (other streams, other host threads) race on it and
 * must be serialised by the caller.  The means are plain FP64 sums in a
 * fixed order (for FP32 snapshots ftwa_moments uses an exact fixed-point sum
 * instead, so the two agree to rounding, about 1e-14, not bit for bit).
 * Errors: FTWA_ERR_INVALID_ARGUMENT (null snap/occ/conn, M < 1,
 * n_times < 1, n_sites outside [1, FTWA_MAX_SITES], bad precision),
 * FTWA_ERR_UNSUPPORTED (size limits), FTWA_ERR_CUDA. */
#define FTWA_MOMENTS_NOALLOC_MAX_TK  131072
int ftwa_moments_noalloc(const void *snap_dev, int32_t precision, int32_t n_sites, int64_t M, int32_t n_times,
                         double *occ_dev, double *conn_dev, double *g2_dev, void *stream);

/* Launch-shape autotuner: times every feasible stepper shape of the plan
 * (variant 1 banded / 2 packed triangle x CTAs per sample 1, 2, 4, 8) on a
 * probe integration of probe_steps steps of min(M, 8192) samples and pins the
 * fastest in the plan (ftwa_get_info reports it).  Synchronous: allocates
 * and frees a temporary state buffer and waits for the probes on `stream`.
 * Errors: FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_UNSUPPORTED (no feasible
 * shape), FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
int ftwa_autotune(ftwa_plan_t *plan, int64_t M, int32_t probe_steps, void *stream);

/* Batched launch of heterogeneous problems (lattices of uneven size,
 * several U): one CUDA graph whose branches are the persistent steppers of
 * the n plans (plans[i] advancing rho_dev[i], M[i] samples, n_steps steps,
 * snapshots into snap_dev[i] if snap_dev and snap_dev[i] are not NULL), all
 * launched by one ftwa_batch_launch.  Shapes are fixed when the batch is
 * created (run ftwa_autotune first to tune them); plans and buffers must
 * outlive the batch.  Errors: FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_UNSUPPORTED,
 * FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
typedef struct ftwa_batch ftwa_batch_t;
int ftwa_batch_create(ftwa_plan_t *const *plans, int32_t n, void *const *rho_dev, const int64_t *M, int64_t n_steps,
                      void *const *snap_dev, ftwa_batch_t **out);
/* One persistent kernel for a batch of heterogeneous problems: plans[i]
 * (FP32, on-site U, lattices of different sizes, any U) advances M[i] samples
 * in rho_dev[i] by n_steps RK4 steps of Eq. 6 (snapshots into snap_dev[i] as
 * for ftwa_evolve, if snap_dev and snap_dev[i] are not NULL).  Every
 * problem's samples are cut into batches of S_i samples (S_i as large as the
 * problem's tiled decomposition fits on chip for the batch's cluster size);
 * the (problem, batch) work items are ordered by cost, largest first, and the
 * launch's clusters (all co-resident clusters of the device) draw them from a
 * queue in device memory until it is empty.  The launch is captured in a CUDA
 * graph (the queue head's reset, then the kernel) replayed by
 * ftwa_batch_launch.  The cluster size is the smallest every problem fits;
 * with tune != 0 the cluster size (that and twice it) and the CTA size (512,
 * 768 threads) are picked by timing a probe of each on scratch states
 * (synchronous).  The batch owns copies of every table it needs; plans and
 * buffers must outlive it.  Errors: FTWA_ERR_INVALID_ARGUMENT,
 * FTWA_ERR_UNSUPPORTED (more than 24 problems, a plan that is not FP32 or has
 * a drive or long-range field, no decomposition on chip),
 * FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
int ftwa_batch_create_persistent(ftwa_plan_t *const *plans, int32_t n, void *const *rho_dev, const int64_t *M,
                                 int64_t n_steps, void *const *snap_dev, int32_t tune, ftwa_batch_t **out);
/* Replay the batch's graph on `stream`. */
int ftwa_batch_launch(ftwa_batch_t *batch, void *stream);
/* Release a batch (NULL is accepted). */
void ftwa_batch_destroy(ftwa_batch_t *batch);

/* Exact diagonalisation on the GPU (Sec. III.A and App. B, the paper's
 * reference method, for lattices of up to 24 sites): the state of Eq. 1 in
 * the basis of Slater determinants with fixed N_up, N_dn, propagated by
 * psi(t) = exp(-iHt) psi(0) (Schroedinger form) with a Chebyshev expansion
 * (truncated where the Bessel coefficients fall below 1e-17) over intervals
 * dt_out.  ftwa_ed_plan builds the hopping matrices of both species (CSR,
 * fermionic signs for spin-up orbitals ordered before spin-down ones, same
 * species counted between the two sites) and allocates four state vectors
 * (16 dim bytes each, dim = C(N, N_up) C(N, N_dn)).  Errors:
 * FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_UNSUPPORTED (N > 24),
 * FTWA_ERR_OUT_OF_MEMORY, FTWA_ERR_CUDA. */
typedef struct ftwa_ed ftwa_ed_t;
int ftwa_ed_plan(const ftwa_lattice *lattice, double U, int32_t n_up, int32_t n_dn, ftwa_ed_t **out);
void ftwa_ed_destroy(ftwa_ed_t *ed);
/* Basis size and the spectral map H~ = (H - b) / a of the Chebyshev series
 * (a, b may be NULL). */
int ftwa_ed_info(const ftwa_ed_t *ed, int64_t *dim, double *spectral_a, double *spectral_b);

/* Propagate the Fock state given by host occupations n_up, n_dn ([N], 0 or
 * 1, counts N_up, N_dn) and record, at t = k dt_out for k = 0 .. n_out,
 * occ_dev[k][s N + i] = <n_i,s> and (if nn_dev is not NULL)
 * nn_dev[k][a][b] = <n_a n_b> over the 2N site-spins a, b (device doubles;
 * the a = b entries hold <n_a>).  Asynchronous on `stream`; the plan's state
 * vectors are reused, so calls on one plan must not overlap.  Errors:
 * FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_CUDA. */
int ftwa_ed_evolve(ftwa_ed_t *ed, const double *n_up, const double *n_dn, double dt_out, int32_t n_out,
                   double *occ_dev, double *nn_dev, void *stream);

/* Synchronise `stream`, then return and clear the plan's device status word
 * (FTWA_OK, FTWA_ERR_DEVICE_TIMEOUT or FTWA_ERR_NONFINITE), or FTWA_ERR_CUDA
 * if the synchronisation itself failed. */
int ftwa_status(ftwa_plan_t *plan, void *stream);

/* Test hook for the timeout path.  While armed (1), every CTA of the next
 * ftwa_evolve first waits, with the plan's bounded-wait limit, on an
 * mbarrier that nothing arrives at; the wait runs out, the kernel records
 * FTWA_ERR_DEVICE_TIMEOUT, skips its work and exits cleanly (the state
 * buffer is left unchanged).  Disarm with 0. */
int ftwa_debug_force_timeout(ftwa_plan_t *plan, int32_t armed);

/* Micro-benchmark of an on-chip peak of the current device, for the
 * roofline denominators of the stepper (not part of the method): kind 0 =
 * FP32 fused multiply-add rate (flop/s, scalar FFMA), 3 = the same with
 * packed pairs (__ffma2_rn), 1 = FP64 FMA rate (flop/s), 2 = shared-memory
 * load bandwidth (bytes/s, conflict-free 16-byte loads, all SMs).  Best of
 * five timed launches on `stream`; synchronous; allocates a small sink
 * buffer.  Errors: FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_CUDA. */
int ftwa_measure_peak(int32_t kind, double *value, void *stream);

/* Host-only consistency check of the tiled stepper's work decomposition
 * (variant 3; the stage state of Eq. 6 split over `cluster` CTAs with
 * `slots` samples each): every shared-memory address the kernel forms for
 * one slot is simulated on the host and checked — reads of active lanes hit
 * the intended element of Eq. 6 (the lane's own element for an empty
 * neighbour slot), all reads stay inside the addressed CTA's buffer, every computed
 * element of the upper triangle is written exactly once per stage and every
 * mirror-band entry exactly once.  Needs no device.  Lattice arguments as
 * for ftwa_plan (t_bond may be NULL: uniform 1).  *violations receives the
 * number of failed checks, msg (if not NULL) a description of the first.
 * Errors: FTWA_ERR_INVALID_ARGUMENT, FTWA_ERR_UNSUPPORTED (no decomposition
 * of that cluster size and slot count). */
int ftwa_debug_tile_check(int32_t n_sites, int32_t n_bonds, const int32_t *bonds, const double *t_bond,
                          int32_t cluster, int32_t slots, int64_t *violations, char *msg, int32_t msg_len);

/* Human-readable text of a status code (static storage). */
const char *ftwa_error_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int ftwa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FTWA_H */
