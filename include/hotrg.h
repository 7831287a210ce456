/*
 * hotrg.h -- C ABI of libhotrg, a GB300 (sm_103a) implementation of the HOTRG
 * coarse-graining step for 2D classical lattice models.
 *
 * The method: the partition function of a 2D spin model is the contraction of
 * N copies of a local tensor, Z = Tr T^N (Sec. II.A, Eq. 2).  One HOTRG step
 * contracts two neighbouring tensors along one bond, fuses the two parallel
 * legs that result and cuts each fused leg back to at most D_cut states by a
 * higher-order SVD that reduces to the SVD of a reshaped matrix (Sec. II.A),
 * here the eigendecomposition of the Hermitian Gram matrix of that reshaped
 * matrix (the Hermitian case of Eq. 5).  Contraction and SVD are the two
 * steps that carry the cost (Sec. II.A, last paragraph).
 *
 * Conventions used throughout:
 *   - A tensor T[x, x', y, y'] has legs (left, right, down, up) and shape
 *     (Dx, Dx, Dy, Dy), stored row-major in FP64 (y' fastest).
 *   - A Y step contracts the up leg of a lower tensor with the down leg of an
 *     upper tensor and cuts the fused x legs; an X step does the same along x
 *     and cuts the fused y legs.  The same isometry U projects both fused legs.
 *   - U is taken from the left or the right environment (Gram matrix of the
 *     two unfoldings of the contracted pair), whichever discards the smaller
 *     eigenvalue weight; ties go to the left.  If Dx^2 <= D_cut nothing is cut.
 *   - After every step the tensor is divided by its max-norm c_n and
 *     ln(c_n) / 2^n is added to an FP64 log-sum; the initial tensor is scaled
 *     by c_0 = max|T0| the same way.  After n steps the network holds 2^n
 *     sites and ln Z / N = logsum + ln(Tr T_n) / 2^n, Tr the periodic trace.
 *
 * Ownership and errors:
 *   - Every host buffer stays owned by the caller; the library copies what it
 *     needs before returning.  A context owns all device memory it uses and
 *     releases it in hotrg_destroy.
 *   - No C++ exception crosses this interface.  Every call returns a status;
 *     the first error seen by a context is latched: later calls on it return
 *     the same status without doing work, and hotrg_last_error() returns a
 *     message.  A NULL context pointer gives HOTRG_EINVAL.
 *   - hotrg_step enqueues work on the context's stream and synchronises that
 *     stream during the step (the eigensolver's convergence checks) and once
 *     at its end, where device-side errors of the step are reported.
 *   - A context may be used by one host thread at a time.
 */
#ifndef HOTRG_H
#define HOTRG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hotrg_ctx hotrg_ctx;

typedef enum {
  HOTRG_OK = 0,
  HOTRG_EINVAL = 1,      /* bad argument (NULL pointer, size, enum value)            */
  HOTRG_ENOMEM = 2,      /* device or host allocation failed                         */
  HOTRG_ECUDA = 3,       /* CUDA runtime or library error                            */
  HOTRG_EEIG = 4,        /* the eigensolver did not converge or rejected its input    */
  HOTRG_ENONFINITE = 5,  /* max-norm or trace is zero, negative or not finite         */
  HOTRG_ETIMEOUT = 6,    /* a bounded device wait ran out                            */
  HOTRG_ESTATE = 7,      /* call not valid in the context's current state            */
  HOTRG_EBOUNDS = 8      /* a mapped index fell outside its buffer: reported only by a
                            library built with -DHOTRG_CHECKED=1 (bounds-checked build,
                            in which every mapped access of the GEMM, gather and epilogue
                            kernels is checked, and a bad one skipped, not performed) */
} hotrg_status;

typedef enum { HOTRG_DIR_X = 0, HOTRG_DIR_Y = 1 } hotrg_dir;

/*
 * Arithmetic of the contraction GEMMs (environment partials, Gram combine,
 * projection chain).  The environment eigendecomposition, the max-norm, the
 * log-sum and the trace are FP64 in every mode.
 *   HOTRG_FP64    FP64 SIMT GEMMs (the plain reference path on the GPU).
 *   HOTRG_TF32    tcgen05 kind::tf32 tensor-core GEMMs, FP32 accumulation.
 *   HOTRG_BF16X3  tcgen05 kind::f16 with each operand split into two BF16
 *                 terms a = a_hi + a_lo; products hi*hi + hi*lo + lo*hi,
 *                 FP32 accumulation.
 *   HOTRG_BF16X6  three-term BF16 split a = a1 + a2 + a3; the six products
 *                 whose term indices sum to at most 4, FP32 accumulation.
 *   HOTRG_BF16XS  exact-slice products (see hotrg_dgemm_emu) with S base-64
 *                 digits (S = 6 unless HOTRG_OPT_XS_DIGITS says otherwise):
 *                 every operand row is scaled by a power of two and rounded to
 *                 6S bits, the digit products are exact and their leading sums
 *                 accumulate exactly on the tensor cores (K split into parts of
 *                 at most 2336), intermediates are FP64.  About 2^-(6S+1) per
 *                 term relative to the row maxima; aimed at free energies
 *                 within 1e-9 of the FP64 result.
 */
typedef enum {
  HOTRG_FP64 = 0, HOTRG_TF32 = 1, HOTRG_BF16X3 = 2, HOTRG_BF16X6 = 3, HOTRG_BF16XS = 4
} hotrg_prec;

/* Per-step diagnostics (all gauge-invariant except ln_c, see hotrg_step_info). */
typedef struct {
  int dir;          /* HOTRG_DIR_X or HOTRG_DIR_Y                                  */
  int Dx;           /* dimension of the fused legs before the step (step's view)   */
  int Dy;           /* dimension of the contracted legs                            */
  int Dn;           /* kept dimension D' = min(Dx^2, D_cut)                         */
  int side;         /* 0 = left env chosen, 1 = right, -1 = nothing cut (U = I)    */
  double ln_c;      /* ln max|T'| before the rescale                               */
  double eps_L;     /* Tr G_L - sum of its D' leading eigenvalues (discarded weight) */
  double eps_R;     /* same for G_R                                               */
  double cut_gap;   /* (lambda_D' - lambda_{D'+1}) / lambda_1 of the chosen side, or
                       +inf when nothing is cut                                     */
  double trace_G;   /* Tr G_L (= ||M||_F^2)                                        */
  int eig_path;     /* eigensolver used: 0 none (no cut), 1 direct Jacobi,
                       2 subspace iteration                                         */
  int eig_iters;    /* subspace iterations (path 2)                                */
  double eig_residual; /* max_i<=D' ||G u_i - lambda_i u_i|| / lambda_1 (path 2)    */
  int eig_rr;       /* Rayleigh-Ritz steps of the subspace iteration (path 2)      */
  int eig_sweeps;   /* most rounds of the FP64 finishing Jacobi of one Rayleigh-Ritz
                       step (path 2): rotations still needed after the first-order
                       corrections (0: none)                                        */
  int eig_sweeps32; /* most FP32 Jacobi sweeps of one Rayleigh-Ritz step (path 2)  */
} hotrg_step_info_t;

/*
 * Initial tensors (Sec. II.A, Eq. 2: the local tensor whose N-fold contraction
 * is Z).  T0[x,x',y,y'] = sum_s w_s W[s,x] W[s,x'] W[s,y] W[s,y'] with W the
 * symmetric square root of the bond Boltzmann matrix B and w_s the site weight.
 *   Ising (J = 1, s = +1, -1 at index 0, 1): B[s,s'] = exp(beta s s'),
 *     w_s = exp(beta h s); T0_out receives 16 doubles.  Needs beta > 0.
 *   Potts (q states, J = 1, no field): B[s,s'] = exp(beta delta_{ss'}), w = 1;
 *     T0_out receives q^4 doubles.  Needs beta > 0 and 2 <= q <= 16.
 * Host-only; no device is touched.  Returns HOTRG_EINVAL on bad arguments.
 */
hotrg_status hotrg_ising_tensor(double beta, double h, double *T0_out);
hotrg_status hotrg_potts_tensor(int q, double beta, double *T0_out);

/*
 * Quantum chains (Sec. II.A: the spin-1/2 antiferromagnetic Heisenberg chain;
 * Sec. II.B: Z = Tr exp(-beta H) of a quantum chain maps onto a 2D classical
 * network with an imaginary-time direction, contracted by HOTRG).
 *
 * hotrg_xxz_tensor: the cell tensor of the XXZ chain
 *   H = sum_i Jxy (Sx_i Sx_i+1 + Sy_i Sy_i+1) + Jz Sz_i Sz_i+1
 * (Jxy = Jz = 1: the antiferromagnetic Heisenberg chain) under the checkerboard
 * Trotter product Z_M = Tr (exp(-tau H_odd) exp(-tau H_even))^M, beta = M tau.
 * One cell is two neighbouring sites (e, o) over one period; T0_out receives
 * 256 doubles, T[x][x'][y][y'] with
 *   y = 2 s_e + s_o  the two spins at the start of the period, y' at its end
 *                    (s = 0: Sz = +1/2, s = 1: Sz = -1/2);
 *   x, x'            the virtual bonds of the odd-bond gates that leave the
 *                    cell on the left and on the right (dimension 4).
 * The bond gate g = exp(-tau h) is expanded as sum_k c_k P_k (x) P_k over the
 * real one-site basis P = (I, sigma_x, [[0,1],[-1,0]], sigma_z); the left site
 * of a bond carries sqrt|c_k| P_k and the right site sign(c_k) sqrt|c_k| P_k.
 *   T[x][x'][(e0 o0)][(e2 o2)]
 *     = sum_{e1,o1} g[(e1 o1)][(e0 o0)] B_x[e2][e1] A_x'[o2][o1]
 * with A_k = sqrt|c_k| P_k, B_k = sign(c_k) sqrt|c_k| P_k.  Needs tau > 0 and
 * finite couplings.  Host-only; returns HOTRG_EINVAL on bad arguments.
 *
 * Schedule of a finite-temperature run (create with D0 = 4):
 *   n_t Y steps   compose imaginary time: beta = 2^n_t tau;
 *   hotrg_trace_y closes the time direction (Z_M is a trace over the
 *                 time-boundary states);
 *   n_x X steps   multiply the closed column matrices: a ring of 2^(n_x + 1)
 *                 sites, the thermodynamic limit as n_x grows.
 * Then ln Z / N_cells = hotrg_log_z_per_site and the free energy per site is
 * f = -(ln Z / N_cells) / (2 tau), i.e. hotrg_free_energy with beta = 2 tau.
 */
hotrg_status hotrg_xxz_tensor(double Jxy, double Jz, double tau, double *T0_out);

/*
 * Close the y direction of every instance of the context:
 *   T[x][x'][0][0] <- sum_y T[x][x'][y][y]   (Dy becomes 1),
 * then the max-norm rescale; ln(c) enters the log-sum with the weight 2^-n of
 * the n steps taken so far (the traced tensor still stands for 2^n sites).  It
 * is not a step: hotrg_dims' step count and the step records are unchanged.
 * Later X steps have trivial fused legs (nothing is cut) and multiply the
 * Dx x Dx column matrices, on the FP64 GEMMs in every precision mode.
 * Synchronises the stream.  Errors: HOTRG_EINVAL (NULL), a sticky context
 * error, HOTRG_ENONFINITE if the traced tensor is zero or not finite.
 */
hotrg_status hotrg_trace_y(hotrg_ctx *ctx);

/*
 * iTEBD ground states of the XXZ chain (Sec. II.A, Eq. 1: the two-site-cell
 * matrix-product state ... lambda_2 A lambda_1 B lambda_2 ..., driven to the
 * ground state by imaginary-time gates U = exp(-tau h); the truncation is an SVD
 * taken, as in Sec. II.B, from the two-sided Jacobi eigendecomposition of a
 * Hermitian matrix: here the bond's reduced density matrix theta^T theta).
 *
 * A context holds n independent chains with the same bond cap D_b; chain i has
 * couplings[3i .. 3i+2] = (Jxy, Jz, tau), h as for hotrg_xxz_tensor.  The state
 * of a chain is (P, Q, lam): P[i][a][j] (outer x 2 x mid) and Q[j][b][m]
 * (mid x 2 x outer), row-major FP64, in right-canonical form (Gamma lambda), and
 * lam the Schmidt values on P's left bond (outer of them); a = 0 is Sz = +1/2.
 * One update applies U to the (P, Q) bond:
 *   phit = U (P Q), theta = lam[i] phit as a (2 outer) x (2 outer) matrix,
 *   Y, w = leading D' = min(D_b, 2 outer) eigenpairs of theta^T theta,
 *   lam' = sqrt(w) / |sqrt(w)|, P' = phit Y / |sqrt(w)| (the state stays
 *   normalised under the non-unitary gate), Q' = Y^T,
 * and continues with (P, Q, lam) <- (Q', P', lam') on the other kind of bond.
 *
 * hotrg_itebd_create: 1 <= n <= 65535, 1 <= D_b <= 48, tau > 0, finite
 *   couplings.  P0s / Q0s / lam0s: per chain, host arrays of D0*2*D0, D0*2*D0
 *   and D0 doubles (borrowed, copied), or all NULL for the Neel state
 *   (P = |up>, Q = |down>, D0 must be 1).  The other bond's Schmidt values start
 *   uniform, 1/sqrt(D0).  stream: a cudaStream_t (NULL = legacy default).  All
 *   device memory is allocated here (HOTRG_ENOMEM if it does not fit).
 * hotrg_itebd_step: nsteps updates of every chain; synchronises once at the
 *   end; HOTRG_ENONFINITE if a bond's density matrix lost all positive weight.
 * hotrg_itebd_energy: energy per site of every chain into out_n[n]: the mean
 *   of <theta|h|theta>/<theta|theta> over the two bonds, theta = lam (P Q) and
 *   lam_other (Q P) (the Schmidt values of each bond's left neighbour).
 * hotrg_itebd_lambda: the current lam of chain inst (cap >= outer); *n = outer.
 * hotrg_itebd_discarded: discarded weight sum_{k >= D'} w_k / sum_k w_k of
 *   chain inst's last update (0 before the first).
 * hotrg_itebd_dims: outer and mid bond dimensions and the updates taken.
 * Errors are sticky per context, as for hotrg_ctx.
 */
typedef struct hotrg_itebd hotrg_itebd;

hotrg_status hotrg_itebd_create(int n, const double *couplings, int D_b, int D0,
                                const double *const *P0s, const double *const *Q0s,
                                const double *const *lam0s, void *stream, hotrg_itebd **out);
hotrg_status hotrg_itebd_step(hotrg_itebd *ctx, int nsteps);
hotrg_status hotrg_itebd_energy(hotrg_itebd *ctx, double *out_n);
hotrg_status hotrg_itebd_lambda(hotrg_itebd *ctx, int inst, double *buf, int cap, int *n);
hotrg_status hotrg_itebd_discarded(hotrg_itebd *ctx, int inst, double *out);
hotrg_status hotrg_itebd_dims(hotrg_itebd *ctx, int *outer, int *mid, long long *nsteps);
const char *hotrg_itebd_last_error(const hotrg_itebd *ctx);
void hotrg_itebd_destroy(hotrg_itebd *ctx);

/*
 * Create a context holding T0 (host, D0^4 doubles, [x,x',y,y'] row-major,
 * borrowed and copied) scaled by its max-norm, ready for steps with cut D_cut.
 * T0 is the local tensor of Sec. II.A, Eq. 2 (Z = Tr T^N): the network of N
 * copies of it is the partition function the steps coarse-grain; c_0 = max|T0|
 * starts the FP64 log-sum with weight 1 (one site).
 * stream: a cudaStream_t (NULL = the legacy default stream); the context
 * enqueues all its work there.  All device memory for steps up to D_cut is
 * allocated here (HOTRG_ENOMEM if it does not fit).  On failure *out is set to
 * NULL.  Requires 1 <= D0 <= 64, 1 <= D_cut <= 64; a T0 whose max-norm is zero
 * or not finite gives HOTRG_ENONFINITE.
 */
hotrg_status hotrg_create(const double *T0, int D0, int D_cut, hotrg_prec prec,
                          void *stream, hotrg_ctx **out);

/*
 * One coarse-graining step in direction dir (Sec. II.A): environments, FP64
 * eigendecomposition and choice of U, projection T' = U^T (T.T) U, max-norm
 * rescale and log-sum update.  See the header comment for the synchronisation.
 * The leading D'+1 eigenpairs of each environment come from a batched FP64
 * eigensolver (both environments at once): for Dx^2 <= 96 a parallel two-sided
 * Jacobi diagonalisation of the whole matrix (Sec. II.B, Eqs. 5-6), otherwise
 * block subspace iteration with Rayleigh-Ritz steps solved by the same Jacobi
 * method, stopped at a residual of 1e-12 relative to the largest eigenvalue.
 * If that bound is not reached within HOTRG_OPT_EIG_MAX_ITERS iterations the
 * step fails with HOTRG_EEIG (latched; the context keeps the state of the last
 * completed step).
 */
hotrg_status hotrg_step(hotrg_ctx *ctx, hotrg_dir dir);

/*
 * ln Z / N after the steps taken so far (Sec. II.A, Eq. 2: Z = Tr T^N over the
 * N = 2^n sites the n steps have fused): logsum + ln(Tr T_n) / 2^n, with Tr the
 * periodic trace over both leg pairs of the normalised tensor.  Synchronises
 * (one small D2H read).  HOTRG_ENONFINITE if the trace is not positive;
 * HOTRG_ESTATE on a context with more than one instance.
 */
hotrg_status hotrg_log_z_per_site(hotrg_ctx *ctx, double *out);

/*
 * Free energy per site f = -(1/beta) ln Z / N (Sec. II.A, Eq. 2, Z = Tr T^N;
 * J = 1).  beta must be > 0 (HOTRG_EINVAL otherwise).  Synchronises; errors as
 * for hotrg_log_z_per_site.
 */
hotrg_status hotrg_free_energy(hotrg_ctx *ctx, double beta, double *f_out);

/* Diagnostics of step `step` (0-based, < number of steps taken). */
hotrg_status hotrg_step_info(hotrg_ctx *ctx, int step, hotrg_step_info_t *out);

/*
 * Normalised spectrum lambda_i / lambda_1 (descending) of the chosen
 * environment of step `step`: the D' kept values, plus lambda_{D'+1} when a
 * cut was made.  Writes min(cap, count) values to buf and the count to *n.
 */
hotrg_status hotrg_spectrum(hotrg_ctx *ctx, int step, double *buf, int cap, int *n);

/*
 * Copy the current normalised tensor to host memory (FP64, [x,x',y,y']
 * row-major).  dims[4] receives (Dx, Dx, Dy, Dy); cap is the capacity of
 * host_out in doubles (HOTRG_EINVAL if too small; dims are still written).
 */
hotrg_status hotrg_get_tensor(hotrg_ctx *ctx, double *host_out, long long cap, int dims[4]);

/*
 * Copy the isometry U of the last step to host memory, column-major
 * (rows = Dx^2 fused index (x1 x2) with x1 slower, cols = D'), and its shape.
 */
hotrg_status hotrg_get_isometry(hotrg_ctx *ctx, double *host_out, long long cap,
                                int *rows, int *cols);

/* Current bond dimensions (Dx, Dy) and number of steps taken. */
hotrg_status hotrg_dims(hotrg_ctx *ctx, int *Dx, int *Dy, int *nsteps);

/*
 * Context options (set between steps; they take effect at the next step).
 *   HOTRG_OPT_EIG_TC_PRODUCTS  1 (default): the eigensolver's products G X run
 *       on the BF16 tensor cores as exact-slice FP64-grade GEMMs (eight base-64
 *       digits per operand row, see hotrg_dgemm_emu); 0: FP64 SIMT kernels.
 *       Either way the eigenpairs meet the same residual bound.
 *   HOTRG_OPT_XS_DIGITS  4..8 (default 6): digits per operand row in the
 *       HOTRG_BF16XS contraction mode (digit products per K step: S(S+1)/2).
 *   HOTRG_OPT_GEMM_AUTOTUNE  1 (default) / 0: the first tensor-core GEMM of
 *       each shape times every tile width (64, 128, 256 columns) on the
 *       context's stream and keeps the fastest; 0 uses a fixed rule.  The
 *       choice never changes results.  Process-wide: it applies to every
 *       context, and the tuned widths are kept until the process exits.
 *   HOTRG_OPT_GRAPHS  1 (default) / 0: the tensor-core contraction chains of
 *       a step (environment, projection) are captured into CUDA graphs the
 *       second time a (direction, bond dimensions, buffer) combination occurs
 *       and replayed afterwards (with the stage profiler on, its events are
 *       part of the graph).  Needs a non-NULL stream (not the legacy default
 *       stream); results are bit-identical either way.
 *   HOTRG_OPT_EIG_MAX_ITERS  1..1000 (default 80): subspace iterations the
 *       eigensolver may take per step before the step fails with HOTRG_EEIG.
 *   HOTRG_OPT_WAIT_CYCLES  >= 1 (default 2e9, about 1 s): bound, in SM clock
 *       cycles, of every pipeline wait in the tensor-core kernels; a wait that
 *       runs out makes the kernel record the failure, let its own copies and
 *       MMAs finish, release its tensor memory and return, and the step reports
 *       HOTRG_ETIMEOUT.  Process-wide (every context), for launches made after
 *       the call; segments already captured into CUDA graphs keep the bound
 *       they were captured with.
 *   HOTRG_OPT_TEST_STALL  1 or 2: testing aid for the timeout path.  The next
 *       tensor-core kernel launched in the process (by any context) of the
 *       chosen kind -- 1: a GEMM, 2: the fused a6 -> a7 kernel -- issues no
 *       operand copies, so its pipeline waits find a barrier nothing arrives at
 *       and run out after HOTRG_OPT_WAIT_CYCLES; one-shot.
 *   HOTRG_OPT_FUSED_CHAIN  0 (default) / 1: with 1, HOTRG_TF32 steps with
 *       Dx = Dy in {16, 32} and D' <= 32 run the products Q = P T and
 *       T' = Q U (Sec. II.B, Eq. 3) as one kernel that keeps Q in on-chip
 *       memory (the second product sums over (x1', x2') in another order, so
 *       results differ from the unfused chain by FP32 rounding).  It saves
 *       Q's write and read (2 x 4 D^5 bytes) but is slower on GB300 (its
 *       second product has N = 16, and such MMAs take the tensor pipe about as
 *       long as N = 128 ones), hence off by default; 0 runs the two GEMMs with
 *       Q in device memory.
 * Returns HOTRG_EINVAL for an unknown option or value.
 */
enum {
  HOTRG_OPT_EIG_TC_PRODUCTS = 0, HOTRG_OPT_XS_DIGITS = 1, HOTRG_OPT_GEMM_AUTOTUNE = 2,
  HOTRG_OPT_GRAPHS = 3, HOTRG_OPT_EIG_MAX_ITERS = 4, HOTRG_OPT_WAIT_CYCLES = 5,
  HOTRG_OPT_TEST_STALL = 6, HOTRG_OPT_FUSED_CHAIN = 7
};
hotrg_status hotrg_set_option(hotrg_ctx *ctx, int option, int value);

/*
 * Stage profiler (tracing, no effect on results).  Stages of one step
 * (Sec. II.A splits the cost into contraction and SVD; the contraction is
 * split further here):
 *   HOTRG_ST_PREP     operand gathers of the tensor-core path (a1)
 *   HOTRG_ST_ENV      environment partials A_L, B_L, A_R, B_R (a2)
 *   HOTRG_ST_GRAM     Gram combine G_L, G_R and FP64 symmetrisation (a3)
 *   HOTRG_ST_EIG      FP64 eigendecomposition and choice of U (a4)
 *   HOTRG_ST_PROJ_P   P = U.T (a5)
 *   HOTRG_ST_PROJ_Q   Q = P.T, the bond contraction (a6)
 *   HOTRG_ST_PROJ_T   T' = Q.U (a7)
 *   HOTRG_ST_RESCALE  max-norm, rescale and log-sum (a8)
 * While enabled, every step records CUDA events around each stage on the
 * context's stream.  hotrg_profile_read synchronises the stream and returns
 * the device time per stage accumulated since the profiler was (re)enabled,
 * the algorithmic flops per stage (each flop counted once: split products
 * and zero padding are not counted), and the number of kernels the library
 * itself launched (library-internal eigensolver kernels are not counted).
 */
enum {
  HOTRG_ST_PREP = 0, HOTRG_ST_ENV, HOTRG_ST_GRAM, HOTRG_ST_EIG, HOTRG_ST_PROJ_P,
  HOTRG_ST_PROJ_Q, HOTRG_ST_PROJ_T, HOTRG_ST_RESCALE, HOTRG_NSTAGES
};

typedef struct {
  int steps;                      /* steps profiled                                  */
  long long launches;             /* own kernel launches in those steps              */
  long long stage_launches[HOTRG_NSTAGES];
  double ms[HOTRG_NSTAGES];       /* accumulated device time per stage (ms)          */
  double flops[HOTRG_NSTAGES];    /* accumulated algorithmic flops per stage         */
} hotrg_profile_t;

/* Enable (1) or disable (0) the profiler; enabling resets the accumulators. */
hotrg_status hotrg_profile_enable(hotrg_ctx *ctx, int enable);
hotrg_status hotrg_profile_read(hotrg_ctx *ctx, hotrg_profile_t *out);

/*
 * Allocation-free max-norm rescale of a caller-owned device tensor (the paper
 * has no counterpart; this is a service for callers that cannot allocate
 * device memory: frameworks that route all device memory through their own
 * pool and forbid other allocators, processes whose device-memory quota such a
 * pool already holds, and latency-critical loops that cannot afford the device
 * synchronisation cudaMalloc implies).
 *   T       device pointer to `count` doubles, rescaled in place: T /= max|T|
 *   count   1 <= count <= 2^26 (67,108,864); larger sizes give HOTRG_EINVAL
 *   weight  finite factor of the log: *logsum += weight * ln(max|T|)
 *   logsum  device pointer to one double, updated in place
 *   stream  cudaStream_t to run on (NULL = legacy default stream)
 * Returns HOTRG_OK, HOTRG_EINVAL, HOTRG_ECUDA, or HOTRG_ENONFINITE when max|T|
 * is zero or not finite (T and *logsum are then left unchanged).  Every call,
 * the first included, copies its status word to host memory and synchronises
 * `stream` before it returns.  It allocates nothing: its scratch (1024 partial
 * maxima and a status word, about 8 KiB) is one file-scope device array that
 * every GPU loading the library holds until the process exits.  The first call
 * on each device resolves that array's device address (with the device
 * current); make that first call before any stream capture.  All calls share
 * the array: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.
 */
hotrg_status hotrg_rescale_noalloc(double *T, long long count, double weight, double *logsum,
                                   void *stream);

/*
 * Batches (many independent lattice models in one context).  Every instance
 * is its own HOTRG run with its own T0 and D_cut -- the step of Sec. II.A
 * (contraction of two tensors along one bond, fused legs cut by the SVD of the
 * reshaped pair) applied to each instance's own Z = Tr T^N (Eq. 2); all
 * instances take the same step directions.  Instances with equal (D0, D_cut) have equal bond
 * dimensions after every step and are grouped: each kernel of a step runs once
 * per group over all its instances, and the eigensolver diagonalises the
 * group's 2G environments as one batch.  Results of an instance do not depend
 * on which other instances share its context.
 *
 * hotrg_batch_create: n instances (1 <= n <= 4096); T0s[i] is a host pointer
 *   to D0s[i]^4 doubles ([x,x',y,y'] row-major, borrowed and copied): the local
 *   tensor of instance i (Sec. II.A, Eq. 2), 1 <= D0s[i] <= 64 and
 *   1 <= Dcuts[i] <= 64.  prec, stream, ownership and errors as for
 *   hotrg_create (all device memory is allocated here).
 * hotrg_batch_step: one coarse-graining step (Sec. II.A) of every instance,
 *   same as hotrg_step.
 * hotrg_batch_size: number of instances.
 * hotrg_batch_log_z: ln Z / N of every instance (Sec. II.A, Eq. 2, as for
 *   hotrg_log_z_per_site), in creation order, into out_n[0..n) (host, n
 *   doubles; synchronises).
 * hotrg_batch_step_info / hotrg_batch_get_tensor: hotrg_step_info and
 *   hotrg_get_tensor for instance `inst` (0-based, creation order).
 * On a context with more than one instance, hotrg_log_z_per_site and
 * hotrg_free_energy return HOTRG_ESTATE; hotrg_step_info, hotrg_spectrum,
 * hotrg_get_tensor, hotrg_get_isometry and hotrg_dims report instance 0.
 */
hotrg_status hotrg_batch_create(int n, const double *const *T0s, const int *D0s,
                                const int *Dcuts, hotrg_prec prec, void *stream,
                                hotrg_ctx **out);
hotrg_status hotrg_batch_step(hotrg_ctx *ctx, hotrg_dir dir);
hotrg_status hotrg_batch_size(hotrg_ctx *ctx, int *n);
hotrg_status hotrg_batch_log_z(hotrg_ctx *ctx, double *out_n);
hotrg_status hotrg_batch_step_info(hotrg_ctx *ctx, int inst, int step, hotrg_step_info_t *out);
hotrg_status hotrg_batch_get_tensor(hotrg_ctx *ctx, int inst, double *host_out, long long cap,
                                    int dims[4]);

/*
 * FP64-grade GEMM on the BF16 tensor cores (the paper has no counterpart; the
 * library's eigensolver uses the same kernels for its products G X, because
 * GB300 runs native FP64 at about 1 TFLOP/s):
 *   C[i * ldc + j] = sum_k A[i * lda + k] * B[j * ldb + k],  0 <= i < M, 0 <= j < N
 * (row-major A: M x K, B: N x K, C: M x N, all FP64 device pointers that stay
 * owned by the caller; C must not overlap A or B).  Each row of A and of B is
 * scaled by a power of two below 1 and cut into `slices` base-64 digits
 * stored as exact BF16 values; products of digit pairs whose indices sum to at
 * most slices + 1 are accumulated on the tensor cores, exactly for the five
 * leading digit sums (K is split into parts of at most 2336 for that), and
 * combined in 64-bit integer and FP64 arithmetic.  Error per term about
 * 2^-(6 slices) relative to the row maxima max|A_i.| max|B_j.| (slices = 8:
 * about 1e-15 of max|A_i.| max|B_j.| K).  4 <= slices <= 8, K >= 1, lda, ldb >= K, ldc >= N.  Allocates its scratch
 * (about 2 slices (M + N) K bytes) with cudaMalloc, runs on `stream` and
 * synchronises it before returning.  Returns HOTRG_OK, HOTRG_EINVAL,
 * HOTRG_ENOMEM, HOTRG_ECUDA, or HOTRG_ETIMEOUT if a bounded device wait ran
 * out.  A row with a non-finite entry gives NaN in its outputs.
 */
hotrg_status hotrg_dgemm_emu(int M, int N, int K, const double *A, long long lda,
                             const double *B, long long ldb, double *C, long long ldc,
                             int slices, void *stream);

/* Release all resources of the context; NULL is accepted and ignored. */
void hotrg_destroy(hotrg_ctx *ctx);

/* Message of the latched error ("" if none); valid until the next call on ctx. */
const char *hotrg_last_error(const hotrg_ctx *ctx);

/* Static name of a status code. */
const char *hotrg_status_string(hotrg_status s);

#ifdef __cplusplus
}
#endif

#endif /* HOTRG_H */
