/*
 * psum -- periodic Coulomb sums on one GPU by the periodisation method of
 * Gumerov & Duraiswami, "A method to compute periodic sums" (arXiv 1310.4374).
 *
 * For N charges q_i at x_i in the box [-d1/2, d1/2) x [-d2/2, d2/2) x [-d3/2, d3/2)
 * with sum q_i = 0 (Sec. 1, Eq. 1) the library returns the periodic potential
 *
 *     phi(y) = sum_{p} sum_i q_i K(y - x_i + p),  K(r) = 1/|r|, K(0) = 0  (Eq. 2)
 *
 * and its gradient at every charge, with the side condition fixed by the paper:
 * periodicity of phi (Eq. 7) and zero mean over the box (Eqs. pfx2-pfx3 with
 * phi_mean = 0, the Ewald convention of App. D).  phi is split into
 *
 *   phi_near: direct sum over the box and its neighbour images (Eq. 3),
 *             evaluated at the charges and at the M check points and their
 *             partners (or as the partners' two-layer difference, PSUM_CHECKS_*), and
 *   phi_far:  C_1 + sum_{t>=2} C_t R_t(y/R0), a regular-solid-harmonic local
 *             expansion of maximum degree p (Eqs. 1.6-1.8) whose coefficients
 *             are the least-squares solution of the periodicity conditions at
 *             M check points on the circumsphere (Eqs. 7-10, algorithms "set"
 *             and "get" of Sec. 2.3).
 *
 * Conventions
 *   p  is the MAXIMUM DEGREE of the expansion: there are P = (p+1)^2 terms,
 *      stacked as t = n(n+1) + m (0-based form of Eq. 1.8).  The paper's
 *      truncation number is p + 1.
 *   M  is the number of check points (the paper's L).  M >= P - 1 is required
 *      (Sec. 4.1, rank condition); about 2P to 3P is a good choice.
 *   All positions, charges and results are float64.  x is row-major N x 3.
 *
 * Memory and streams
 *   Every device pointer is owned by the caller and must stay valid until the
 *   work queued on `stream` has finished.  An evaluation forks part of its work onto two
 *   internal streams of the plan and joins them again before it returns to `stream`, so
 *   completion of `stream` covers all of it (also inside a graph capture of `stream`).  `stream` is a cudaStream_t passed
 *   as void* (NULL = the legacy default stream).  A plan owns its check
 *   points, its factorisation, the image list and its scratch memory; the
 *   scratch grows on demand inside psum_eval (a cudaMalloc, which synchronises
 *   the device) and is then reused, so the first call of a given size should
 *   not be made inside a stream capture.  A plan may be used by one stream at
 *   a time.
 *
 * Errors
 *   Every call returns a status code (PSUM_OK = 0).  psum_eval validates its
 *   arguments on the host and queues the work; conditions only the device can
 *   see (non-neutral charges, positions outside the box, non-finite results)
 *   are written to a device status word that psum_sync returns.  After a
 *   device-side error the outputs are filled with NaN.
 */
#ifndef PSUM_H
#define PSUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PSUM_OK              0
#define PSUM_ERR_ARG         1  /* invalid argument (NULL pointer, p < 1, M < P-1, d <= 0, ...) */
#define PSUM_ERR_NONNEUTRAL  2  /* |sum q| > 1e-12 sum |q|: Eq. 1 requires a neutral box */
#define PSUM_ERR_OUT_OF_BOX  3  /* a position outside [-d/2, d/2) or not finite */
#define PSUM_ERR_RANK        4  /* the fitting matrix A is rank deficient (|R_kk| < 1e-13 |R_11|) */
#define PSUM_ERR_CUDA        5  /* a CUDA runtime call failed */
#define PSUM_ERR_TIMEOUT     6  /* a bounded device-side wait gave up */
#define PSUM_ERR_NOMEM       7  /* host or device allocation failed */
#define PSUM_ERR_NONFINITE   8  /* a result is not finite (e.g. two charges closer than FP32 resolves) */
#define PSUM_ERR_INTERNAL    9  /* a debug build's bounds check refused an access (psum_debug_checks) */
#define PSUM_ERR_IO         10  /* a plan file cannot be read or written, or does not match (psum_plan_load) */

/* ---- options ------------------------------------------------------------ */
#define PSUM_FP64   0  /* near-field pair sum in float64 */
#define PSUM_FP32C  1  /* pair arithmetic in float32 on tile-relative coordinates,
                          compensated (two-sum) accumulation, float64 elsewhere */
#define PSUM_FF     2  /* pair arithmetic in float-float (a float32 pair carrying about 44 bits)
                          on the float32 pipe: float64-class results (the float64 tolerance)
                          without float64 pair arithmetic; float64 elsewhere.  Offsets are
                          relative to 128-point groups, so where charges sit far closer than
                          their groups' size (a cluster of 1e-6 inside a box of 1) the relative
                          accuracy falls toward 2^-48 times that ratio. */
/* Both float32 precisions take two charges closer than 2^-37 R0 (R0 the half diagonal of the
   box) as coincident (K(0) = 0); PSUM_FP64 drops exact zeros only. */

#define PSUM_POINTS_FIBONACCI 0  /* M check points on a spherical Fibonacci lattice */
#define PSUM_POINTS_GAUSS     1  /* the Gauss spherical grid of Sec. 2.2: polar angles at the zeros of
                                    P_{p+1}(cos theta), 2p+1 equispaced azimuths; M = (p+1)(2p+1) */

#define PSUM_BASIS_SPHERICAL 0  /* regular solid harmonics R^_n^m(y/R0), n <= p (Eqs. 1.6-1.8); P = (p+1)^2 */
#define PSUM_BASIS_RBF       1  /* kernel functions 1/|y - x_t| centred outside S_b (Eq. 5); P = n_rbf + 1 */

/* pair kernel of the near sum at the charges (psum_opts.pair_kernel) */
#define PSUM_PAIRS_AUTO       0  /* symmetric where it applies: FP32C from 12 tiles of 512 charges (5633
                                    charges), FF from 6 tiles (2561), FP64 at every size; one-sided
                                    otherwise */
#define PSUM_PAIRS_ONE_SIDED  1  /* every (target, source, image) term computed on its own */
#define PSUM_PAIRS_SYMMETRIC  2  /* where it applies, at any size: the pair (i, j, p) and its mirror
                                    (j, i, -p) share one offset and one 1/r (FP32C, FF and FP64 plans
                                    without ball trimming, potential and field at the charges, psum_eval,
                                    psum_eval_host, psum_eval_graph and psum_energy, and FP32C batches;
                                    one-sided elsewhere).  Same sums, different rounding order. */

/* form of the right-hand side f_l = phi_near(y~_l) - phi_near(y_l) (psum_opts.check_form).
 * The partner y~_l = y_l - s d_k e_k (s = +-1) sees the near block shifted by one period
 * along k, so the two block sums differ by two image layers only:
 *   f_l = sum_i q_i [ sum_{i_k = s (K_k + 1)} K(y_l - x_i - p) - sum_{i_k = -s K_k} K(y_l - x_i - p) ]
 * (the other two image indices over their block ranges): 2 (2K_a+1)(2K_b+1) images at M
 * points instead of (2K_1+1)(2K_2+1)(2K_3+1) images at 2M points (18 x M against 27 x 2M for
 * the 3x3x3 block). */
#define PSUM_CHECKS_AUTO    0  /* layers where they apply (plans without ball trimming, every
                                  precision, single systems and batches) and take no more (target
                                  tile, image) units than the points; points otherwise */
#define PSUM_CHECKS_POINTS  1  /* phi_near at y_l and at y~_l, differenced in float64 */
#define PSUM_CHECKS_LAYERS  2  /* the two-layer form; PSUM_ERR_ARG for ball-trimmed plans (the ball
                                  is not a block of images).  Float32 plans whose layers exceed the
                                  pair kernel's shared memory (K = 3 along two axes) keep the
                                  points; psum_check_form reports the form taken. */

/* float32 pair terms of PSUM_FP32C plans (psum_opts.fp32_terms).  The float32 term q/r carries
 * the rounding of its offsets, of r^2, of the rsqrt estimate and of the product, about one
 * float32 unit in the last place (rms) of the term; the potential's error is that times
 * kappa = sqrt(sum of squared terms) / rms(phi), the cancellation of the near sum.  Random
 * charges have kappa of a few (about 4.7e-7 at 1e5 charges); tight dipoles of 2e5 charges about
 * 20 (1.3e-6). */
#define PSUM_TERMS_FAST     0  /* plain float32 terms */
#define PSUM_TERMS_REFINED  1  /* the charge sums' far terms with 1/r as a float pair (the rsqrt
                                  estimate plus its Newton correction) fused into the sums
                                  unrounded, the targets' offsets rounded once, and the potential's
                                  running sums cut every 8 steps: about 0.6 of the fast terms' error
                                  for about 1.7x the symmetric charge kernel's time.  Applies to
                                  the symmetric charge kernel (psum_pair_kernel); the one-sided
                                  kernels and batches keep the fast terms. */

#define PSUM_MEAN_ZERO 0  /* C_1 makes the box mean of phi zero (Eq. pfx3, phi_mean = 0) */
#define PSUM_MEAN_NONE 1  /* C_1 = 0 (potential defined up to a constant, Sec. 3) */

typedef struct psum_plan_s *psum_plan_t;

typedef struct psum_opts {
    double d[3];     /* box edge lengths, > 0 */
    int p;           /* maximum degree of the local expansion, 1 <= p <= 40 */
    int M;           /* number of check points, M >= (p+1)^2 - 1 */
    int precision;   /* PSUM_FP64, PSUM_FP32C or PSUM_FF */
    int mean_mode;   /* PSUM_MEAN_ZERO or PSUM_MEAN_NONE */
    int K[3];        /* near block: images |i_k| <= K[k] of the box (Eq. 3, Omega_b); 1 = 3x3x3 */
    int points;      /* PSUM_POINTS_FIBONACCI or PSUM_POINTS_GAUSS (then M must be 0 or (p+1)(2p+1)) */
    double lambda;   /* 0: the near set is the block of images above.  lambda > 1: the near set
                        is trimmed to the ball S_b of radius Rb = lambda R0 (algorithm "get",
                        step 2): a source image x_i + p counts only if |x_i + p| <= Rb, tested
                        in float64 as ((a*a + b*b) + c*c) <= Rb*Rb without contraction; K is
                        then ignored and the block is the smallest one that covers the ball,
                        K_k = ceil(Rb/d_k + 1/2).  Trimmed plans serve psum_eval, psum_eval_host,
                        psum_eval_noalloc and psum_energy; psum_energy_backward and the batch
                        API reject them (PSUM_ERR_ARG). */
    int basis;       /* PSUM_BASIS_SPHERICAL or PSUM_BASIS_RBF.  With the RBF basis (Eq. 5) the far
                        field is C_1 + sum_t C_t / |y - x_t| over n_rbf centres x_t on a spherical
                        Fibonacci lattice of radius rbf_radius R0; p then only sizes the Gauss grid,
                        and M >= n_rbf is required.  psum_get_coeffs returns C_1, C_2..C_{n_rbf+1}.
                        psum_energy_backward and the batch API reject RBF plans (PSUM_ERR_ARG). */
    int n_rbf;       /* number of RBF centres, 1..4096 (0: 256, the paper's choice) */
    double rbf_radius;  /* centres at rbf_radius R0, > 1 (0: on S_b, i.e. at lambda_eff R0) */
    int pair_kernel;    /* PSUM_PAIRS_AUTO, PSUM_PAIRS_ONE_SIDED or PSUM_PAIRS_SYMMETRIC */
    int check_form;     /* PSUM_CHECKS_AUTO, PSUM_CHECKS_POINTS or PSUM_CHECKS_LAYERS */
    int fp32_terms;     /* PSUM_TERMS_FAST or PSUM_TERMS_REFINED (PSUM_FP32C plans; ignored otherwise) */
} psum_opts;

typedef struct psum_info {
    double d[3];
    double R0;          /* circumradius (algorithm "set", step 1) */
    double lambda_eff;  /* distance from the centre to the nearest excluded image box, over R0 */
    double cond_est;    /* max |R_kk| / min |R_kk| of the pivoted QR of A (a condition estimate) */
    int rank;           /* numerical rank of A (= P - 1 for a usable plan) */
    int p, P, M;
    int K[3];
    int n_images;       /* (2K1+1)(2K2+1)(2K3+1) */
    int precision, mean_mode;
} psum_info;

/* Fill `o` with the defaults: unit cube, p = 8, M = 200, PSUM_FP64,
   PSUM_MEAN_ZERO, K = (1,1,1), PSUM_POINTS_FIBONACCI, lambda = 0, PSUM_BASIS_SPHERICAL,
   n_rbf = 256, rbf_radius = 0, PSUM_PAIRS_AUTO, PSUM_CHECKS_AUTO, PSUM_TERMS_FAST. */
void psum_opts_default(psum_opts *o);

/* Algorithm "set" (Sec. 2.3.1): circumradius R0 (step 1), M check points on the
 * sphere of radius R0 (step 2; a spherical Fibonacci lattice), their periodic
 * partners (step 3), the M x (P-1) fitting matrix A_lt = R_t(y_l) - R_t(y~_l)
 * without the constant column (step 4, Sec. 3), its column-pivoted Householder
 * QR and pseudo-inverse (step 5, Eq. 10), and the box integrals R_t^(0) by
 * Gauss-Legendre quadrature (step 6, App. B).  Runs on the host in float64 and
 * uploads the results to the current CUDA device.
 * Returns PSUM_ERR_ARG, PSUM_ERR_RANK, PSUM_ERR_NOMEM or PSUM_ERR_CUDA on failure;
 * *out is set only on success.  psum_plan_create uses FP64 and the defaults. */
int psum_plan_create(double d1, double d2, double d3, int p, int M, psum_plan_t *out);
int psum_plan_create_ex(const psum_opts *o, psum_plan_t *out);

/* Keep algorithm "set"'s factorisation (Sec. 2.1 recommends storing the decomposition, and the
 * set time is the cost of a new plan, Sec. 4.2): psum_plan_save writes the plan's options, the
 * fingerprint of its check points and partners, the rank, the condition estimate and the
 * (P-1) x M pseudo-inverse to `path`, with a checksum; psum_plan_load reads such a file and builds
 * the plan without factoring A again (check points, box integrals and tables are recomputed: they
 * are cheap and deterministic).  The loaded plan evaluates exactly as the saved one.  Errors:
 * PSUM_ERR_ARG for NULL arguments; PSUM_ERR_IO when the file cannot be written or read, is
 * truncated, fails its checksum or magic word, was written by a library with another psum_opts
 * layout, or its check points do not hash to the ones this library computes for its options;
 * otherwise those of psum_plan_create_ex.  *out is set only on success.  Host files are
 * little-endian IEEE doubles. */
int psum_plan_save(psum_plan_t plan, const char *path);
int psum_plan_load(const char *path, psum_plan_t *out);

/* Algorithm "get" (Sec. 2.3.2) with Y0 = X0 (Remark 1): phi[i] and grad[3i..3i+2]
 * at every charge.  x (N x 3), q (N), phi (N) and grad (N x 3, may be NULL) are
 * DEVICE pointers on the plan's device; N >= 1.  Queued on `stream`; returns
 * after queueing.  Host-side checks give PSUM_ERR_ARG; device-side conditions
 * are reported by psum_sync. */
int psum_eval(psum_plan_t plan, int64_t N, const double *x, const double *q,
              double *phi, double *grad, void *stream);

/* psum_eval through a CUDA graph: the first call for a given (N, x, q, phi, grad) captures
   the whole evaluation (about 25 kernels and memsets) on an internal stream and later calls
   with the same arguments replay it on `stream`, which removes the per-kernel launch cost
   (it dominates below ~5000 charges).  The inputs may change between replays in the same
   buffers.  Results, status reporting (psum_sync) and asynchrony are those of psum_eval;
   psum_profile timings are not recorded by replays.  The first call of a size allocates
   scratch, so it must not be made inside a stream capture of the caller. */
int psum_eval_graph(psum_plan_t plan, int64_t N, const double* x, const double* q, double* phi,
                    double* grad, void* stream);

/* Algorithm "get" at separate evaluation points (the general problem of Sec. 1: the
   potential and its gradient at points y of the box due to the N charges; psum_eval is the
   case Y0 = X0 of Remark 1).
     x, q      : the charges as in psum_eval (device, caller-owned).
     y         : T x 3 float64 evaluation points, row-major, device, inside the half-open box.
     phi, grad : T and T x 3 float64 outputs (grad may be NULL).
   A point that coincides exactly with a charge drops that pair (K(0) = 0, Eq. 1).  Works
   with every precision, point scheme, basis and the ball-trimmed near set.  Asynchronous on
   `stream`; a point outside the box gives PSUM_ERR_OUT_OF_BOX at psum_sync. */
int psum_eval_points(psum_plan_t plan, int64_t N, const double* x, const double* q, int64_t T,
                     const double* y, double* phi, double* grad, void* stream);

/* The same with HOST pointers: copies x and q to the device, evaluates, copies
 * phi and grad back and waits for the stream.  Returns the final status
 * (including device-side conditions). */
int psum_eval_host(psum_plan_t plan, int64_t N, const double *x, const double *q,
                   double *phi, double *grad, void *stream);

/* psum_eval without any allocation at evaluation time.  The paper has no counterpart:
 * this entry exists for callers that cannot call cudaMalloc when they evaluate --
 * code running inside a CUDA stream capture (an allocation there breaks the graph
 * being recorded), real-time loops that cannot take the device-wide synchronisation
 * of a cudaMalloc or cudaFree, and runtimes that own all device memory through their
 * own pool.  psum_eval grows a per-plan scratch buffer with cudaMalloc the first time
 * it sees a size; this call instead takes all of its scratch from one 16 MiB device
 * array inside the library, which every GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Arguments, results and status reporting are those of psum_eval (device pointers,
 * queued on `stream`, device-side conditions reported by psum_sync).  The results
 * agree with psum_eval to rounding: the pair sum is split into at most 256 work items, so
 * partial sums are grouped differently.  Limits: an evaluation whose scratch does not
 * fit in the 16 MiB array returns PSUM_ERR_ARG; that holds up to N = 32768 charges
 * for plans with p <= 16 and M <= 800 in either precision (larger p or M lower it).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other plans, other threads)
 * race and corrupt each other's results -- serialise them, e.g. on one stream.  Like
 * psum_eval, a call replaces the plan's coefficients (psum_get_coeffs, and the C that
 * psum_energy_backward uses). */
int psum_eval_noalloc(psum_plan_t plan, int64_t N, const double *x, const double *q,
                      double *phi, double *grad, void *stream);

/* Wait for `stream`, then return and clear the plan's device status word. */
int psum_sync(psum_plan_t plan, void *stream);

/* E = 1/2 sum_i q_i phi[i] into the device scalar *E (deterministic reduction).
 * q and phi are device arrays of length N (phi from psum_eval). */
int psum_energy(psum_plan_t plan, int64_t N, const double *q, const double *phi, double *E, void *stream);

/* Exact derivatives of the method's energy E = 1/2 sum_i q_i phi(x_i).  The method is
 * linear in q but its far field is a least-squares fit, so the adjoint of the fit enters:
 * with w_t = sum_i q_i R_t(x_i/R0) and u = (A^+)^T w,
 *   psi(x)    = sum_l u_l [G(y~_l - x) - G(y_l - x)]   (G: the near-block image kernel),
 *   dEdq[i]   = gE (phi_i - phi_far(x_i)/2 + psi(x_i)/2),
 *   dEdx[3i+k]= gE q_i (grad_i - grad phi_far(x_i)/2 + grad psi(x_i)/2)_k.
 * x, q, phi, grad (device) must be the inputs and outputs of the LAST evaluation of this
 * plan -- psum_eval, psum_eval_host, psum_eval_graph or psum_eval_noalloc, each of which
 * replaces the plan's coefficients C, which are used here (psum_energy_backward_c takes
 * them as an argument instead).  gE is a device scalar multiplying the result (the
 * upstream gradient), or NULL for 1.  dEdq or dEdx may be NULL (not both).  The 27 N^2
 * pair sum is not repeated: psi is a sum over the 2M check points. */
int psum_energy_backward(psum_plan_t plan, int64_t N, const double *x, const double *q,
                         const double *phi, const double *grad, const double *gE,
                         double *dEdq, double *dEdx, void *stream);

/* Queue a copy of the P coefficients C_1..C_P of the plan's last evaluation (stacked by
 * Eq. 1.8) into the DEVICE array C (caller-owned, P doubles, on the plan's device) on
 * `stream`; no synchronisation.  Made right after an evaluation, it keeps that evaluation's
 * far-field expansion (Eq. 1.8 with the fitted C of Eq. 10) for psum_energy_backward_c.
 * PSUM_ERR_ARG for a NULL plan or array. */
int psum_coeffs_device(psum_plan_t plan, double *C, void *stream);

/* psum_energy_backward with the coefficients of the forward evaluation passed in: C (device,
 * P doubles, as psum_coeffs_device writes them) replaces the plan's last coefficients in the
 * moments w_t and in phi_far and grad phi_far at the charges, so the derivatives belong to
 * the evaluation that produced (x, q, phi, grad, C) however many evaluations of the plan
 * came after it (as in an autograd graph with several forwards through one plan).  The
 * same adjoint formulas, arguments and errors as psum_energy_backward, plus PSUM_ERR_ARG for
 * a NULL C. */
int psum_energy_backward_c(psum_plan_t plan, int64_t N, const double *x, const double *q,
                           const double *phi, const double *grad, const double *C, const double *gE,
                           double *dEdq, double *dEdx, void *stream);

/* Copy the P coefficients C_1..C_P of the last evaluation to host memory
 * (stacked by Eq. 1.8; C[0] is the constant C_1).  Waits for `stream`. */
int psum_get_coeffs(psum_plan_t plan, double *C, void *stream);

int psum_plan_info(psum_plan_t plan, psum_info *info);

/* The pair kernel psum_eval runs for N charges on this plan, after the automatic choice:
 * *kernel = PSUM_PAIRS_ONE_SIDED or PSUM_PAIRS_SYMMETRIC; *image_groups (may be NULL) = the
 * symmetric kernel's image groups per tile pair (work items = tile pairs x groups), else 0.
 * Host only; PSUM_ERR_ARG for a null plan or kernel pointer or N < 0. */
int psum_pair_kernel(psum_plan_t plan, int64_t N, int *kernel, int *image_groups);

/* Device scratch psum_eval takes for N charges on this plan (*bytes: the plan's buffer grows to
 * this size), and *bands (may be NULL): the number of bands of row tiles the symmetric charge
 * kernel runs in turn, each reduced before the next, so that its partial sums stay within 1.5 GiB
 * (0 with the one-sided kernel).  Host only; PSUM_ERR_ARG for a null plan or bytes, or N < 1. */
int psum_scratch_bytes(psum_plan_t plan, int64_t N, int64_t *bytes, int *bands);

/* The form of the check-point sums psum_eval runs on this plan, after the automatic choice:
 * *form = PSUM_CHECKS_POINTS or PSUM_CHECKS_LAYERS.  Host only; PSUM_ERR_ARG for a null plan
 * or form pointer. */
int psum_check_form(psum_plan_t plan, int *form);

/* Stage timing.  With profiling enabled, psum_eval records CUDA events on its
 * stream around each stage; psum_last_timings waits for `stream` and writes the
 * PSUM_NUM_STAGES durations (milliseconds) of the last evaluation:
 *   [0] validation, spatial sort and packing
 *   [1] near-field sum at the charges (potential and gradient)
 *   [2] the charges' reduction, and what is left of the check-point sums and the box mean:
 *       those run on an internal stream of the lowest priority from the end of [0], beside
 *       the charge sum, and fill the SMs it releases as it finishes
 *   [3] right-hand side, least squares and C_1
 *   [4] far field, combination and write-back
 * Returns PSUM_ERR_ARG if profiling is off. */
#define PSUM_NUM_STAGES 5
int psum_profile(psum_plan_t plan, int enable);
int psum_last_timings(psum_plan_t plan, double *ms, void *stream);

/* Number of CUDA kernels this plan has queued since it was created. */
int psum_launch_count(psum_plan_t plan, int64_t *count);

/* ---- batches of independent systems -------------------------------------- */
typedef struct psum_batch_s *psum_batch_t;

typedef struct psum_batch_info {
    int B;               /* systems */
    int64_t N_total;     /* charges over all systems */
    int64_t units;       /* (tile, chunk, image) work units of the charge pair sum */
    int64_t pairs;       /* pair interactions of one evaluation (charges and check points) */
    int ctas;            /* CTAs of the persistent pair-sum launch */
    int variant;         /* pair-kernel variant chosen by the autotuner: 0 and 1 the one-sided
                            kernel at 4 and 6 CTAs per SM, 2 the symmetric kernel (FP32C) */
    double tuned_ms;     /* its measured time for one charge pair sum and its reduction, ms
                            (0 before tuning) */
} psum_batch_info;

/* B independent periodic systems evaluated together (algorithm "get" for each), with one
 * persistent launch (fixed work items, taken dynamically) for all charge pair sums and one for all check-point pair
 * sums.  plans[b] fixes system b's box, degree, check points and near block; all plans
 * must share the precision and the current device (a plan may appear several times).
 * Each system's check sums take its plan's form (psum_check_form).
 * offsets (host, B+1 entries, offsets[0] = 0, increasing) delimit system b's charges in
 * the concatenated arrays: rows offsets[b] .. offsets[b+1]-1.  1 <= B <= 65535.  All
 * device memory of the batch is allocated here.  The plans must outlive the batch. */
int psum_batch_create(const psum_plan_t *plans, int B, const int64_t *offsets, psum_batch_t *out);

/* psum_eval for every system: x (N_total x 3), q, phi, grad (may be NULL) are device
 * arrays over the concatenated charges.  The first evaluation times the pair-kernel
 * variants on these inputs and keeps the fastest (cached per batch shape).  With
 * use_graph != 0 the whole sequence is captured once into a CUDA graph for these
 * pointers and replayed on `stream` afterwards (a capture for new pointers replaces it). */
int psum_batch_eval(psum_batch_t batch, const double *x, const double *q, double *phi,
                    double *grad, int use_graph, void *stream);

/* Wait for `stream`; write the per-system status codes to status (host, B entries, may
 * be NULL), clear them, and return the first non-zero one. */
int psum_batch_sync(psum_batch_t batch, int *status, void *stream);

/* System b's P coefficients of the last evaluation (host array), as psum_get_coeffs. */
int psum_batch_get_coeffs(psum_batch_t batch, int b, double *C, void *stream);

int psum_batch_get_info(psum_batch_t batch, psum_batch_info *info);

/* Release the batch (waits for the device). NULL is a no-op. */
void psum_batch_destroy(psum_batch_t batch);

/* Test hook of the failure path (the paper has no counterpart).  While enabled, the charge
   pair kernel of this plan (float32 packing: PSUM_FP32C and PSUM_FF) arms its chunk-copy
   barrier for 16 bytes more than the copies bring, so each wait runs out after a short
   iteration limit: the kernel flags the evaluation, which then reports PSUM_ERR_TIMEOUT at
   psum_sync and writes NaN, and the CUDA context stays usable.  Off by default; returns
   PSUM_ERR_ARG for a NULL plan. */
int psum_debug_inject_timeout(psum_plan_t plan, int enable);

/* Debug builds (the paper has no counterpart).  A library compiled with -DPSUM_DEBUG_CHECKS=1
   range-checks every write and read of the pair kernels' partial sums against the buffer's size:
   an access outside it is skipped and flagged, psum_sync returns PSUM_ERR_INTERNAL and the outputs
   are NaN, and the CUDA context stays usable (no trap).  psum_debug_checks() returns 1 in such a
   build, 0 otherwise.  psum_debug_bounds_limit is its test hook: the checks see the partial
   buffers as `doubles` long (0: their real size), so that a smaller value makes them fire without
   any access leaving the real buffer; it has no effect on other builds.  PSUM_ERR_ARG for a NULL
   plan or doubles < 0. */
int psum_debug_checks(void);
int psum_debug_bounds_limit(psum_plan_t plan, int64_t doubles);

/* Test hook of the failure path (the paper has no counterpart): the next `count` growths of
   this plan's scratch buffer fail as an out-of-memory cudaMalloc would -- the call that needed
   it returns PSUM_ERR_NOMEM, queues nothing and leaves the plan without scratch, so a later call
   grows it again.  No allocation is attempted for a failed growth.  PSUM_ERR_ARG for a NULL plan
   or count < 0. */
int psum_debug_fail_allocs(psum_plan_t plan, int count);

/* Test hook of the banded partial sums (the paper has no counterpart): caps the symmetric charge
   kernel's partial slots per band at `bytes` (0 restores 1.5 GiB), so that small systems run
   several bands.  Results agree with the single band to rounding (the same slots, reduced in
   another grouping).  PSUM_ERR_ARG for a NULL plan or bytes < 0. */
int psum_debug_band_bytes(psum_plan_t plan, int64_t bytes);

/* Release the plan and its device memory (waits for the device). NULL is a no-op. */
void psum_destroy(psum_plan_t plan);

/* Static, NUL-terminated description of a status code. */
const char *psum_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* PSUM_H */
