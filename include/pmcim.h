/*
 * pmcim.h -- C ABI of the GB300 contour-integral eigensolver library (libpmcim.so).
 *
 * Problem class (Sec. 1): find lambda in a bounded region with T(lambda) x = 0,
 * where T(z) = sum_k f_k(z) A_k with dense complex n x n coefficients A_k and
 * scalar functions f_k drawn from a fixed set: monomials z^d and exp(-tau z).
 * The region is covered by disks circumscribing squares (Sec. 3, start); each
 * disk is discretised by the N-node trapezoid rule (Eq. 3.2-3.3).
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved (re, im) pairs of double.
 *   - Matrices are column-major with leading dimension n; indices are 0-based.
 *   - Every buffer argument may be a host pointer or a CUDA device pointer (the
 *     library uses unified addressing to tell them apart). The caller owns all
 *     buffers; no call keeps a caller pointer after it returns.
 *   - Calls are synchronous: the library's work starts after everything queued
 *     on opt->cuda_stream before the call, runs on a stream of the problem
 *     handle's own (levels are launched as CUDA graphs, which the legacy
 *     default stream cannot capture), and has finished when the call returns,
 *     with all results in the caller's buffers.
 *   - Every call returns 0 (PMCIM_OK) or a negative PMCIM_E* code; the message
 *     of the last failure on the calling thread is pmcim_last_error(). Problems
 *     with one disk (a saturated rank test, an exactly singular node) never fail
 *     a call: they are reported in per-region status bits, because the method
 *     prefers spurious candidates, removed later, to missed eigenvalues
 *     (Sec. 3.2, robustness remark).
 *   - One problem handle must not be used by two host threads at once.
 *   - There is no CPU fallback: without a usable CUDA device every call returns
 *     PMCIM_ECUDA.
 */
#ifndef PMCIM_H
#define PMCIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define PMCIM_OK 0
#define PMCIM_EINVAL (-1)    /* bad argument (size, NULL, odd N, ...)        */
#define PMCIM_ENOMEM (-2)    /* device allocation failed                     */
#define PMCIM_ECUDA (-3)     /* CUDA runtime error or no device              */
#define PMCIM_ETIMEOUT (-4)  /* a bounded device wait ran out                */
#define PMCIM_ECAPACITY (-5) /* more eigenvalues than the caller's capacity  */
#define PMCIM_ENOTSUP (-6)   /* option not supported for this problem size   */

/* ---- per-region status bits ---------------------------------------------- */
#define PMCIM_RS_CANDIDATE 1      /* indicator I > tol_ind (pmCIMb step 1.c)        */
#define PMCIM_RS_SATURATED 2      /* rank p reached min(n, l) in Beyn's SVD test    */
#define PMCIM_RS_SPLIT 4          /* saturated disk was split into four children   */
#define PMCIM_RS_SINGULAR_NODE 8  /* an LU met an exactly zero pivot at some node  */
#define PMCIM_RS_IR_FALLBACK 16   /* refinement did not converge; FP64 re-solve    */
#define PMCIM_RS_NO_EIG 32        /* candidate disk whose Beyn step kept no value  */
#define PMCIM_RS_SCREENED 64      /* the learned screen skipped the full indicator */

/* ---- scalar functions f_k ------------------------------------------------ */
#define PMCIM_F_MONOMIAL 0 /* f(z) = z^degree                                   */
#define PMCIM_F_EXP_NEG 1  /* f(z) = exp(-tau z)                                */
/* A boundary-integral term (the scattering-pole problem of Sec. 4.2): the term
   is c K_n(z), c = id_re + i id_im, where K_n(z) is the Nystrom matrix of the
   2-D Helmholtz double-layer operator
     (K phi)(x) = 2 int_C d/dnu(y) [(i/4) H_0^(1)(z |x - y|)] phi(y) ds(y)
   on a smooth closed curve C, discretised by Kress's rule for kernels with a
   logarithmic singularity (R. Kress, Linear Integral Equations, Sec. 12.3) on
   the n points x(t_j), t_j = 2 pi j / n. The paper's T(z) = (I + K_n(z)) / 2 is
   the identity term 0.5 I plus this term with c = 0.5. Its coefficient pointer
   A[k] holds 6 n doubles: the rows x1(t_j), x2(t_j), x1'(t_j), x2'(t_j),
   x1''(t_j), x2''(t_j), each of n values (derivatives in t, the curve traversed
   counter-clockwise). n must be even and at least 4; a problem holds at most
   one such term. It runs in every precision form; PMCIM_PREC_AUTO takes
   PMCIM_PREC_FP32_IR for it, and pmcim_residual refuses it (EINVAL: the
   tensor-core residual needs coefficient matrices). The entries are formed on
   the device from J_1 and H_1^(1) of complex argument w = z r (ascending series
   for |w| <= 13, Hankel's expansion above), for Re(z) > 0: relative error at
   most about 5e-12 where Im(w) <= 0 (the scattering poles lie in Im z < 0) and
   4e-11 for 0 < Im(w) <= 2; above that the series loses about e^{2 Im w}
   rounding units to cancellation in H_1^(1) = J_1 + i Y_1. */
#define PMCIM_F_HELMHOLTZ_DLP 2

typedef struct {
  int32_t kind;   /* PMCIM_F_MONOMIAL, PMCIM_F_EXP_NEG or PMCIM_F_HELMHOLTZ_DLP */
  int32_t degree; /* monomial degree, 0..16                                     */
  double tau;     /* delay, used by PMCIM_F_EXP_NEG                             */
  double id_re;   /* when the coefficient pointer is NULL the term is           */
  double id_im;   /*   (id_re + i id_im) * I * f(z), never stored densely       */
} pmcim_fterm;

/* One disk: centre c, radius r, N trapezoid nodes (N even, 2..4096). */
typedef struct {
  double c_re;
  double c_im;
  double r;
  int32_t N;
  int32_t depth; /* split depth; callers pass 0 */
} pmcim_region;

/* Arithmetic of the LU factorisation (the solves are always refined to FP64
   accuracy when a reduced precision is chosen). */
#define PMCIM_PREC_FP64 0      /* plain FP64 LU                                  */
#define PMCIM_PREC_FP32_IR 1   /* FP32 LU + FP64 iterative refinement            */
#define PMCIM_PREC_AUTO 2      /* per problem, whichever of the forms solves
                                  nodes fastest on this device, measured on first
                                  use for each (n bucket, l, dense-term count) and
                                  kept for the process; all meet the same accuracy.
                                  A problem with a boundary-integral term takes
                                  PMCIM_PREC_FP32_IR without being timed */
#define PMCIM_PREC_TF32X3_IR 3 /* FP32 LU whose trailing updates are complex
                                  products on the tensor cores, each FP32 operand
                                  split into two TF32 parts (3 products per real
                                  product, FP32 accumulation), + FP64 refinement  */
#define PMCIM_PREC_BF16X3_IR 4 /* FP32 LU whose trailing updates are complex
                                  products in the 3M form (3 real products) on the
                                  tensor cores, each FP32 operand split into three
                                  BF16 parts (6 part products per real product,
                                  FP32 accumulation), + FP64 refinement           */

typedef struct {
  double tol_ind;          /* indicator threshold, paper default 0.1 (Sec. 3.1)        */
  double tol_svd;          /* absolute singular-value threshold, 1e-6 (Sec. 3.2)        */
  double tol_verify;       /* sigma_min acceptance, 1e-6 (pmCIMb step 3.b)              */
  int32_t precision;       /* PMCIM_PREC_*                                             */
  int32_t max_ir_sweeps;   /* refinement sweeps for reduced precision (default 6)      */
  int32_t max_split_depth; /* splits of saturated disks (default 8)                    */
  /* moment pairs of Beyn's step (default 1, Eq. 2.8 on C0 and C1). K > 1
     (at most 8, K l <= 64): the block Hankel matrices of the 2K moments
     M_p = sum_j w_j ((z_j - c)/r)^p X_j (Beyn's higher moments) take C0's and
     C1's places, so a disk holds up to K l eigenvalues before it is saturated
     and split. */
  int32_t beyn_K;
  void* cuda_stream;       /* cudaStream_t the call is ordered after; NULL = default   */
  /* learned screen (pmcim_solve / pmcim_batch_solve): NULL = off; else the
     PMCIM_SCREEN_PARAMS trained parameters (host or device). Every disk first
     gets the coarse indicators of screen_N nodes (one probe column); a disk
     skips the full indicator and Beyn (status PMCIM_RS_SCREENED) only when
     its screen probability is below screen_threshold and both coarse
     indicators (8 and 16 nodes) are at or below tol_ind; every other disk
     goes on exactly as without the screen. */
  const float* screen_params;
  double screen_threshold;
  int32_t screen_N;        /* coarse nodes, a multiple of 16 (default 16)            */
  /* pmcim_solve / pmcim_batch_solve / pmcim_beyn: 0 = one N per disk serves the
     indicator and Beyn; > 0 = the paper's two-pass schedule (Appendix pmCIMb
     driver): the indicator gates each disk on an indicator_N-node rule (even;
     every disk's N a multiple of it), then Beyn runs on the candidates with the
     disk's N, reusing the indicator pass's solves (its nodes are every
     (N / indicator_N)-th node of the full rule). Disks the indicator does not
     gate (depth-0 disks of pmcim_beyn) go straight to Beyn. */
  int32_t indicator_N;
  /* refinement stop (reduced precisions): a node's sweeps end when the estimated
     remaining error |delta_s|^2 / |delta_{s-1}| is at most tol_ir |X| (max
     norms); 0 = the default 1e-11. Must lie in [1e-15, 1e-6]. */
  double tol_ir;
  /* reduced precisions: where the refinement residuals R = V - T(z_j) X are
     formed. 0 (default): on the tensor cores, from exact BF16 digits of the
     coefficients and of f_k(z_j) X (7 digits of 7 bits each per number, the
     digit products accumulated exactly in FP32 and combined in FP64; about the
     accuracy of an FP64 product, see pmcim_residual). 1: on the FP64 pipe. */
  int32_t residual_fp64;
  /* FP64 node kernel: the trailing update's tile, 32 (32 x 32, less padding on
     small matrices) or 64 (64 x 64). 0 (default): 64, or under PMCIM_PREC_AUTO
     the autotuner's choice per (n bucket, l, dense terms), timed up to n = 256. */
  int32_t fp64_tile;
} pmcim_options;

/* Statistics of one pmcim_solve call. */
typedef struct {
  int64_t solves;          /* linear systems T(z_j) X = V solved (one per node)  */
  int32_t regions;         /* disks processed, children included                 */
  int32_t candidates;      /* disks with I > tol_ind                             */
  int32_t splits;          /* saturated disks split                              */
  int32_t unverified;      /* filtered values rejected by verification           */
  int32_t ir_fallbacks;    /* nodes re-solved in FP64 after refinement stalled  */
  int32_t singular_nodes;  /* nodes whose LU met an exactly zero pivot           */
  int64_t ir_sweeps;       /* refinement sweeps summed over nodes (FP32_IR)      */
  int32_t certified;       /* values accepted by the eigenvector certificate     */
  int32_t graphs;          /* CUDA graphs launched (one per level of disks)      */
  int32_t tuned_fp64;      /* problems the autotuner ran in FP64                 */
  int32_t tuned_mixed;     /* problems the autotuner ran in PMCIM_PREC_FP32_IR    */
  int32_t screened_out;    /* disks the learned screen skipped                   */
  int32_t screen_solves;   /* coarse node solves spent on the screen             */
  int32_t tuned_tc;        /* problems the autotuner ran in a tensor-core form
                              (PMCIM_PREC_TF32X3_IR or PMCIM_PREC_BF16X3_IR)      */
  int32_t tc_timeouts;     /* nodes whose tensor-core wait ran out (their LU was
                              finished on the FMA pipes or the node re-solved in
                              FP64; results stay refined)                        */
  int32_t node_ctas;       /* largest number of CTAs (one per SM) the precision
                              form's node kernel ran with in the call: fewer than
                              the SMs when device memory was short               */
} pmcim_stats;

typedef struct pmcim_problem_s* pmcim_problem;

/* Fill *opt with the paper's parameters (tol_ind 0.1, tol_svd 1e-6,
   tol_verify 1e-6), FP64, up to 6 refinement sweeps, split depth 8, default
   stream. */
void pmcim_default_options(pmcim_options* opt);

/* Create a problem handle for T(z) = sum_{k<K} f_k(z) A_k  (Sec. 1).
   A[k] points to n*n complex values (2*n*n doubles, column-major) or is NULL
   for the identity term (f[k].id_re + i f[k].id_im) * I; for a
   PMCIM_F_HELMHOLTZ_DLP term it points to the curve's 6 n samples. The handle
   copies the coefficients to the device; the caller may free A afterwards.
   Errors: EINVAL (n < 1, K < 1, K > 16, bad kind/degree, a boundary-integral
   term with odd n, n < 4, a NULL curve, a second such term, or a curve whose
   samples are not finite or coincide), ENOMEM, ECUDA. */
int pmcim_problem_create(int32_t n, int32_t K, const double* const* A, const pmcim_fterm* f,
                         pmcim_problem* out);
int pmcim_problem_destroy(pmcim_problem p);

/* Quadrature moments of each disk (Eq. 3.2-3.3 and the two P f sums of Eq. 3.1):
   at the nodes z_j = c + r e^{2 pi i j/N}, weights w_j = (r/N) e^{2 pi i j/N},
   X_j = T(z_j)^{-1} V is computed by LU with partial pivoting, and
     C0[g] = sum_j w_j X_j,  C1[g] = sum_j w_j z_j X_j          (n x l each),
     pf_half[g] = sum_{j odd} 2 w_j X_j[:,0]                   (n),
     pf_abs[g]  = sum_j |w_j| |X_j[:,0]|  elementwise           (n),
   so that P f|_N = C0[g][:,0] with f = V[:,0]. V is n x l with l in 1..64.
   Outputs are R consecutive blocks; any output may be NULL. */
int pmcim_moments(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
                  int32_t l, const double* V, double* C0, double* C1, double* pf_half,
                  double* pf_abs);

/* pmCIMb step 1 (Sec. 3.2; indicator of Eq. 3.1) for R disks:
   ind[g] = || C0[:,0] ./ pf_half ||_2 / sqrt(n), candidate[g] = ind[g] > tol_ind.
   pf_norm[g] = ||P f|_N||_2 and pf_scale[g] = ||pf_abs||_2 (a size of the summed
   terms, for judging whether P f is above rounding noise) may be NULL. */
int pmcim_indicator(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
                    int32_t l, const double* V, double* ind, double* pf_norm, double* pf_scale,
                    uint8_t* candidate);

/* pmCIMb step 2 (Sec. 3.2, steps 2.b-2.f; Eq. 2.8) on the given disks, without the
   indicator gate on them: SVD of C0, p = #{sigma > tol_svd}, D = V0^H C1 W0 Sigma0^-1,
   eig(D), eigenvectors V0 s (unit norm, largest entry real positive), square filter.
   A disk whose rank saturates (p = min(n,l)) is split into four children, which
   pass the indicator gate and are re-run, up to opt->max_split_depth.
   Output: *count values lambda[2*count], vecs[n*2*count] (may be NULL),
   region_of[count] (index of the input disk), region_status[R] (OR of the bits
   of the disk and its children; may be NULL). ECAPACITY if more than cap. */
int pmcim_beyn(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
               int32_t l, const double* V, int32_t cap, double* lambda, double* vecs,
               int32_t* region_of, int32_t* count, int32_t* region_status);

/* The residuals of m linear systems T(z_j) X_j = V (Eq. 2.4), R_j = V - T(z_j) X_j,
   formed as the precision forms' refinement forms them on the tensor cores
   (exact products of BF16 digits: every row of each dense A_k and every column
   of f_k(z_j) X_j is written as 48 bits in 7 digits of 7 bits, the digit pairs
   of total order <= 9 are multiplied with exact FP32 accumulation, and the
   results are combined in FP64; the error is of the order of 2^-47 of
   sum_i |A_k||f_k X|, comparable with an FP64 product). z: m complex points;
   V: n x l; X and R: m blocks of n x l (column-major, complex). ETIMEOUT if a
   bounded wait of the kernel ran out (R not valid). */
int pmcim_residual(pmcim_problem p, const pmcim_options* opt, int32_t m, const double* z, int32_t l,
                   const double* V, const double* X, double* R);

/* pmCIMb step 3: sigma_min[i] = smallest singular value of T(lambda_i) by LU and
   inverse iteration on (T^H T)^{-1}; accept[i] = sigma_min <= tol_verify *
   max(1, ||T(lambda_i)||_F / sqrt(n)). accept may be NULL. */
int pmcim_verify(pmcim_problem p, const pmcim_options* opt, int32_t m, const double* lambda,
                 double* sigma_min, uint8_t* accept);

/* Certificates of approximate eigenpairs (pmCIMb step 3 without the full
   sigma_min). For each lambda_i (m complex) with start vector c_i (column i of
   vecs, n x m complex column-major, host or device memory; c_i != 0; normally an
   approximate right eigenvector), an upper bound of sigma_min(T(lambda_i)):
   first ||T c_i|| / ||c_i||; where that does not accept the value, also
   ||T^H y|| / ||y|| for the bordered inverse-iteration step y = T(lambda_i)^-H c_i
   (FP32 LU of T^H with column s = argmax |c_i| replaced by c_i, residuals in FP64,
   FP32 corrections; a plain FP64 solve for n <= 32). sigma_min(T^H) =
   sigma_min(T), and from an approximate right eigenvector the second bound comes
   close to sigma_min itself. cert[i] = the smaller bound; accept[i] = cert[i] <=
   tol_verify * max(1, ||T(lambda_i)||_F / sqrt(n)), so an accepted value is one
   the sigma_min rule of pmcim_verify accepts; a value not accepted is undecided
   (only the full sigma_min can reject). accept may be NULL. */
int pmcim_certify(pmcim_problem p, const pmcim_options* opt, int32_t m, const double* lambda,
                  const double* vecs, double* cert, uint8_t* accept);

/* pmCIMa (Sec. 3.1): the spectral indicator alone, level by level. Each level
   computes the indicator (Eq. 3.1, the disk's N nodes, probe column V, n x 1)
   of every disk; a candidate (I > tol_ind) is quadrisected into four disks of
   half the radius centred at the centres of its square's quarters, until the
   disk's level count L = ceil(log2(r / tol_eps)) + 2 (the Appendix listing's
   count; the last disks' radius is at most tol_eps / 2). The last level's
   candidate centres approximate the eigenvalues (step 1.c); centres closer than
   tol_eps are merged into their mean (the remark after the algorithm). Step 2:
   sigma_min of T(lambda) and its unit right singular vector, by FP64 LU and
   inverse iteration as in pmcim_verify. Outputs: lambda (cap complex, sorted by
   real then imaginary part), vecs (n x cap, may be NULL), sigma_min (cap, may
   be NULL), *count; stats may be NULL. ECAPACITY when more than cap values
   (*count holds the number), or when a level exceeds 2^20 disks. */
int pmcim_pmcima(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
                 const double* V, double tol_eps, int32_t cap, double* lambda, double* vecs,
                 double* sigma_min, int32_t* count, pmcim_stats* stats);

/* Whole pmCIMb (steps 1-3) over R disks with one N per disk for both the
   indicator and the moments: one LU per node serves both. Outputs the verified
   eigenvalues (sorted by real, then imaginary part) with eigenvectors (may be
   NULL), sigma_min and source disk; ind[R] and region_status[R] may be NULL;
   stats may be NULL. ECAPACITY if more than cap values are verified.
   Verification first evaluates, in FP64, the certificate ||T(lambda) v|| of
   the unit eigenvector v from Beyn's step; since sigma_min <= ||T(lambda) v||,
   a value whose certificate is already below the acceptance threshold is
   accepted, and sigma_min[i] then holds that certificate (an upper bound of
   the smallest singular value). A value it does not accept gets the bordered
   inverse-iteration step of pmcim_certify from v and its certificate (again an
   upper bound of sigma_min). Every value still not accepted gets the full
   sigma_min of pmcim_verify. Accept/reject decisions equal those of the
   sigma_min rule. */
int pmcim_solve(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
                int32_t l, const double* V, int32_t cap, double* lambda, double* vecs,
                double* sigma_min, int32_t* region_of, int32_t* count, double* ind,
                int32_t* region_status, pmcim_stats* stats);

/* One problem of a batch: its handle, disks and probe block (as in pmcim_solve). */
typedef struct {
  pmcim_problem problem;
  int32_t R;
  const pmcim_region* regions;
  int32_t l;
  const double* V;
} pmcim_batch_item;

/* pmCIMb (steps 1-3) for P independent problems of any sizes in one call: the
   nodes of every disk of every problem form one work list per level, solved by
   one persistent launch per arithmetic form (largest n first), and each level
   is launched as one CUDA graph. Options apply to all problems; with
   PMCIM_PREC_AUTO each problem gets the faster form for its size. Outputs the
   verified eigenvalues of all problems sorted by (problem, Re, Im), with
   sigma_min (as in pmcim_solve), the problem index and the index of the disk
   within that problem's list; any of them may be NULL except lambda and count.
   A handle may appear only once per batch; while the call runs, none of its
   handles may be used by another thread. ECAPACITY if more than cap values. */
int pmcim_batch_solve(int32_t P, const pmcim_batch_item* items, const pmcim_options* opt, int32_t cap,
                      double* lambda, double* sigma_min, int32_t* problem_of, int32_t* region_of,
                      int32_t* count, pmcim_stats* stats);

/* ---- learned screen (no counterpart in the paper; it decides which disks
   need the full indicator of Eq. 3.1) ------------------------------------
   Features of a disk: (log10 I_8, log10 I_16, log10 r), with I_M the ratio
   indicator of Eq. 3.1 on the first M nodes of the disk's trapezoid rule
   (M divides N). Network: 3 -> 64 -> 64 -> 1, ReLU, sigmoid output, FP32
   master parameters in the order W1[64][3], b1[64], W2[64][64], b2[64],
   W3[64], b3; the forward and backward passes use their BF16 rounding with
   FP32 accumulation. */
#define PMCIM_SCREEN_PARAMS 4481

/* Indicators I_8, I_16 and I_N (ind3, R x 3) and the features (feats, R x 3
   floats) of R disks; N must be a multiple of 16; f = V[:,0]. Any output may
   be NULL. */
int pmcim_screen_features(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
                          int32_t l, const double* V, double* ind3, float* feats);

/* Train on M samples (features row-major M x 3, labels 0/1) with Adam for
   `epochs` passes in the given order, minibatches of `batch`, class weight
   pos_weight on the positives. params (PMCIM_SCREEN_PARAMS floats) holds the
   initial values on entry and the trained ones on return. epoch_loss
   (epochs doubles, may be NULL) receives each epoch's mean weighted
   cross-entropy. */
int pmcim_screen_train(int32_t M, const float* feats, const uint8_t* labels, int32_t epochs, int32_t batch,
                       double lr, double pos_weight, float* params, double* epoch_loss, void* cuda_stream);

/* Screen probabilities of M feature rows. */
int pmcim_screen_apply(int32_t M, const float* feats, const float* params, float* prob, void* cuda_stream);

/* Gradient (PMCIM_SCREEN_PARAMS floats) and value of the mean weighted loss
   over M samples at the BF16 rounding of params (for checking the training
   kernels against an independent implementation). */
int pmcim_screen_gradient(int32_t M, const float* feats, const uint8_t* labels, double pos_weight,
                          const float* params, float* grad, double* loss, void* cuda_stream);

const char* pmcim_status_string(int code);
const char* pmcim_last_error(void);

/* Node solves that allocate nothing (the paper has no counterpart; this serves
   callers that cannot allocate device memory while they run, e.g. a host
   application whose own pool owns all device memory, or a latency-bound loop
   that must not stall on the device-wide synchronisation of cudaFree).
   Computes X_j = T(z_j)^{-1} V for j < m with the same assembly, LU with
   partial pivoting and solve as pmcim_moments, at the caller's points z.
   Arguments: f[K] and dense[K] (host; dense[k] != 0 means term k has a dense
   coefficient), A = the dense coefficients in term order, each n*n complex
   column-major, contiguous (device); z = m complex points (device); V = n x l
   complex column-major (device); X = m blocks of n x l complex (device,
   output); info = m int32 (device, output, may be NULL): 0, or 1 + the first
   column whose pivot was exactly zero.
   Workspace: a fixed 32 MiB array compiled into the library, held by every GPU
   that loads it until the process exits. A problem whose one-CTA workspace,
   n (n + l) * 16 + n * 4 bytes, exceeds 32 MiB (n above about 1440 at l = 16)
   is rejected with PMCIM_ENOTSUP. Every call looks up the array's device
   address (cudaGetSymbolAddress, which allocates nothing) with the calling
   thread's current device, so the address stays right after the host
   application resets the device and its context is created again. Every call
   shares the array, so calls that overlap on the GPU race; nothing in it needs
   clearing between calls. Synchronous on cuda_stream. No cudaMalloc, no
   cudaFree. */
int pmcim_solve_points_noalloc(int32_t n, int32_t K, const pmcim_fterm* f, const uint8_t* dense,
                               const double* A, int32_t m, const double* z, int32_t l, const double* V,
                               double* X, int32_t* info, void* cuda_stream);

/* ---- instrumentation (no counterpart in the paper) ----------------------
   Every kernel launch of the library is counted per kernel kind. When timing
   is enabled, CUDA events are recorded around each launch on the stream it is
   launched on, and the elapsed device time is accumulated once the calling
   API function has synchronised that stream. Process-wide, thread-safe. */
#define PMCIM_K_FACTOR 0  /* assembly + LU + solve at the nodes (FP64)       */
#define PMCIM_K_REDUCE 1  /* segmented quadrature reduction                  */
#define PMCIM_K_INDICATOR 2
#define PMCIM_K_BEYN 3
#define PMCIM_K_VERIFY 4
#define PMCIM_K_GATHER 5
#define PMCIM_K_FACTOR32 6 /* assembly + LU + solve at the nodes (FP32 LU)   */
#define PMCIM_K_SCREEN 7   /* learned screen: MLP forward / training          */
#define PMCIM_K_COUNT 8
#define PMCIM_PHASE_COUNT 16

typedef struct {
  int64_t launches[PMCIM_K_COUNT];
  double ms[PMCIM_K_COUNT]; /* summed event time; 0 unless timing was on */
  /* precision-form node kernel, with timing on: SM clock cycles summed over
     CTAs per phase: assembly, LU panels, first solve, FP64 residual,
     correction solves, FP64 fallback, node set-up, LU triangular solves
     (U12), LU trailing updates, factor group waiting for a free slot, refine
     group waiting for a factored node, then the CTAs' lifetimes in ns
     (globaltimer, summed), then the LU panels' row interchanges on the columns
     outside the panel (counted apart from the panels); 3 unused */
  double mixed_phase_cycles[PMCIM_PHASE_COUNT];
} pmcim_profile;

void pmcim_profile_enable(int on);
void pmcim_profile_reset(void);
void pmcim_profile_read(pmcim_profile* out);

/* Limits, in SM clock cycles, of the two kinds of bounded device waits in the
   precision-form node kernel (no counterpart in the paper; for testing the
   paths taken when a wait runs out). tc_wait_cycles bounds each wait for a
   tensor-core commit inside the LU's trailing update: when one runs out the
   node's LU is finished on the FMA pipes, the node is counted in
   stats.tc_timeouts, and its refinement (or its FP64 re-solve) still delivers
   an FP64-accurate solution. handoff_wait_cycles bounds each wait between the
   kernel's two thread groups: when one runs out both groups end and the call
   returns PMCIM_ETIMEOUT; the handle stays usable. 0 restores a default
   (2^30 and 2^35 cycles, about 0.5 s and 16 s at 2 GHz). Process-wide; takes
   effect for launches prepared after the call. The final wait for a commit in
   flight before the kernel frees its tensor memory always uses the default.
   EINVAL for a negative limit. */
int pmcim_debug_wait_limits(int64_t tc_wait_cycles, int64_t handoff_wait_cycles);

#ifdef __cplusplus
}
#endif
#endif /* PMCIM_H */
