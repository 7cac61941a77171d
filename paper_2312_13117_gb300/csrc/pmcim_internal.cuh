// Internal declarations shared by the CUDA translation units of libpmcim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pmcim.h"
#include "bie.cuh"

#define PMCIM_MAX_TERMS 16
// ||P f|_N|| at or below this fraction of ||sum_j |w_j| |x_j||| counts as zero
constexpr double kPfFloor = 1e-10;
#define PMCIM_MAX_L 64
#define PMCIM_MAX_BEYN_K 8  // moment pairs of the block Hankel form of Beyn's step

// ---------------------------------------------------------------------------
// Complex helpers on double2 / float2 (re, im). Division uses Smith's scaling
// (R. L. Smith, CACM 1962) so that |b| near the overflow or underflow limits
// does not overflow the denominator.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// acc -= a * b
__device__ __forceinline__ void cfms(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// 1 / b  (Smith)
__host__ __device__ __forceinline__ double2 crecip(double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double t = b.y / b.x, d = b.x + b.y * t;
    return make_double2(1.0 / d, -t / d);
  } else {
    double t = b.x / b.y, d = b.x * t + b.y;
    return make_double2(t / d, -1.0 / d);
  }
}
// a / b  (Smith)
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double t = b.y / b.x, d = b.x + b.y * t;
    return make_double2((a.x + a.y * t) / d, (a.y - a.x * t) / d);
  } else {
    double t = b.x / b.y, d = b.x * t + b.y;
    return make_double2((a.x * t + a.y) / d, (a.y * t - a.x) / d);
  }
}
__device__ __forceinline__ double l1abs(double2 a) { return fabs(a.x) + fabs(a.y); }

// float2 counterparts used by the FP32 factorisation
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cfms(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ float2 crecip(float2 b) {
  if (fabsf(b.x) >= fabsf(b.y)) {
    float t = b.y / b.x, d = b.x + b.y * t;
    return make_float2(1.0f / d, -t / d);
  } else {
    float t = b.x / b.y, d = b.x * t + b.y;
    return make_float2(t / d, -1.0f / d);
  }
}
__host__ __device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  if (fabsf(b.x) >= fabsf(b.y)) {
    float t = b.y / b.x, d = b.x + b.y * t;
    return make_float2((a.x + a.y * t) / d, (a.y - a.x * t) / d);
  } else {
    float t = b.x / b.y, d = b.x * t + b.y;
    return make_float2((a.x * t + a.y) / d, (a.y * t - a.x) / d);
  }
}
__device__ __forceinline__ float l1abs(float2 a) { return fabsf(a.x) + fabsf(a.y); }
template <typename T2> __device__ __forceinline__ T2 czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.0f, 0.0f); }
__device__ __forceinline__ bool cis_zero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
__device__ __forceinline__ bool cis_zero(float2 a) { return a.x == 0.0f && a.y == 0.0f; }

// ---------------------------------------------------------------------------
// Problem description as the kernels see it.
// ---------------------------------------------------------------------------
struct TermDesc {
  int32_t kind;
  int32_t degree;
  double tau;
  double2 id;          // identity coefficient when dense == 0
  int32_t dense;       // 1: coefficient is the dense matrix at offset mat_index * n * n
  int32_t mat_index;
};

struct ProblemDesc {
  int32_t n;
  int32_t K;
  int32_t n_dense;
  TermDesc term[PMCIM_MAX_TERMS];
};

// f_k(z) for one term (Sec. 1 problem class with the fixed scalar-function set).
// A boundary-integral term's entries depend on z itself: its value is z.
__device__ __forceinline__ double2 eval_f(const TermDesc& t, double2 z) {
  if (t.kind == PMCIM_F_HELMHOLTZ_DLP) return z;
  if (t.kind == PMCIM_F_MONOMIAL) {
    double2 p = make_double2(1.0, 0.0);
    for (int d = 0; d < t.degree; ++d) p = cmul(p, z);
    return p;
  }
  // exp(-tau z) = exp(-tau x) (cos(tau y) - i sin(tau y))
  double m = exp(-t.tau * z.x);
  double s, c;
  sincos(t.tau * z.y, &s, &c);
  return make_double2(m * c, -m * s);
}

// Node z_j and weight w_j = (r/N) e^{i theta_j}, theta_j = 2 pi j / N (Eq. 3.2).
__device__ __forceinline__ void node_weight(double cre, double cim, double r, int N, int j, double2* z,
                                            double2* w) {
  double s, c;
  sincospi(2.0 * (double)j / (double)N, &s, &c);
  *z = make_double2(cre + r * c, cim + r * s);
  double h = r / (double)N;
  *w = make_double2(h * c, h * s);
}

// ---------------------------------------------------------------------------
// Batched work description. One launch can carry nodes of many problems of
// different sizes: every disk names its problem and the offsets of its blocks.
// ---------------------------------------------------------------------------
struct ProblemDev {
  int32_t n, K, l, n_dense;
  const double2* A;    // n_dense * n * n, column-major, in term order
  const double2* V;    // n x l probe block
  const float2* A32;   // the same coefficients rounded to complex64 (FP32 LU assembly)
  // the coefficients as exact BF16 digits for the tensor-core refinement residual
  // (ozaki.cuh; NULL until made), and the row exponents [dense term][row blocks x 128]
  const unsigned char* Adig;
  const int32_t* Aexp;
  // geometry of the boundary-integral term (bie.cuh, 6 n + 1 doubles), NULL without one
  const double* bie;
  int32_t bie_circ;  // 1: its matrix is circulant (the curve is invariant under t_j -> t_{j+1})
  TermDesc term[PMCIM_MAX_TERMS];
};

// Entry (row, col) of one non-dense term: the identity term's diagonal, or the
// boundary-integral term's c K_n(z) entry (fz = z for it). Dense terms are read by
// the callers from the coefficients. The kernels that assemble T are instantiated
// twice: BIE = false (no problem of the launch has a boundary-integral term) leaves
// out the entry's code and its registers.
template <bool BIE>
__device__ __forceinline__ void cfma_term(double2& v, const ProblemDev& P, const TermDesc& t, double2 fz, int row,
                                          int col) {
  if (BIE && t.kind == PMCIM_F_HELMHOLTZ_DLP) cfma(v, t.id, bie::dlp_entry(P.bie, P.n, row, col, fz));
  else if (row == col) cfma(v, fz, t.id);
}

struct RegionDev {
  double cre, cim, r;
  int32_t N;
  int32_t prob;      // index into the problem table
  int32_t node_off;  // index of node 0 in the launch's node_info array
  int32_t gate;      // 1: Beyn runs only when the indicator marks a candidate
  int32_t lu_tc;     // the precision form's trailing updates: 0 FMA pipes, 1 tensor cores in
                     // 3xTF32, 2 tensor cores in BF16 3M
  int32_t border;    // 0, or s + 1: the node solves the bordered system of a certificate, T(z)
                     // (T(z)^H when herm) with column s replaced by the column at NodeArgs::border + v_off
  int32_t herm;      // 1: the node's matrix is T(z)^H (precision form: FP64-pipe residuals, t64 set)
  int64_t x_off;     // double2 offset of node 0's solution in X (node j at x_off + j n l)
  int64_t c_off;     // double2 offset of the disk's C0 / C1 blocks (n l)
  int64_t p_off;     // offset of the disk's P f blocks (n)
  int64_t w_off;     // double2 offset of the disk's Beyn scratch (2 n l + 4 l^2)
  int64_t v_off;     // double2 offset of the disk's eigenvector block (n l)
};

struct NodeItem {
  int32_t region;
  int32_t j;
};

// Copy a problem descriptor into shared memory (all threads; caller syncs).
__device__ __forceinline__ void load_problem(ProblemDev* dst, const ProblemDev* src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(ProblemDev) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

// ---------------------------------------------------------------------------
// Launchers (host side), implemented in the .cu files.
// ---------------------------------------------------------------------------
struct NodeArgs {
  const ProblemDev* probs;
  const RegionDev* regions;
  const NodeItem* items;    // in scheduling order (largest n first)
  int n_items;
  int* counter;             // work counter, zero before the launch
  double2* X;
  int32_t* node_info;       // FP64: 0 or 1 + zero-pivot column. Mixed: bits 0-23 the same,
                            // 24-29 sweeps run, 30 FP64 fallback
  char* work;               // slots * slot_bytes
  size_t slot_bytes;
  int32_t* piv;             // slots * max_n
  int max_n;
  int slots;
  int max_sweeps;             // mixed kernel: refinement sweeps; 0 = the FP32 solve only
  double tol_ir;
  unsigned long long* phase;  // NULL, or slots * PMCIM_PHASES clock64 counters (mixed kernel)
  int32_t* err;               // mixed kernel: set to 1 when a wait between its thread groups ran out
  double2* t64;               // mixed kernel: per slot, T(z_j) in FP64 for the residuals (problems
  size_t t64_stride;          // with two or more dense terms); double2 elements per slot
  int oz;                     // mixed kernel: 1 = refinement residuals on the tensor cores
  unsigned char* ysl;         // mixed kernel: per slot, the digits of f_k X (ozaki.cuh)
  size_t ysl_stride;          // bytes per slot
  long long tc_wait_cycles;       // mixed kernel: limit of a wait for a tensor-core commit
  long long handoff_wait_cycles;  // mixed kernel: limit of a wait between its thread groups
  const double2* border;          // mixed kernel: the replacement columns of bordered nodes
  int fp64_tile;                  // FP64 kernel: trailing-update tile, 32 or 64 (0: 64)
  int bie;                        // FP64 and small kernels: a problem has a boundary-integral term
};
// Limits of the precision-form kernel's bounded waits (clock64 cycles): the
// defaults, or the values a test set with pmcim_debug_wait_limits.
long long wait_limit_tc();
long long wait_limit_handoff();
cudaError_t prepare_factor_fp64();   // shared-memory limits; call outside graph capture
cudaError_t prepare_factor_mixed();
cudaError_t launch_factor_solve_fp64(const NodeArgs& a, cudaStream_t s);
cudaError_t launch_factor_solve_mixed(const NodeArgs& a, cudaStream_t s);
int mixed_slots_per_cta();  // workspace slots each CTA of the mixed kernel cycles through
// dst[i] = complex64(src[i]), i < count (the FP32 copy of the coefficients)
cudaError_t round_coefficients_c64(const double2* src, float2* dst, size_t count, cudaStream_t s);
// Exact BF16 digits of the n_dense dense coefficients (ozaki.cu): row exponents
// into exps ([n_dense][row blocks x 128]) and digit tiles into dig.
cudaError_t make_coefficient_digits(const double2* A, int n, int n_dense, int32_t* exps, unsigned char* dig,
                                    cudaStream_t s);
// Bytes of the coefficient digits of a problem, and of one slot's digits of f_k X.
size_t coefficient_digit_bytes(int n, int n_dense);
size_t y_digit_scratch_bytes(int n, int n_dense);
// R_j = V - T(z_j) X_j for m points, one node per CTA, on the tensor cores
// (ozaki.cu). ysl: per-CTA Y-digit scratch of ysl_stride bytes for `ctas` CTAs;
// status[j] = 0, or 1 when a wait ran out (R_j not valid).
cudaError_t launch_residual_points(const ProblemDev* prob, const double2* z, int m, const double2* X, double2* R,
                                   unsigned char* ysl, size_t ysl_stride, int ctas, int32_t* status,
                                   long long wait_cycles, cudaStream_t s);
// warp-per-node FP64 kernel for small problems (lu_small.cu)
bool small_kernel_fits(int n, int l);
cudaError_t prepare_factor_small();
cudaError_t launch_factor_solve_small(const NodeArgs& a, cudaStream_t s);
int factor_slots_fp64(int n, int l);
// Phases of the precision-form node kernel timed with clock64 when profiling.
// assemble, LU panels, first solve, residual, correction solves, fallback, set-up,
// LU triangular solves, LU trailing updates, 3 unused
#define PMCIM_PHASES PMCIM_PHASE_COUNT
__host__ __device__ inline size_t mixed_residual_offset(int n, int l) {
  return (((size_t)n * (n + l) * 8) + 255) & ~(size_t)255;
}
// the LU panels' row permutations (ints), after the FP64 residual
__host__ __device__ inline size_t mixed_lists_offset(int n, int l) {
  return (mixed_residual_offset(n, l) + (size_t)n * l * 16 + 255) & ~(size_t)255;
}
size_t mixed_slot_bytes(int n, int l);

struct LevelArgs {
  const ProblemDev* probs;
  const RegionDev* regions;
  int R;
  int max_nl;
  const double2* X;
  double2* C0;
  double2* C1;
  int K;                    // 1: Beyn on C0, C1 (Eq. 2.8); > 1: block Hankel of 2K scaled moments
  double2* Cm;              // K > 1: per disk 2K blocks n x l at 2K c_off: M_p = sum_j w_j e^{i p theta_j} X_j
  double2* pf_half;
  double* pf_abs;
  double tol_ind;
  double tol_svd;
  double* ind;
  double* pf_norm;
  double* pf_scale;
  uint8_t* cand;
  // Beyn outputs; sigma, lam, kept are indexed g * PMCIM_MAX_L + k
  double2* bwork;
  double* sigma;
  int32_t* p;               // -1 when the disk was gated out
  double2* lam;
  double2* vecs;            // at region.v_off
  uint8_t* kept;
  int32_t* status;
};
cudaError_t launch_reduce_moments(const LevelArgs& a, cudaStream_t s);
cudaError_t launch_indicator(const LevelArgs& a, cudaStream_t s);
cudaError_t launch_beyn(const LevelArgs& a, cudaStream_t s);

struct ValueArgs {
  const ProblemDev* probs;
  const int32_t* prob_of;   // per value
  const double2* lam;
  const int64_t* vec_off;   // certificate: double2 offset of the value's unit eigenvector
  const double2* vecs;
  int m;
  double tol_verify;
  double* sigma;
  uint8_t* accept;
  double2* work;            // verify: slots * max_n * max_n
  double2* vec;             // verify: slots * 3 * max_n
  int32_t* piv;             // verify: slots * max_n
  int slots;
  int max_n;
  double2* vec_out;         // verify: NULL, or m * max_n: the unit right singular vector for sigma_min
  int herm;                 // certificate: 1 = ||T(lambda)^H v|| (sigma_min(T^H) = sigma_min(T))
  int bie;                  // a problem has a boundary-integral term (k_certify, k_verify_fp64)
};
cudaError_t launch_certify(const ValueArgs& a, cudaStream_t s);
// Certificates from coefficient products (reduce.cu), for problems with 1 to
// gram_max_dense() dense terms: launch_gram fills gram_entries() values of a
// problem's Gram data (partial: gram_partial_count() x gram_entries() scratch);
// launch_apply_dense forms W_d = A_d [v_1 .. v_m] (n x m per dense term d, the
// vectors at vecs + vec_off[i]); launch_certify_products then evaluates each
// value's certificate from its problem's W (column w_col[i], w_m[i] values) and
// Gram data (gram + prob_of[i] x gram_entries()).
size_t gram_partial_count();
size_t gram_entries();
int gram_max_dense();
cudaError_t launch_gram(const ProblemDev* prob, double2* partial, double2* gram, cudaStream_t s);
cudaError_t launch_apply_dense(const ProblemDev* prob, int n, int n_dense, const double2* vecs,
                               const int64_t* vec_off, int m, double2* W, cudaStream_t s);
cudaError_t launch_certify_products(const ValueArgs& a, const double2* W, const int64_t* w_col, const int32_t* w_m,
                                    const double2* gram, cudaStream_t s);
cudaError_t launch_verify_fp64(const ValueArgs& a, cudaStream_t s);

// learned screen (screen.cu)
cudaError_t launch_screen_features(const LevelArgs& a, double* ind3, cudaStream_t s);
cudaError_t launch_make_features(int R, const double* ind3, const RegionDev* regions, float* feats, cudaStream_t s);
cudaError_t screen_forward(int M, const float* d_feats, const float* d_params, float* d_prob, void* d_scratch,
                           cudaStream_t s);  // scratch: 2 * PMCIM_SCREEN_PARAMS bytes
size_t screen_grad_scratch_bytes(int B);
size_t screen_train_scratch_bytes(int B);
cudaError_t screen_gradient(int B, const float* d_feats, const uint8_t* d_labels, float pos_weight,
                            const float* d_params, float* d_grad, double* d_loss, void* d_scratch, cudaStream_t s);
cudaError_t screen_train(int M, const float* d_feats, const uint8_t* d_labels, int epochs, int B, float lr,
                         float pos_weight, float* d_params, double* d_epoch_loss, void* d_scratch, cudaStream_t s);

struct VecItem {
  int64_t src;   // double2 offset in the source
  int64_t dst;   // double2 offset in the destination
  int32_t n;
  int32_t pad;
};
// A certificate's bordered inverse step (reduce.cu): for each value m with
// off[m] >= 0, the start vector at vecs + vec_off[m] gives the replaced column s
// (regions[m].border = s + 1), b = -T e_s at out + off[m] and the scaled
// replacement column after it; T = T(lambda), or T(lambda)^H when a.herm.
cudaError_t launch_border_rhs(const ValueArgs& a, const int64_t* off, double2* out, RegionDev* regions,
                              cudaStream_t s);
cudaError_t launch_gather_vecs(const double2* src, double2* dst, const VecItem* items, int count, int max_n,
                               cudaStream_t s);

// ---------------------------------------------------------------------------
// Launch accounting (api.cu): count every launch; with timing on, bracket it
// with events on its stream. prof_flush() resolves pending events after the
// caller has synchronised the stream.
// ---------------------------------------------------------------------------
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s);
void prof_flush();
