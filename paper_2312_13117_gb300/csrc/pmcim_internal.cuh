// Internal declarations shared by the CUDA translation units of libpmcim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pmcim.h"

#define PMCIM_MAX_TERMS 16
#define PMCIM_MAX_L 64

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
__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }
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
__device__ __forceinline__ double l1abs(float2 a) { return (double)(fabsf(a.x) + fabsf(a.y)); }
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
__device__ __forceinline__ double2 eval_f(const TermDesc& t, double2 z) {
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

// Work item of the factor/solve kernels: one node of one disk.
struct RegionDev {
  double cre, cim, r;
  int32_t N;
  int32_t node_off;  // index of node 0 of this disk in the node list of the launch
};

// ---------------------------------------------------------------------------
// Launchers (host side), implemented in the .cu files.
// ---------------------------------------------------------------------------
struct FactorArgs {
  ProblemDesc prob;
  const double2* A;         // device, n_dense * n * n
  const double2* V;         // device, n x l
  int l;
  const RegionDev* regions; // device
  const int32_t* node_region;  // device, per node: region index
  int n_nodes;
  double2* X;               // device, n_nodes * n * l
  int32_t* node_info;       // device, per node: 0 or 1 + first zero-pivot column
  double2* work;            // device, slots * n * (n + l)
  int32_t* piv;             // device, slots * n
  int slots;
};
cudaError_t launch_factor_solve_fp64(const FactorArgs& a, cudaStream_t s);
int factor_slots_fp64(int n, int l);
size_t factor_smem_fp64();

struct MixedArgs {
  ProblemDesc prob;
  const double2* A;
  const double2* V;
  int l;
  const RegionDev* regions;
  const int32_t* node_region;
  int n_nodes;
  double2* X;               // FP64 solutions, n_nodes * n * l
  int32_t* node_info;       // bits 0-23: 0 or 1 + zero-pivot column; 24-29: sweeps; 30: FP64 fallback
  char* work;               // slots * slot_bytes
  size_t slot_bytes;
  int32_t* piv;             // slots * n
  int slots;
  int max_sweeps;
  double tol_ir;
  unsigned long long* phase;  // NULL, or slots * PMCIM_PHASES clock64 counters
};
// Phases of the precision-form node kernel timed with clock64 when profiling.
#define PMCIM_PHASES 8  // assemble, LU, first solve, residual, correction solve, fallback, other
__host__ __device__ inline size_t mixed_residual_offset(int n, int l) {
  return (((size_t)n * (n + l) * 8) + 255) & ~(size_t)255;
}
size_t mixed_slot_bytes(int n, int l);
cudaError_t launch_factor_solve_mixed(const MixedArgs& a, cudaStream_t s);

struct ReduceArgs {
  const double2* X;
  int n, l;
  const RegionDev* regions;
  int R;
  double2* C0;       // R * n * l
  double2* C1;       // R * n * l
  double2* pf_half;  // R * n
  double* pf_abs;    // R * n
};
cudaError_t launch_reduce_moments(const ReduceArgs& a, cudaStream_t s);

struct IndicatorArgs {
  const double2* C0;
  const double2* pf_half;
  const double* pf_abs;
  int n, l, R;
  double tol_ind;
  double* ind;
  double* pf_norm;
  double* pf_scale;
  uint8_t* candidate;
};
cudaError_t launch_indicator(const IndicatorArgs& a, cudaStream_t s);

struct BeynArgs {
  const double2* C0;         // per region slot, n x l
  const double2* C1;
  const int32_t* slot_of;    // per candidate: slot index into C0/C1
  const RegionDev* regions;  // per candidate: geometry
  int n, l, m;               // m candidates
  double tol_svd;
  double2* work;             // m * n * l  (rotated columns)
  double* sigma;             // m * l (descending)
  int32_t* p;                // m
  double2* lam;              // m * l
  double2* vecs;             // m * n * l
  uint8_t* kept;             // m * l
  int32_t* status;           // m
};
cudaError_t launch_beyn(const BeynArgs& a, cudaStream_t s);

struct VerifyArgs {
  ProblemDesc prob;
  const double2* A;
  const double2* lam;        // m
  int m;
  double tol_verify;
  double* sigma_min;         // m
  uint8_t* accept;           // m
  double2* work;             // slots * n * n
  double2* vec;              // slots * 3 * n
  int32_t* piv;              // slots * n
  int slots;
};
cudaError_t launch_verify_fp64(const VerifyArgs& a, cudaStream_t s);
int verify_slots_fp64(int n);

struct CertifyArgs {
  ProblemDesc prob;
  const double2* A;
  const double2* lam;        // m
  const double2* vecs;       // m * n, unit eigenvectors
  int m;
  double tol_verify;
  double* cert;              // m: ||T(lambda) v|| / ||v||
  uint8_t* certified;        // m: cert <= tol_verify * max(1, ||T||_F / sqrt(n))
};
cudaError_t launch_certify(const CertifyArgs& a, cudaStream_t s);

struct GatherArgs {
  const double2* vecs;       // m * n * l (beyn outputs)
  const int32_t* src;        // count: cand * l + k
  double2* dst;              // count * n
  int n, l, count;
};
cudaError_t launch_gather_vecs(const GatherArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launch accounting (api.cu): count every launch; with timing on, bracket it
// with events on its stream. prof_flush() resolves pending events after the
// caller has synchronised the stream.
// ---------------------------------------------------------------------------
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s);
void prof_flush();
