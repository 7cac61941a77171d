// Coefficient digits for the tensor-core refinement residual, and a residual
// kernel over explicit points (ozaki.cuh describes the splitting).
#include "ozaki.cuh"

namespace {

using namespace lucore;

// Row exponents of every dense coefficient: exps[d][i] = e with
// max_j max(|Re a_ij|, |Im a_ij|) <= 2^e (0 for an all-zero or padding row).
__global__ void k_coeff_exponents(const double2* __restrict__ A, int n, int npad, int32_t* __restrict__ exps) {
  const int d = blockIdx.y;
  const size_t nn = (size_t)n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    double m = 0.0;
    if (i < n)
      for (int j = 0; j < n; ++j) {
        const double2 a = A[d * nn + (size_t)j * n + i];
        m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
      }
    exps[(size_t)d * npad + i] = ozk::exponent_of(m);
  }
}

// Digit tiles of one (term d, row block rb, inner chunk kc): thread t takes row
// t % 128 and the 16 inner indices 16 (t / 128) .. + 15, as two groups of 8 that
// become one 16-byte store per digit and part.
__global__ void __launch_bounds__(256) k_coeff_digits(const double2* __restrict__ A, int n, int RB, int KCN,
                                                      const int32_t* __restrict__ exps,
                                                      unsigned char* __restrict__ dig) {
  const int kc = blockIdx.x, rb = blockIdx.y, d = blockIdx.z;
  const int r = threadIdx.x & 127, h = threadIdx.x >> 7;
  const int i = rb * ozk::TM + r;
  const size_t nn = (size_t)n * n;
  const int e = exps[(size_t)d * RB * ozk::TM + i];
  unsigned char* base = dig + (((size_t)d * RB + rb) * KCN + kc) * ozk::S * ozk::A_STAGE;
  for (int grp = 0; grp < 2; ++grp) {
    const int k0 = 16 * h + 8 * grp;
    long long Nr[8], Ni[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = kc * ozk::KC + k0 + u;
      double2 a = make_double2(0.0, 0.0);
      if (i < n && j < n) a = A[d * nn + (size_t)j * n + i];
      Nr[u] = __double2ll_rn(scalbn(a.x, ozk::DIGIT_SHIFT - e));
      Ni[u] = __double2ll_rn(scalbn(a.y, ozk::DIGIT_SHIFT - e));
    }
    const int off = ozk::tile_off(r, k0);
#pragma unroll 1
    for (int t = ozk::S - 1; t >= 0; --t) {
      uint32_t pr[4], pi[4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const int v0 = ozk::next_digit(Nr[u], t), v1 = ozk::next_digit(Nr[u + 1], t);
        const int v2 = ozk::next_digit(Ni[u], t), v3 = ozk::next_digit(Ni[u + 1], t);
        pr[u / 2] = (uint32_t)ozk::bf16_of_int(v0) | ((uint32_t)ozk::bf16_of_int(v1) << 16);
        pi[u / 2] = (uint32_t)ozk::bf16_of_int(v2) | ((uint32_t)ozk::bf16_of_int(v3) << 16);
      }
      unsigned char* stage = base + (size_t)t * ozk::A_STAGE;
      *reinterpret_cast<uint4*>(stage + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(stage + ozk::A_TILE + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

struct ResidualSmem {
  ozk::Smem st;
  ozk::Bars bars;
  ProblemDev P;
  double2 fz[PMCIM_MAX_TERMS];
  int g[PMCIM_MAX_TERMS * ozk::LC];
  double red[THREADS];
  uint32_t tmem;
};

struct ResidualArgs {
  const ProblemDev* prob;
  const double2* z;
  int m;
  const double2* X;
  double2* R;
  unsigned char* ysl;
  size_t ysl_stride;
  int32_t* status;
  long long wait_cycles;
};

// One point per CTA at a time: R_j = V - T(z_j) X_j.
__global__ void __launch_bounds__(THREADS, 1) k_residual_points(ResidualArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  ResidualSmem& sm = *reinterpret_cast<ResidualSmem*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid < 32) tcu::tmem_alloc_cols(&sm.tmem, ozk::TMEM_COLS);
  if (tid == 0) ozk::init_bars(sm.bars);
  load_problem(&sm.P, a.prob);
  tcu::fence_async_smem();
  tcu::fence_before();
  __syncthreads();
  tcu::fence_after();
  const size_t nl = (size_t)sm.P.n * sm.P.l;
  unsigned char* ysl = a.ysl + (size_t)blockIdx.x * a.ysl_stride;
  for (int j = blockIdx.x; j < a.m; j += gridDim.x) {
    if (tid < sm.P.K) sm.fz[tid] = eval_f(sm.P.term[tid], a.z[j]);
    __syncthreads();
    const bool ok = ozk::residual(sm.P, sm.fz, a.X + (size_t)j * nl, a.R + (size_t)j * nl, sm.st, sm.bars, ysl,
                                  sm.tmem, sm.g, sm.red, a.wait_cycles);
    if (tid == 0) a.status[j] = ok ? 0 : 1;
    __syncthreads();
  }
  tcu::fence_before();
  __syncthreads();
  tcu::fence_after();
  if (tid < 32) tcu::tmem_dealloc_cols(sm.tmem, ozk::TMEM_COLS);
}

}  // namespace

size_t coefficient_digit_bytes(int n, int n_dense) { return ozk::coeff_digit_bytes(n, n_dense); }
size_t y_digit_scratch_bytes(int n, int n_dense) { return n > 0 ? ozk::y_digit_bytes(n, n_dense) : 0; }

cudaError_t make_coefficient_digits(const double2* A, int n, int n_dense, int32_t* exps, unsigned char* dig,
                                    cudaStream_t s) {
  if (n_dense <= 0) return cudaSuccess;
  const int RB = ozk::row_blocks(n), KCN = ozk::k_chunks(n), npad = RB * ozk::TM;
  k_coeff_exponents<<<dim3((npad + 127) / 128, n_dense), 128, 0, s>>>(A, n, npad, exps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_coeff_digits<<<dim3(KCN, RB, n_dense), 256, 0, s>>>(A, n, RB, KCN, exps, dig);
  return cudaGetLastError();
}

cudaError_t launch_residual_points(const ProblemDev* prob, const double2* z, int m, const double2* X, double2* R,
                                   unsigned char* ysl, size_t ysl_stride, int ctas, int32_t* status,
                                   long long wait_cycles, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int smem = (int)sizeof(ResidualSmem) + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_residual_points, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  ResidualArgs a{prob, z, m, X, R, ysl, ysl_stride, status, wait_cycles};
  k_residual_points<<<ctas < m ? ctas : m, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}
