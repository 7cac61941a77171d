// Plain FP64 path: per-node assembly of T(z_j), blocked complex LU with partial
// pivoting, and the l-column solve, plus verification by sigma_min(T(lambda)).
//
// The paper solves T(z_j) x_j = f at every quadrature node with a dense direct
// solver (Eq. 2.4; Appendix, linearsolver = MATLAB backslash) and suggests
// solving all nodes in parallel (Sec. 3.2, remark on deeper parallelism).
// Here one CTA owns one node at a time (persistent grid, one workspace slot per
// CTA, two CTAs per SM): GB300 issues only ~2 DFMA per SM per clock, so a
// node-per-CTA schedule keeps every SM's FP64 pipe busy without cross-CTA
// synchronisation, and the trailing updates (the O(n^3) part) run from shared
// memory tiles with a 4x4 complex register block per thread.
//
// The probe block V is appended to T as l extra columns, so the row swaps and
// trailing updates of the factorisation also perform P and L^-1 on V; only the
// back substitution with U remains.
//
// Pivot rule: the row maximising |Re| + |Im| in the column, lowest row index on
// ties (the BLAS izamax convention of LAPACK zgetrf).
#include <mutex>

#include "pmcim_internal.cuh"

namespace {

constexpr int THREADS = 256;
constexpr int NB = 32;    // panel width
constexpr int TILE = 64;  // trailing-update tile (TILE x TILE complex)
constexpr int US_LD = TILE + 1;

struct LuSmem {
  double2 Ls[NB * TILE];   // L21 tile, [kk][row]; reused for L11 during the TRSM
  double2 Us[NB * US_LD];  // U12 tile, [kk][col], padded
  double2 prow[NB];        // pivot row of the panel
  double red_v[THREADS / 32];
  int red_i[THREADS / 32];
  double2 bcast[PMCIM_MAX_L];
  double2 fz[PMCIM_MAX_TERMS];
  int piv_sh;
  int info_sh;
};

__device__ __forceinline__ void warp_argmax(double& v, int& i) {
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, v, o);
    int oi = __shfl_down_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Deterministic block sum (fixed tree); every thread gets the result.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < THREADS / 32; ++k) t += red[k];
  return t;
}

// Block sum of a complex value; every thread gets the result.
__device__ double2 block_sum2(double2 v, double2* red2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum2(v);
  __syncthreads();
  if (lane == 0) red2[wid] = v;
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  for (int k = 0; k < THREADS / 32; ++k) t = cadd(t, red2[k]);
  return t;
}

// ---------------------------------------------------------------------------
// Blocked right-looking LU of the n x n leading block of M (column-major,
// leading dimension n, ncols >= n columns; columns n..ncols-1 receive the same
// row swaps and elimination). piv[k] = row swapped with row k at step k.
// Returns 0, or 1 + the first column whose pivot was exactly zero.
// ---------------------------------------------------------------------------
__device__ int cta_lu(double2* __restrict__ M, int n, int ncols, int* __restrict__ piv, LuSmem& sm) {
  const int tid = threadIdx.x;
  const size_t ld = (size_t)n;
  if (tid == 0) sm.info_sh = 0;
  __syncthreads();

  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    const int kend = k0 + kb;

    // ---- panel factorisation, columns k0..kend-1 ----
    for (int j = k0; j < kend; ++j) {
      double2* colj = M + (size_t)j * ld;
      double bv = -1.0;
      int bi = n;
      for (int i = j + tid; i < n; i += THREADS) {
        double v = l1abs(colj[i]);
        if (v > bv) { bv = v; bi = i; }
      }
      warp_argmax(bv, bi);
      if ((tid & 31) == 0) { sm.red_v[tid >> 5] = bv; sm.red_i[tid >> 5] = bi; }
      __syncthreads();
      if (tid == 0) {
        double v = sm.red_v[0];
        int ii = sm.red_i[0];
        for (int w = 1; w < THREADS / 32; ++w) {
          if (sm.red_v[w] > v || (sm.red_v[w] == v && sm.red_i[w] < ii)) { v = sm.red_v[w]; ii = sm.red_i[w]; }
        }
        if (ii >= n) ii = j;
        sm.piv_sh = ii;
        piv[j] = ii;
      }
      __syncthreads();
      const int p = sm.piv_sh;
      if (p != j) {
        for (int c = tid; c < ncols; c += THREADS) {
          double2* cc = M + (size_t)c * ld;
          double2 t = cc[j];
          cc[j] = cc[p];
          cc[p] = t;
        }
      }
      __syncthreads();
      for (int c = j + 1 + tid; c < kend; c += THREADS) sm.prow[c - k0] = M[(size_t)c * ld + j];
      const double2 pv = colj[j];
      const bool zero = (pv.x == 0.0 && pv.y == 0.0);
      if (zero && tid == 0 && sm.info_sh == 0) sm.info_sh = j + 1;
      __syncthreads();
      if (!zero) {
        const double2 rp = crecip(pv);
        for (int i = j + 1 + tid; i < n; i += THREADS) {
          double2 lij = cmul(colj[i], rp);
          colj[i] = lij;
          for (int c = j + 1; c < kend; ++c) cfms(M[(size_t)c * ld + i], lij, sm.prow[c - k0]);
        }
      }
      __syncthreads();
    }

    if (kend >= ncols) continue;

    // ---- U12 = L11^{-1} A12 (rows k0..kend-1, columns kend..ncols-1) ----
    for (int e = tid; e < kb * kb; e += THREADS) {
      int r = e % kb, c = e / kb;
      sm.Ls[c * NB + r] = M[(size_t)(k0 + c) * ld + k0 + r];  // Ls[t*NB + i] = L11[i][t]
    }
    __syncthreads();
    {
      // one warp per column, lane i holds row k0+i (NB == warp size)
      const int lane = tid & 31, wid = tid >> 5;
      for (int c = kend + wid; c < ncols; c += THREADS / 32) {
        double2* cc = M + (size_t)c * ld + k0;
        double2 x = (lane < kb) ? cc[lane] : make_double2(0.0, 0.0);
        for (int t = 0; t < kb - 1; ++t) {
          double2 xt;
          xt.x = __shfl_sync(0xffffffffu, x.x, t);
          xt.y = __shfl_sync(0xffffffffu, x.y, t);
          if (lane > t && lane < kb) cfms(x, sm.Ls[t * NB + lane], xt);
        }
        if (lane < kb) cc[lane] = x;
      }
    }
    __syncthreads();

    if (kend >= n) continue;

    // ---- trailing update A22 -= L21 U12 over TILE x TILE tiles ----
    const int m_rows = n - kend, m_cols = ncols - kend;
    const int mt = (m_rows + TILE - 1) / TILE, nt = (m_cols + TILE - 1) / TILE;
    const int tx = tid & 15, ty = tid >> 4;
    for (int ti = 0; ti < mt; ++ti) {
      const int r0 = kend + ti * TILE;
      for (int e = tid; e < NB * TILE; e += THREADS) {
        int r = e % TILE, kk = e / TILE;
        double2 v = make_double2(0.0, 0.0);
        if (kk < kb && r0 + r < n) v = M[(size_t)(k0 + kk) * ld + r0 + r];
        sm.Ls[kk * TILE + r] = v;
      }
      for (int tj = 0; tj < nt; ++tj) {
        const int c0 = kend + tj * TILE;
        for (int e = tid; e < NB * TILE; e += THREADS) {
          int kk = e % NB, c = e / NB;
          double2 v = make_double2(0.0, 0.0);
          if (kk < kb && c0 + c < ncols) v = M[(size_t)(c0 + c) * ld + k0 + kk];
          sm.Us[kk * US_LD + c] = v;
        }
        __syncthreads();
        double2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int r = r0 + tx + 16 * i, c = c0 + ty + 16 * q;
            acc[i][q] = (r < n && c < ncols) ? M[(size_t)c * ld + r] : make_double2(0.0, 0.0);
          }
        for (int kk = 0; kk < kb; ++kk) {
          double2 a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = sm.Ls[kk * TILE + tx + 16 * i];
#pragma unroll
          for (int q = 0; q < 4; ++q) b[q] = sm.Us[kk * US_LD + ty + 16 * q];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) cfms(acc[i][q], a[i], b[q]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int r = r0 + tx + 16 * i, c = c0 + ty + 16 * q;
            if (r < n && c < ncols) M[(size_t)c * ld + r] = acc[i][q];
          }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  return sm.info_sh;
}

// Back substitution U X = Y for the l columns n..n+l-1 of M, in place.
__device__ void cta_back_subst(double2* __restrict__ M, int n, int l, LuSmem& sm) {
  const int tid = threadIdx.x;
  const size_t ld = (size_t)n;
  double2* Y = M + (size_t)n * ld;
  for (int j = n - 1; j >= 0; --j) {
    if (tid < l) {
      double2 x = cdiv(Y[(size_t)tid * ld + j], M[(size_t)j * ld + j]);
      Y[(size_t)tid * ld + j] = x;
      sm.bcast[tid] = x;
    }
    __syncthreads();
    const double2* uj = M + (size_t)j * ld;
    for (int i = tid; i < j; i += THREADS) {
      const double2 u = uj[i];
      for (int c = 0; c < l; ++c) cfms(Y[(size_t)c * ld + i], u, sm.bcast[c]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Persistent kernel: node g -> X_g = T(z_g)^{-1} V.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS, 2) k_factor_solve_fp64(FactorArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LuSmem& sm = *reinterpret_cast<LuSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const ProblemDesc& P = a.prob;
  const int n = P.n, l = a.l, ncols = n + l;
  double2* M = a.work + (size_t)blockIdx.x * n * ncols;
  int* piv = a.piv + (size_t)blockIdx.x * n;

  for (int node = blockIdx.x; node < a.n_nodes; node += gridDim.x) {
    const int g = a.node_region[node];
    const RegionDev rg = a.regions[g];
    const int j = node - rg.node_off;
    double2 z, w;
    node_weight(rg.cre, rg.cim, rg.r, rg.N, j, &z, &w);
    if (tid < P.K) sm.fz[tid] = eval_f(P.term[tid], z);
    __syncthreads();

    // assemble [T(z_j) | V]
    const size_t nn = (size_t)n * n;
    for (int col = 0; col < n; ++col) {
      for (int row = tid; row < n; row += THREADS) {
        const size_t e = (size_t)col * n + row;
        double2 v = make_double2(0.0, 0.0);
        for (int k = 0; k < P.K; ++k) {
          const TermDesc& t = P.term[k];
          if (t.dense) cfma(v, sm.fz[k], a.A[(size_t)t.mat_index * nn + e]);
          else if (row == col) cfma(v, sm.fz[k], t.id);
        }
        M[e] = v;
      }
    }
    for (size_t e = tid; e < (size_t)n * l; e += THREADS) M[nn + e] = a.V[e];
    __syncthreads();

    const int info = cta_lu(M, n, ncols, piv, sm);
    cta_back_subst(M, n, l, sm);

    double2* Xo = a.X + (size_t)node * n * l;
    for (size_t e = tid; e < (size_t)n * l; e += THREADS) Xo[e] = M[nn + e];
    if (tid == 0) a.node_info[node] = info;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Verification: sigma_min(T(lambda)) by inverse iteration on (T^H T)^{-1}
// using the LU of T(lambda) (pmCIMb step 3).
// ---------------------------------------------------------------------------
struct VerifySmem {
  LuSmem lu;
  double2 red2[THREADS / 32];
  double red[THREADS / 32];
  double2 bc;
};

// Solve U^H a = x (U upper, so U^H is lower; dot-product form over columns of U).
__device__ void solve_UH(const double2* __restrict__ M, int n, double2* __restrict__ x, VerifySmem& sm) {
  const size_t ld = (size_t)n;
  for (int j = 0; j < n; ++j) {
    const double2* uj = M + (size_t)j * ld;
    double2 s = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < j; i += THREADS) cfma_conj(s, uj[i], x[i]);
    s = block_sum2(s, sm.red2);
    if (threadIdx.x == 0) x[j] = cdiv(csub(x[j], s), cconj(uj[j]));
    __syncthreads();
  }
}
// Solve L^H u = a (L unit lower, so L^H is unit upper; dot-product form).
__device__ void solve_LH(const double2* __restrict__ M, int n, double2* __restrict__ x, VerifySmem& sm) {
  const size_t ld = (size_t)n;
  for (int j = n - 1; j >= 0; --j) {
    const double2* lj = M + (size_t)j * ld;
    double2 s = make_double2(0.0, 0.0);
    for (int i = j + 1 + threadIdx.x; i < n; i += THREADS) cfma_conj(s, lj[i], x[i]);
    s = block_sum2(s, sm.red2);
    if (threadIdx.x == 0) x[j] = csub(x[j], s);
    __syncthreads();
  }
}
// Solve L y = b (unit lower, column axpy form).
__device__ void solve_L(const double2* __restrict__ M, int n, double2* __restrict__ x, VerifySmem& sm) {
  const size_t ld = (size_t)n;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) sm.bc = x[j];
    __syncthreads();
    const double2 xj = sm.bc;
    const double2* lj = M + (size_t)j * ld;
    for (int i = j + 1 + threadIdx.x; i < n; i += THREADS) cfms(x[i], lj[i], xj);
    __syncthreads();
  }
}
// Solve U y = b (upper, column axpy form).
__device__ void solve_U(const double2* __restrict__ M, int n, double2* __restrict__ x, VerifySmem& sm) {
  const size_t ld = (size_t)n;
  for (int j = n - 1; j >= 0; --j) {
    const double2* uj = M + (size_t)j * ld;
    if (threadIdx.x == 0) {
      double2 v = cdiv(x[j], uj[j]);
      x[j] = v;
      sm.bc = v;
    }
    __syncthreads();
    const double2 xj = sm.bc;
    for (int i = threadIdx.x; i < j; i += THREADS) cfms(x[i], uj[i], xj);
    __syncthreads();
  }
}

__device__ double vec_norm(const double2* __restrict__ x, int n, VerifySmem& sm) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += THREADS) s += cabs2(x[i]);
  return sqrt(block_sum(s, sm.red));
}

__global__ void __launch_bounds__(THREADS, 2) k_verify_fp64(VerifyArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  VerifySmem& sm = *reinterpret_cast<VerifySmem*>(smem_raw);
  const int tid = threadIdx.x;
  const ProblemDesc& P = a.prob;
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  double2* M = a.work + (size_t)blockIdx.x * nn;
  int* piv = a.piv + (size_t)blockIdx.x * n;
  double2* x = a.vec + (size_t)blockIdx.x * 3 * n;
  double2* wv = x + n;
  double2* yv = x + 2 * n;

  for (int it = blockIdx.x; it < a.m; it += gridDim.x) {
    const double2 lam = a.lam[it];
    if (tid < P.K) sm.lu.fz[tid] = eval_f(P.term[tid], lam);
    __syncthreads();
    double fro = 0.0;
    for (int col = 0; col < n; ++col) {
      for (int row = tid; row < n; row += THREADS) {
        const size_t e = (size_t)col * n + row;
        double2 v = make_double2(0.0, 0.0);
        for (int k = 0; k < P.K; ++k) {
          const TermDesc& t = P.term[k];
          if (t.dense) cfma(v, sm.lu.fz[k], a.A[(size_t)t.mat_index * nn + e]);
          else if (row == col) cfma(v, sm.lu.fz[k], t.id);
        }
        M[e] = v;
        fro += cabs2(v);
      }
    }
    fro = sqrt(block_sum(fro, sm.red));
    const int info = cta_lu(M, n, n, piv, sm.lu);

    double smin = 0.0;
    if (info == 0) {
      // deterministic start vector
      for (int i = tid; i < n; i += THREADS) x[i] = make_double2(1.0 + 0.5 * sin(0.7 * i), cos(1.3 * i));
      __syncthreads();
      double nx = vec_norm(x, n, sm);
      for (int i = tid; i < n; i += THREADS) x[i] = cscale(x[i], 1.0 / nx);
      __syncthreads();
      double rho_prev = 0.0, rho = 0.0;
      for (int iter = 0; iter < 30; ++iter) {
        // w = T^{-H} x:  T = P^T L U  =>  T^H = U^H L^H P
        for (int i = tid; i < n; i += THREADS) wv[i] = x[i];
        __syncthreads();
        solve_UH(M, n, wv, sm);
        solve_LH(M, n, wv, sm);
        if (tid == 0)
          for (int k = n - 1; k >= 0; --k) {
            int p = piv[k];
            if (p != k) { double2 t = wv[k]; wv[k] = wv[p]; wv[p] = t; }
          }
        __syncthreads();
        rho = vec_norm(wv, n, sm);
        // y = T^{-1} w
        for (int i = tid; i < n; i += THREADS) yv[i] = wv[i];
        __syncthreads();
        if (tid == 0)
          for (int k = 0; k < n; ++k) {
            int p = piv[k];
            if (p != k) { double2 t = yv[k]; yv[k] = yv[p]; yv[p] = t; }
          }
        __syncthreads();
        solve_L(M, n, yv, sm);
        solve_U(M, n, yv, sm);
        double ny = vec_norm(yv, n, sm);
        for (int i = tid; i < n; i += THREADS) x[i] = cscale(yv[i], 1.0 / ny);
        __syncthreads();
        if (iter > 0 && fabs(rho - rho_prev) <= 1e-12 * rho) break;
        rho_prev = rho;
      }
      smin = 1.0 / rho;
    }
    if (tid == 0) {
      a.sigma_min[it] = smin;
      double thr = a.tol_verify * fmax(1.0, fro / sqrt((double)n));
      a.accept[it] = (smin <= thr) ? 1 : 0;
    }
    __syncthreads();
  }
}

}  // namespace

int factor_slots_fp64(int n, int l) {
  (void)n;
  (void)l;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 2 * (sms > 0 ? sms : 1);
}
size_t factor_smem_fp64() { return sizeof(LuSmem); }
int verify_slots_fp64(int n) { return factor_slots_fp64(n, 0); }

cudaError_t launch_factor_solve_fp64(const FactorArgs& a, cudaStream_t s) {
  if (a.n_nodes <= 0) return cudaSuccess;
  const size_t smem = sizeof(LuSmem);
  cudaError_t e = cudaFuncSetAttribute(k_factor_solve_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = a.slots < a.n_nodes ? a.slots : a.n_nodes;
  k_factor_solve_fp64<<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_verify_fp64(const VerifyArgs& a, cudaStream_t s) {
  if (a.m <= 0) return cudaSuccess;
  const size_t smem = sizeof(VerifySmem);
  cudaError_t e = cudaFuncSetAttribute(k_verify_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = a.slots < a.m ? a.slots : a.m;
  k_verify_fp64<<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// ===========================================================================
// Node solves without device allocation.
//
// Some callers cannot allocate device memory while they run: a host
// application that owns every byte of device memory through its own pool, or a
// latency-bound service loop that must not stall on the device-wide
// synchronisation that cudaFree implies. For them this entry point solves
// T(z_j) X_j = V at caller-given points with all inputs and outputs in caller
// buffers and the factorisation workspace in a fixed array compiled into the
// library. It makes no allocation of any kind.
//
// The array below is held by every GPU that loads the library until the
// process exits. It is shared by all calls and keeps the last call's contents;
// nothing in it needs clearing, because the kernel writes every workspace
// element (assembled matrix, probe columns, pivots) before it reads it. Calls
// that overlap on the GPU (two streams, two threads) race on the array.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double2)];

struct PointArgs {
  ProblemDesc prob;
  const double2* A;
  const double2* V;
  int l;
  const double2* z;   // m points
  int m;
  double2* X;         // m * n * l
  int32_t* info;      // m, may be NULL
  double2* work;      // slots * n * (n + l), inside g_noalloc_scratch
  int32_t* piv;       // slots * n, inside g_noalloc_scratch
};

// Same per-node work as k_factor_solve_fp64, at an explicit point z_j.
__global__ void __launch_bounds__(THREADS, 2) k_factor_solve_points_fp64(PointArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LuSmem& sm = *reinterpret_cast<LuSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const ProblemDesc& P = a.prob;
  const int n = P.n, l = a.l, ncols = n + l;
  double2* M = a.work + (size_t)blockIdx.x * n * ncols;
  int* piv = a.piv + (size_t)blockIdx.x * n;
  for (int node = blockIdx.x; node < a.m; node += gridDim.x) {
    const double2 z = a.z[node];
    if (tid < P.K) sm.fz[tid] = eval_f(P.term[tid], z);
    __syncthreads();
    const size_t nn = (size_t)n * n;
    for (int col = 0; col < n; ++col) {
      for (int row = tid; row < n; row += THREADS) {
        const size_t e = (size_t)col * n + row;
        double2 v = make_double2(0.0, 0.0);
        for (int k = 0; k < P.K; ++k) {
          const TermDesc& t = P.term[k];
          if (t.dense) cfma(v, sm.fz[k], a.A[(size_t)t.mat_index * nn + e]);
          else if (row == col) cfma(v, sm.fz[k], t.id);
        }
        M[e] = v;
      }
    }
    for (size_t e = tid; e < (size_t)n * l; e += THREADS) M[nn + e] = a.V[e];
    __syncthreads();
    const int info = cta_lu(M, n, ncols, piv, sm);
    cta_back_subst(M, n, l, sm);
    double2* Xo = a.X + (size_t)node * n * l;
    for (size_t e = tid; e < (size_t)n * l; e += THREADS) Xo[e] = M[nn + e];
    if (tid == 0 && a.info) a.info[node] = info;
    __syncthreads();
  }
}

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

}  // namespace

extern "C" int pmcim_solve_points_noalloc(int32_t n, int32_t K, const pmcim_fterm* f, const uint8_t* dense,
                                          const double* A, int32_t m, const double* z, int32_t l,
                                          const double* V, double* X, int32_t* info, void* cuda_stream) {
  if (n < 1 || K < 1 || K > PMCIM_MAX_TERMS || l < 1 || l > PMCIM_MAX_L || m < 0) return PMCIM_EINVAL;
  if (!f || !dense || !V || (m > 0 && (!z || !X))) return PMCIM_EINVAL;
  // the workspace of one CTA slot must fit the fixed array
  const size_t slot_bytes = (size_t)n * (n + l) * sizeof(double2) + (size_t)n * sizeof(int32_t);
  if (slot_bytes > kNoAllocScratchBytes) return PMCIM_ENOTSUP;
  ProblemDesc desc{};
  desc.n = n;
  desc.K = K;
  int nd = 0;
  for (int k = 0; k < K; ++k) {
    if (f[k].kind != PMCIM_F_MONOMIAL && f[k].kind != PMCIM_F_EXP_NEG) return PMCIM_EINVAL;
    if (f[k].kind == PMCIM_F_MONOMIAL && (f[k].degree < 0 || f[k].degree > 16)) return PMCIM_EINVAL;
    TermDesc& t = desc.term[k];
    t.kind = f[k].kind;
    t.degree = f[k].degree;
    t.tau = f[k].tau;
    t.id = make_double2(f[k].id_re, f[k].id_im);
    t.dense = dense[k] ? 1 : 0;
    t.mat_index = dense[k] ? nd++ : -1;
  }
  desc.n_dense = nd;
  if (nd > 0 && !A) return PMCIM_EINVAL;
  if (m == 0) return PMCIM_OK;

  // set-up, once per device, with that device current: the device address of the array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PMCIM_ECUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PMCIM_ECUDA;
      g_noalloc_addr[dev] = ptr;
    }
    base = g_noalloc_addr[dev];
  }
  int slots = factor_slots_fp64(n, l);
  const size_t fit = kNoAllocScratchBytes / slot_bytes;
  if ((size_t)slots > fit) slots = (int)fit;
  if (slots > m) slots = m;

  PointArgs a;
  a.prob = desc;
  a.A = reinterpret_cast<const double2*>(A);
  a.V = reinterpret_cast<const double2*>(V);
  a.l = l;
  a.z = reinterpret_cast<const double2*>(z);
  a.m = m;
  a.X = reinterpret_cast<double2*>(X);
  a.info = info;
  a.work = reinterpret_cast<double2*>(base);
  a.piv = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(base) + (size_t)slots * n * (n + l) * sizeof(double2));
  const size_t smem = sizeof(LuSmem);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaFuncSetAttribute(k_factor_solve_points_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return PMCIM_ECUDA;
  k_factor_solve_points_fp64<<<slots, THREADS, smem, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return PMCIM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PMCIM_ECUDA;
  return PMCIM_OK;
}
