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
#include "lu_core.cuh"

namespace {

using namespace lucore;

// ---------------------------------------------------------------------------
// Persistent kernel: node g -> X_g = T(z_g)^{-1} V.
// ---------------------------------------------------------------------------
// Shared memory of the node kernel: the LU tiles plus the node's problem.
struct NodeSmem {
  LuSmem lu;
  ProblemDev P;
  int item;
};

// RI: the trailing update's register block (4: 64 x 64 tiles; 2: 32 x 32 tiles).
template <int RI, bool BIE>
__global__ void __launch_bounds__(THREADS, 2) k_factor_solve_fp64(NodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeSmem& sm = *reinterpret_cast<NodeSmem*>(smem_raw);
  const int tid = threadIdx.x;
  double2* M = reinterpret_cast<double2*>(a.work + (size_t)blockIdx.x * a.slot_bytes);
  int* piv = a.piv + (size_t)blockIdx.x * a.max_n;

  for (;;) {
    // largest-first list, handed out by an atomic counter (no waiting on other CTAs)
    if (tid == 0) sm.item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int idx = sm.item;
    if (idx >= a.n_items) break;
    const NodeItem it = a.items[idx];
    const RegionDev rg = a.regions[it.region];
    load_problem(&sm.P, a.probs + rg.prob);
    __syncthreads();
    const ProblemDev& P = sm.P;
    const int n = P.n, l = P.l, ncols = n + l;
    double2 z, w;
    node_weight(rg.cre, rg.cim, rg.r, rg.N, it.j, &z, &w);
    if (tid < P.K) sm.lu.fz[tid] = eval_f(P.term[tid], z);
    __syncthreads();

    // assemble [T(z_j) | V]
    const size_t nn = (size_t)n * n;
    // a circulant boundary-integral term: its n distinct entries K_{m,0}, formed once per
    // node in the slot's probe-block columns (V is written there below)
    double2* circ = M + nn;
    const bool use_circ = BIE && P.bie_circ;
    if (use_circ) {
      for (int m = tid; m < n; m += THREADS) circ[m] = bie::dlp_entry(P.bie, n, m, 0, z);
      __syncthreads();
    }
    for (int col = 0; col < n; ++col) {
      for (int row = tid; row < n; row += THREADS) {
        const size_t e = (size_t)col * n + row;
        double2 v = make_double2(0.0, 0.0);
        for (int k = 0; k < P.K; ++k) {
          const TermDesc& t = P.term[k];
          if (t.dense) {
            cfma(v, sm.lu.fz[k], P.A[(size_t)t.mat_index * nn + e]);
          } else if (use_circ && t.kind == PMCIM_F_HELMHOLTZ_DLP) {
            const int m = row >= col ? row - col : row - col + n;
            cfma(v, t.id, circ[m]);
          } else {
            cfma_term<BIE>(v, P, t, sm.lu.fz[k], row, col);
          }
        }
        M[e] = v;
      }
    }
    if (use_circ) __syncthreads();  // circ is read above and overwritten by V below
    for (size_t e = tid; e < (size_t)n * l; e += THREADS) M[nn + e] = P.V[e];
    __syncthreads();

    const int info = cta_lu<double2, RI>(M, n, ncols, piv, sm.lu);
    cta_back_blocked(M, n, l, sm.lu);

    double2* Xo = a.X + rg.x_off + (size_t)it.j * n * l;
    for (size_t e = tid; e < (size_t)n * l; e += THREADS) Xo[e] = M[nn + e];
    if (tid == 0) a.node_info[rg.node_off + it.j] = info;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Verification: sigma_min(T(lambda)) by inverse iteration on (T^H T)^{-1}
// using the LU of T(lambda) (pmCIMb step 3).
// ---------------------------------------------------------------------------
struct VerifySmem {
  LuSmem lu;
  ProblemDev P;
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

template <bool BIE>
__global__ void __launch_bounds__(THREADS, 2) k_verify_fp64(ValueArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  VerifySmem& sm = *reinterpret_cast<VerifySmem*>(smem_raw);
  const int tid = threadIdx.x;
  double2* M = a.work + (size_t)blockIdx.x * a.max_n * a.max_n;
  int* piv = a.piv + (size_t)blockIdx.x * a.max_n;
  double2* x = a.vec + (size_t)blockIdx.x * 3 * a.max_n;

  for (int it = blockIdx.x; it < a.m; it += gridDim.x) {
    load_problem(&sm.P, a.probs + a.prob_of[it]);
    __syncthreads();
    const ProblemDev& P = sm.P;
    const int n = P.n;
    const size_t nn = (size_t)n * n;
    double2* wv = x + n;
    double2* yv = x + 2 * n;
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
          if (t.dense) cfma(v, sm.lu.fz[k], P.A[(size_t)t.mat_index * nn + e]);
          else cfma_term<BIE>(v, P, t, sm.lu.fz[k], row, col);
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
      a.sigma[it] = smin;
      double thr = a.tol_verify * fmax(1.0, fro / sqrt((double)n));
      a.accept[it] = (smin <= thr) ? 1 : 0;
    }
    if (a.vec_out)  // the inverse iteration's last unit vector (zero when the LU met an exact zero pivot)
      for (int i = tid; i < n; i += THREADS)
        a.vec_out[(size_t)it * a.max_n + i] = info == 0 ? x[i] : make_double2(0.0, 0.0);
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

cudaError_t prepare_factor_fp64() {
  const void* fns[4] = {(const void*)k_factor_solve_fp64<4, false>, (const void*)k_factor_solve_fp64<2, false>,
                        (const void*)k_factor_solve_fp64<4, true>, (const void*)k_factor_solve_fp64<2, true>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(NodeSmem));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Launch only; prepare_factor_fp64() must have set the shared-memory limit (it
// is not called here so that the launch can be captured into a graph).
cudaError_t launch_factor_solve_fp64(const NodeArgs& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  const size_t smem = sizeof(NodeSmem);
  int grid = a.slots < a.n_items ? a.slots : a.n_items;
  if (a.bie) {
    if (a.fp64_tile == 32) k_factor_solve_fp64<2, true><<<grid, THREADS, smem, s>>>(a);
    else k_factor_solve_fp64<4, true><<<grid, THREADS, smem, s>>>(a);
  } else {
    if (a.fp64_tile == 32) k_factor_solve_fp64<2, false><<<grid, THREADS, smem, s>>>(a);
    else k_factor_solve_fp64<4, false><<<grid, THREADS, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_verify_fp64(const ValueArgs& a, cudaStream_t s) {
  if (a.m <= 0) return cudaSuccess;
  const size_t smem = sizeof(VerifySmem);
  const void* fn = a.bie ? (const void*)k_verify_fp64<true> : (const void*)k_verify_fp64<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = a.slots < a.m ? a.slots : a.m;
  if (a.bie) k_verify_fp64<true><<<grid, THREADS, smem, s>>>(a);
  else k_verify_fp64<false><<<grid, THREADS, smem, s>>>(a);
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
    // the flattened element index keeps every thread busy for any n
    for (size_t e = tid; e < nn; e += THREADS) {
      const size_t row = e % n, col = e / n;
      double2 v = make_double2(0.0, 0.0);
      for (int k = 0; k < P.K; ++k) {
        const TermDesc& t = P.term[k];
        if (t.dense) cfma(v, sm.fz[k], a.A[(size_t)t.mat_index * nn + e]);
        else if (row == col) cfma(v, sm.fz[k], t.id);
      }
      M[e] = v;
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

  // The device address of the array, looked up on every call with the calling
  // thread's device current. The lookup allocates nothing; it is not cached,
  // because a context torn down and created again (cudaDeviceReset by the host
  // application) can place the array at a new address.
  void* base = nullptr;
  if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) return PMCIM_ECUDA;
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
