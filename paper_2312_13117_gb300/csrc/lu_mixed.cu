// Precision form of the node solves: FP32 LU with FP64 iterative refinement.
//
// The method's cost is the linear solve at every quadrature node (Eq. 2.4;
// Sec. 2.1 cost remark). On GB300 the FP32 pipe issues 64 times as many FMAs
// per clock as the FP64 pipe, so the O(n^3) factorisation runs in FP32 and
// FP64 is kept for what needs it: the residual R = V - T(z_j) X, formed from
// the FP64 coefficients A_k, and the accumulated solution X.
//
// Per node (one CTA, persistent grid):
//   1. assemble T(z_j) in FP64 and round to complex64, append V;
//   2. FP32 blocked LU with partial pivoting (also eliminates V), back
//      substitution -> X_0 (promoted to FP64);
//   3. sweeps s = 1..max: R = V - T(z_j) X in FP64; delta = LU^-1 (R / |R|max)
//      in FP32, scaled back; X += delta. Stop when the estimated remaining
//      error |delta_s|^2 / |delta_{s-1}| (|delta_0| = |X_0|) is below
//      tol_ir |X| (max norms);
//   4. no convergence within max sweeps (or growth) -> the node is solved
//      again by the FP64 LU in the same workspace and flagged.
// node_info: bits 0-23 = 0 or 1 + first zero-pivot column, bits 24-29 = sweeps
// run, bit 30 = FP64 fallback.
#include "lu_core.cuh"

namespace {

using namespace lucore;

// Residual tiles: 256 rows x 16 columns per pass, depth 16; thread (tx, ty) owns
// rows tx + 64 i and columns ty + 4 q (i, q < 4) of the tile: a 4 x 4 complex
// register block, the same shape as the LU's trailing update.
constexpr int RT_ROWS = 256;
constexpr int RT_COLS = 16;
constexpr int RT_K = 16;

struct ResSmem {
  double2 As[RT_K * RT_ROWS];   // A_k tile [kk][row]
  double2 Xs[RT_K * RT_COLS];   // f_k X tile [kk][col]
};

union MixedSmemU {
  LuSmemT<float2> lu32;
  LuSmemT<double2> lu64;
  ResSmem res;
};

struct MixedSmem {
  MixedSmemU u;
  ProblemDev P;
  double2 fz[PMCIM_MAX_TERMS];
  double red[THREADS / 32];
  int item;
};

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < THREADS / 32; ++k) t = fmax(t, red[k]);
  return t;
}

// R = V - sum_k f_k(z) A_k X  (FP64), R and X column-major n x l.
__device__ void residual_fp64(const double2* __restrict__ X, double2* __restrict__ R, MixedSmem& sm) {
  const ProblemDev& P = sm.P;
  const int n = P.n, l = P.l;
  const int tid = threadIdx.x;
  const size_t nn = (size_t)n * n;
  const int tx = tid & 63, ty = tid >> 6;
  ResSmem& rs = sm.u.res;
  double2 idsum = make_double2(0.0, 0.0);  // sum of identity-term coefficients f_k id_k
  for (int k = 0; k < P.K; ++k)
    if (!P.term[k].dense) idsum = cadd(idsum, cmul(sm.fz[k], P.term[k].id));
  for (int c0 = 0; c0 < l; c0 += RT_COLS) {
    for (int r0 = 0; r0 < n; r0 += RT_ROWS) {
      double2 acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + tx + 64 * i, c = c0 + ty + 4 * q;
          double2 v = make_double2(0.0, 0.0);
          if (row < n && c < l) {
            v = P.V[(size_t)c * n + row];
            cfms(v, idsum, X[(size_t)c * n + row]);
          }
          acc[i][q] = v;
        }
      for (int k = 0; k < P.K; ++k) {
        const TermDesc& t = P.term[k];
        if (!t.dense) continue;
        const double2* Ak = P.A + (size_t)t.mat_index * nn;
        const double2 fk = sm.fz[k];
        for (int k0 = 0; k0 < n; k0 += RT_K) {
          __syncthreads();
          for (int e = tid; e < RT_K * RT_ROWS; e += THREADS) {
            const int r = e % RT_ROWS, kk = e / RT_ROWS;
            double2 v = make_double2(0.0, 0.0);
            if (r0 + r < n && k0 + kk < n) v = Ak[(size_t)(k0 + kk) * n + r0 + r];
            rs.As[kk * RT_ROWS + r] = v;
          }
          {
            const int kk = tid % RT_K, c = tid / RT_K;  // 256 threads = 16 x 16
            double2 v = make_double2(0.0, 0.0);
            if (k0 + kk < n && c0 + c < l) v = cmul(fk, X[(size_t)(c0 + c) * n + k0 + kk]);
            rs.Xs[kk * RT_COLS + c] = v;
          }
          __syncthreads();
#pragma unroll 4
          for (int kk = 0; kk < RT_K; ++kk) {
            double2 av[4], xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = rs.As[kk * RT_ROWS + tx + 64 * i];
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] = rs.Xs[kk * RT_COLS + ty + 4 * q];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int q = 0; q < 4; ++q) cfms(acc[i][q], av[i], xv[q]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + tx + 64 * i, c = c0 + ty + 4 * q;
          if (row < n && c < l) R[(size_t)c * n + row] = acc[i][q];
        }
    }
  }
  __syncthreads();
}

// T(z_j) into the FP32 matrix (rounded) or, for the fallback, the FP64 matrix.
__device__ void assemble(MixedSmem& sm, float2* M32, double2* M64) {
  const ProblemDev& P = sm.P;
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  for (int col = 0; col < n; ++col) {
    for (int row = threadIdx.x; row < n; row += THREADS) {
      const size_t e = (size_t)col * n + row;
      double2 v = make_double2(0.0, 0.0);
      for (int k = 0; k < P.K; ++k) {
        const TermDesc& t = P.term[k];
        if (t.dense) cfma(v, sm.fz[k], P.A[(size_t)t.mat_index * nn + e]);
        else if (row == col) cfma(v, sm.fz[k], t.id);
      }
      if (M32) M32[e] = make_float2((float)v.x, (float)v.y);
      else M64[e] = v;
    }
  }
}

// Phase clock: thread 0 adds the cycles since the last mark to counter p.
struct PhaseClock {
  unsigned long long* c;
  long long t;
  __device__ explicit PhaseClock(unsigned long long* base) : c(base), t(0) { t = (long long)clock64(); }
  __device__ void mark(int p) {
    if (c && threadIdx.x == 0) {
      const long long u = (long long)clock64();
      c[p] += (unsigned long long)(u - t);
      t = u;
    }
  }
};

__global__ void __launch_bounds__(THREADS, 2) k_factor_solve_mixed(NodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MixedSmem& sm = *reinterpret_cast<MixedSmem*>(smem_raw);
  const int tid = threadIdx.x;
  char* slot = a.work + (size_t)blockIdx.x * a.slot_bytes;
  float2* M32 = reinterpret_cast<float2*>(slot);
  double2* M64 = reinterpret_cast<double2*>(slot);  // fallback only; aliases M32
  int* piv = a.piv + (size_t)blockIdx.x * a.max_n;
  PhaseClock pc(a.phase ? a.phase + (size_t)blockIdx.x * PMCIM_PHASES : nullptr);

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
    const size_t nn = (size_t)n * n, nl = (size_t)n * l;
    double2* R = reinterpret_cast<double2*>(slot + mixed_residual_offset(n, l));
    int* perm = reinterpret_cast<int*>(slot + mixed_residual_offset(n, l) + nl * sizeof(double2));
    double2 z, w;
    node_weight(rg.cre, rg.cim, rg.r, rg.N, it.j, &z, &w);
    if (tid < P.K) sm.fz[tid] = eval_f(P.term[tid], z);
    __syncthreads();
    double2* X = a.X + rg.x_off + (size_t)it.j * nl;
    pc.mark(6);

    // 1-2: FP32 factorisation and first solution
    assemble(sm, M32, nullptr);
    for (size_t e = tid; e < nl; e += THREADS) M32[nn + e] = make_float2((float)P.V[e].x, (float)P.V[e].y);
    __syncthreads();
    pc.mark(0);
    int info = cta_lu(M32, n, ncols, piv, sm.u.lu32);
    pc.mark(1);
    bool ok = (info == 0);
    int sweeps = 0;
    if (ok) {
      cta_back_blocked(M32, n, l, sm.u.lu32);
      cta_pivots_to_perm(piv, perm, n);
      double xm = 0.0;
      for (size_t e = tid; e < nl; e += THREADS) {
        const float2 y = M32[nn + e];
        const double2 x = make_double2((double)y.x, (double)y.y);
        X[e] = x;
        xm = fmax(xm, fmax(fabs(x.x), fabs(x.y)));
      }
      xm = block_max(xm, sm.red);
      pc.mark(2);
      double dprev = xm;
      bool conv = false;
      // 3: refinement
      for (int s = 1; s <= a.max_sweeps && ok; ++s) {
        residual_fp64(X, R, sm);
        pc.mark(3);
        double rm = 0.0;
        for (size_t e = tid; e < nl; e += THREADS) rm = fmax(rm, fmax(fabs(R[e].x), fabs(R[e].y)));
        rm = block_max(rm, sm.red);
        if (rm == 0.0) { conv = true; break; }
        const double inv = 1.0 / rm;
        // right-hand side P R / |R|max: the row swaps as one gather
        for (size_t e = tid; e < nl; e += THREADS) {
          const size_t c = e / n, i = e % n;
          const double2 rv = R[c * n + perm[i]];
          M32[nn + e] = make_float2((float)(rv.x * inv), (float)(rv.y * inv));
        }
        __syncthreads();
        cta_fwd_blocked(M32, n, l, sm.u.lu32);
        cta_back_blocked(M32, n, l, sm.u.lu32);
        double dm = 0.0, xmx = 0.0;
        for (size_t e = tid; e < nl; e += THREADS) {
          const float2 d = M32[nn + e];
          double2 x = X[e];
          const double dx = (double)d.x * rm, dy = (double)d.y * rm;
          x.x += dx;
          x.y += dy;
          X[e] = x;
          dm = fmax(dm, fmax(fabs(dx), fabs(dy)));
          xmx = fmax(xmx, fmax(fabs(x.x), fabs(x.y)));
        }
        dm = block_max(dm, sm.red);
        xmx = block_max(xmx, sm.red);
        pc.mark(4);
        sweeps = s;
        if (!(dm < dprev) && s > 1) { ok = false; break; }          // no contraction
        if (dm * dm <= a.tol_ir * xmx * dprev) { conv = true; break; }
        dprev = dm;
      }
      if (!conv) ok = false;
    }
    if (!ok) {
      // 4: FP64 fallback in the same workspace
      __syncthreads();
      assemble(sm, nullptr, M64);
      for (size_t e = tid; e < nl; e += THREADS) M64[nn + e] = P.V[e];
      __syncthreads();
      info = cta_lu(M64, n, ncols, piv, sm.u.lu64);
      cta_back_blocked(M64, n, l, sm.u.lu64);
      for (size_t e = tid; e < nl; e += THREADS) X[e] = M64[nn + e];
      pc.mark(5);
    }
    if (tid == 0) a.node_info[rg.node_off + it.j] = info | (sweeps << 24) | (ok ? 0 : (1 << 30));
    __syncthreads();
  }
}

}  // namespace

// Slot layout: [FP32 matrix n x (n + l)] [FP64 residual n x l] [row permutation n],
// or, after a fallback, the FP64 matrix n x (n + l) over the whole slot.
size_t mixed_slot_bytes(int n, int l) {
  const size_t fp64 = (size_t)n * (n + l) * sizeof(double2);
  const size_t mixed = mixed_residual_offset(n, l) + (size_t)n * l * sizeof(double2) + (size_t)n * sizeof(int);
  const size_t b = fp64 > mixed ? fp64 : mixed;
  return (b + 255) & ~(size_t)255;
}

cudaError_t prepare_factor_mixed() {
  return cudaFuncSetAttribute(k_factor_solve_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(MixedSmem));
}

// Launch only; prepare_factor_mixed() must have set the shared-memory limit.
cudaError_t launch_factor_solve_mixed(const NodeArgs& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  const size_t smem = sizeof(MixedSmem);
  int grid = a.slots < a.n_items ? a.slots : a.n_items;
  k_factor_solve_mixed<<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}
