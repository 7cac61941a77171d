// Node solves for small problems (n <= 32, l <= 16): one warp per node.
//
// The same work as the CTA kernels (assembly of T(z_j), LU with partial
// pivoting on [T | V], back substitution), but a whole node lives in one
// warp's slice of shared memory with lane i owning row i, so every step is
// warp-synchronous: no block barriers, and an SM holds many nodes at once.
// Pivot rule as everywhere: largest |Re| + |Im| in the column, lowest row on
// ties.
#include "pmcim_internal.cuh"

namespace {

constexpr int WARPS = 4;
constexpr int SN = 32;            // largest n
constexpr int SL = 16;            // largest l
constexpr int LDC = SN + SL + 1;  // padded row length (complex entries)

struct SmallSmem {
  double2 M[WARPS][SN * LDC];
  ProblemDev P[WARPS];
  double2 fz[WARPS][PMCIM_MAX_TERMS];
};

template <bool BIE>
__global__ void __launch_bounds__(WARPS * 32) k_factor_solve_small(NodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSmem& sm = *reinterpret_cast<SmallSmem*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* M = sm.M[w];
  ProblemDev& P = sm.P[w];
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(a.counter, 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= a.n_items) break;
    const NodeItem it = a.items[idx];
    const RegionDev rg = a.regions[it.region];
    {
      const int* s = reinterpret_cast<const int*>(a.probs + rg.prob);
      int* d = reinterpret_cast<int*>(&P);
      for (int i = lane; i < (int)(sizeof(ProblemDev) / sizeof(int)); i += 32) d[i] = s[i];
    }
    __syncwarp();
    const int n = P.n, l = P.l, ncols = n + l;
    double2 z, wgt;
    node_weight(rg.cre, rg.cim, rg.r, rg.N, it.j, &z, &wgt);
    if (lane < P.K) sm.fz[w][lane] = eval_f(P.term[lane], z);
    __syncwarp();
    const size_t nn = (size_t)n * n;
    // assemble [T(z_j) | V] (T(z_j)^H for a certificate's step with rg.herm), row `lane`
    if (lane < n) {
      double2* row = M + lane * LDC;
      for (int c = 0; c < n; ++c) {
        double2 v = make_double2(0.0, 0.0);
        const size_t e = rg.herm ? (size_t)lane * n + c : (size_t)c * n + lane;
        for (int k = 0; k < P.K; ++k) {
          const TermDesc& t = P.term[k];
          if (t.dense) cfma(v, sm.fz[w][k], P.A[(size_t)t.mat_index * nn + e]);
          else if (BIE && t.kind == PMCIM_F_HELMHOLTZ_DLP)  // T^H: entry (c, lane), conjugated below
            cfma(v, t.id, bie::dlp_entry(P.bie, n, rg.herm ? c : lane, rg.herm ? lane : c, sm.fz[w][k]));
          else if (c == lane) cfma(v, sm.fz[w][k], t.id);
        }
        if (rg.herm) v.y = -v.y;
        row[c] = v;
      }
      for (int c = 0; c < l; ++c) row[n + c] = P.V[(size_t)c * n + lane];
    }
    __syncwarp();
    int info = 0;
    for (int j = 0; j < n; ++j) {
      double bv = -1.0;
      int bi = n;
      if (lane >= j && lane < n) {
        bv = l1abs(M[lane * LDC + j]);
        bi = lane;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      int p = __shfl_sync(0xffffffffu, bi, 0);
      if (p >= n) p = j;
      if (p != j)
        for (int c = lane; c < ncols; c += 32) {
          const double2 t = M[j * LDC + c];
          M[j * LDC + c] = M[p * LDC + c];
          M[p * LDC + c] = t;
        }
      __syncwarp();
      const double2 pv = M[j * LDC + j];
      if (pv.x == 0.0 && pv.y == 0.0) {
        if (info == 0) info = j + 1;
      } else if (lane > j && lane < n) {
        const double2 lij = cmul(M[lane * LDC + j], crecip(pv));
        M[lane * LDC + j] = lij;
        for (int c = j + 1; c < ncols; ++c) cfms(M[lane * LDC + c], lij, M[j * LDC + c]);
      }
      __syncwarp();
    }
    // back substitution U X = Y on the l right-hand columns
    for (int j = n - 1; j >= 0; --j) {
      if (lane < l) M[j * LDC + n + lane] = cdiv(M[j * LDC + n + lane], M[j * LDC + j]);
      __syncwarp();
      if (lane < j)
        for (int c = 0; c < l; ++c) cfms(M[lane * LDC + n + c], M[lane * LDC + j], M[j * LDC + n + c]);
      __syncwarp();
    }
    if (lane < n) {
      double2* Xo = a.X + rg.x_off + (size_t)it.j * n * l;
      for (int c = 0; c < l; ++c) Xo[(size_t)c * n + lane] = M[lane * LDC + n + c];
    }
    if (lane == 0) a.node_info[rg.node_off + it.j] = info;
    __syncwarp();
  }
}

}  // namespace

bool small_kernel_fits(int n, int l) { return n <= SN && l <= SL; }

cudaError_t prepare_factor_small() {
  cudaError_t e = cudaFuncSetAttribute(k_factor_solve_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(SmallSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_factor_solve_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SmallSmem));
}

// Launch only; prepare_factor_small() must have set the shared-memory limit.
cudaError_t launch_factor_solve_small(const NodeArgs& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = 2 * (sms > 0 ? sms : 1);
  const int need = (a.n_items + WARPS - 1) / WARPS;
  if (grid > need) grid = need;
  if (a.bie) k_factor_solve_small<true><<<grid, WARPS * 32, sizeof(SmallSmem), s>>>(a);
  else k_factor_solve_small<false><<<grid, WARPS * 32, sizeof(SmallSmem), s>>>(a);
  return cudaGetLastError();
}
