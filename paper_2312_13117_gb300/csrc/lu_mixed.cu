// Precision form of the node solves: FP32 LU with FP64 iterative refinement.
//
// The method's cost is the linear solve at every quadrature node (Eq. 2.4;
// Sec. 2.1 cost remark). On GB300 the FP32 pipe issues 64 times as many FMAs
// per clock as the FP64 pipe, so the O(n^3) factorisation runs in FP32 and
// FP64 is kept for what needs it: the residual R = V - T(z_j) X, formed from
// the FP64 coefficients A_k, and the accumulated solution X.
//
// Per node:
//   1. assemble T(z_j) in FP64 and round to complex64, append V;
//   2. FP32 blocked LU with partial pivoting (also eliminates V), back
//      substitution -> X_0 (promoted to FP64);
//   3. sweeps s = 1..max: R = V - T(z_j) X in FP64; delta = LU^-1 (R / |R|max)
//      in FP32, scaled back; X += delta. Stop when the estimated remaining
//      error |delta_s|^2 / |delta_{s-1}| (|delta_0| = |X_0|) is below
//      tol_ir |X| (max norms);
//   4. no convergence within max sweeps (or growth) -> the node is solved
//      again by the FP64 LU in the same workspace and flagged.
// Steps 1-2 are FP32 (or tensor-core) work, step 3 is FP64 work. One
// persistent CTA per SM runs them in two warp-specialised groups of 256
// threads: the factor group (warps 0-7) does steps 1-2 for node k+1 while the
// refine group (warps 8-15) does steps 3-4 for node k, so the FP64 pipe and
// the FP32 / tensor pipes of the SM work at the same time. Nodes pass between
// the groups through three workspace slots per CTA (the factor group can run up
// to two nodes ahead), each guarded by a pair of mbarriers (full: factor ->
// refine, empty: refine -> factor); every wait on them is bounded and a wait
// that runs out ends both groups with an error. The trailing updates of step 2
// run on the FMA pipes, or, for regions marked lu_tc, as complex products on the
// tensor cores: 3xTF32 (tc_update.cuh) or BF16 3M (tc_update_bf16.cuh).
// node_info: bits 0-23 = 0 or 1 + first zero-pivot column, bits 24-28 = sweeps
// run, bit 29 = a tensor-core wait ran out, bit 30 = FP64 fallback.
#include "ozaki.cuh"
#include "tc_update_bf16.cuh"

namespace {

using namespace lucore;

// Residual tiles: 128 rows x 16 columns per pass, depth 16; thread (tx, ty) owns
// rows tx + 64 i (i < 2) and columns ty + 4 q (q < 4) of the tile. The FP64
// pipe issues so slowly that shared-memory traffic is no constraint here; the
// small register block leaves room for the rest of the refinement loop.
constexpr int RT_ROWS = 128;
constexpr int RT_COLS = 16;
constexpr int RT_K = 16;
constexpr int RT_RI = RT_ROWS / 64;  // rows per thread
static_assert(RT_K * RT_COLS == THREADS, "one X-slice element per thread");
static_assert((RT_K * RT_ROWS) % THREADS == 0 && THREADS % RT_ROWS == 0, "tile copy mapping");

struct ResSmem {
  double2 As[2][RT_K * RT_ROWS];  // A_k tiles [kk][row], double-buffered
  double2 Xs[RT_K * RT_COLS];     // f_k X tile [kk][col]
};

__device__ __forceinline__ void cp_async_16(void* dst, const void* src, bool ok) {
  // 16 bytes global -> shared; zero-filled (nothing read) when !ok
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most the most recent group is still in flight
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Issue the copies of A_k rows r0.., columns k0..k0+RT_K-1 into dst [kk][row];
// thread (pr, pk) copies rows pr of columns pk + (THREADS / RT_ROWS) u. Out of
// range elements are zero-filled from a valid address.
__device__ __forceinline__ void res_tile_async(double2* dst, const double2* __restrict__ Ak, int n, int r0, int k0,
                                               int pr, int pk) {
#pragma unroll
  for (int u = 0; u < RT_K * RT_ROWS / THREADS; ++u) {
    const int kk = pk + (THREADS / RT_ROWS) * u;
    const bool ok = r0 + pr < n && k0 + kk < n;
    cp_async_16(dst + kk * RT_ROWS + pr, ok ? Ak + (size_t)(k0 + kk) * n + r0 + pr : Ak, ok);
  }
}

constexpr int GROUPS = 2;                        // factor group, refine group
constexpr int CTA_THREADS = GROUPS * THREADS;
constexpr int SLOTS = 3;                         // node slots per CTA

// A group's node context.
struct NodeCtx {
  ProblemDev P;
  double2 fz[PMCIM_MAX_TERMS];
  float2 fz32[PMCIM_MAX_TERMS];  // f_k(z) rounded to complex64
  float2 fid32;                  // sum over identity terms of f_k(z) id_k, complex64
  double red[THREADS / 32];
  int item;
};

struct FactorSmem {
  union {
    LuSmemT<float2> lu32;
    // lu32 followed by the tensor-core operand stage, which starts at lu32.Ls
    unsigned char tc[offsetof(LuSmemT<float2>, Ls) + tcu::STAGE_BYTES];
  } u;
  NodeCtx c;
};

struct RefineSmem {
  union {
    LuSmemT<float2> lu32;   // correction solves
    LuSmemT<double2> lu64;  // FP64 fallback
    ResSmem res;            // residual tiles (FP64 pipe)
    ozk::Smem oz;           // residual operand stages (tensor cores)
  } u;
  NodeCtx c;
  int ozg[PMCIM_MAX_TERMS * ozk::LC];  // column exponents of the digits of f_k X
  double ozred[THREADS];
};

// What the factor group hands over with a slot.
struct Slot {
  int item;        // node item, or -1: no more nodes
  int info;        // 0, or 1 + first zero-pivot column of the FP32 LU
  int tc_timeout;  // a tensor-core wait ran out during the LU
};

struct MixedSmem {
  FactorSmem f;
  RefineSmem r;
  Slot slot[SLOTS];
  uint64_t full[SLOTS];   // THREADS arrivals of the factor group
  uint64_t empty[SLOTS];  // THREADS arrivals of the refine group
  uint64_t mbar_tc[2];    // tensor-core completion, one per accumulator
  ozk::Bars ozb;          // the refine group's tensor-core residual: stage rings, drains
  uint32_t tmem_base;     // TMEM_ALL columns: the factor group's from 0, the refine group's from 256
  int tc_bad;             // a tensor-core wait ran out: FMA pipes from then on
};

__device__ __forceinline__ void mbar_init_count(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tcu::smem_u32(bar)), "r"(count) : "memory");
}

// Arrival with release semantics: this thread's earlier writes (shared and
// global) are visible to a thread whose wait on the phase succeeds.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(tcu::smem_u32(bar))
               : "memory");
}

// Phase clock: the group's thread 0 adds the cycles since the last mark to counter p.
struct PhaseClock {
  unsigned long long* c;
  long long t;
  __device__ explicit PhaseClock(unsigned long long* base) : c(base), t(0) { t = (long long)clock64(); }
  __device__ void mark(int p) {
    if (c && gtid() == 0) {
      const long long u = (long long)clock64();
      c[p] += (unsigned long long)(u - t);
      t = u;
    }
  }
};

// Phase-clock slots. Factor group: assemble, LU panels / TRSM / updates, first
// solve, set-up, waiting for a free slot; refine group: residual, correction
// solves, fallback, waiting for a factored node.
enum { PH_ASSEMBLE = 0, PH_PANEL = 1, PH_FIRST_SOLVE = 2, PH_RESIDUAL = 3, PH_CORRECTION = 4, PH_FALLBACK = 5,
       PH_SETUP = 6, PH_TRSM = 7, PH_UPDATE = 8, PH_FACTOR_WAIT = 9, PH_REFINE_WAIT = 10,
       PH_CTA_WALL_NS = 11,  // ns of CTA lifetime, not cycles
       PH_SWAPS = 12 };      // the panel's row interchanges on the columns outside it
static_assert(PH_SWAPS < PMCIM_PHASES, "phase slots");

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The FP32 blocked LU of lucore::cta_lu, with the trailing updates on the
// tensor cores (use_tc, while no wait has run out) or on the FMA pipes.
// Factor group only: its warps 0-7 are the TMEM lane owners.
// tc: 0 = trailing updates on the FMA pipes, 1 = 3xTF32 on the tensor cores, 2 = BF16 3M on the tensor cores
__device__ int cta_lu32(float2* __restrict__ M, int n, int ncols, int* __restrict__ piv, int* __restrict__ lists,
                        LuSmemT<float2>& sm, tcu::Ctx& cx, int tc, PhaseClock& pc) {
  if (gtid() == 0) sm.info_sh = 0;
  gsync();
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    const int kend = k0 + kb;
    // the panel in shared-memory sub-panels, in the tensor-core stage (idle during the
    // panel), while one sub-panel column fits there; else in global memory
    constexpr int kScratch = tcu::STAGE_BYTES / (int)sizeof(float2);
    // row interchanges in LINPACK's order (none on the L columns left of the panel);
    // each panel's permutation goes to lists for the forward solves
    int* list = lists + (size_t)(k0 / NB) * SWAP_LIST_INTS;
    if (n - k0 + NB * 8 + 40 <= kScratch) {
      const int sb = cta_lu_panel_sub(M, n, ncols, k0, kb, piv, sm, reinterpret_cast<float2*>(cx.stage), kScratch);
      pc.mark(PH_PANEL);
      cta_panel_swaps_lp(M, n, ncols, k0, kb, piv, sb, list, cx.stage, tcu::STAGE_BYTES);
      pc.mark(PH_SWAPS);
    } else {
      cta_lu_panel(M, n, ncols, k0, kb, piv, sm, k0);
      if (gtid() == 0) compose_swaps(piv, k0, kend, list);
      gsync();
      pc.mark(PH_PANEL);
    }
    if (kend >= ncols) continue;
    cta_lu_trsm(M, n, ncols, k0, kb, sm);
    pc.mark(PH_TRSM);
    if (kend >= n) continue;
    if (tc == 2 && !*cx.bad) tcb::update(M, n, ncols, k0, kb, cx);
    else if (tc == 1 && !*cx.bad) tcu::update(M, n, ncols, k0, kb, cx);
    else cta_lu_update_simt(M, n, ncols, k0, kb, sm);
    pc.mark(PH_UPDATE);
  }
  gsync();
  return sm.info_sh;
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  gsync();
  if ((gtid() & 31) == 0) red[gtid() >> 5] = v;
  gsync();
  double t = 0.0;
  for (int k = 0; k < THREADS / 32; ++k) t = fmax(t, red[k]);
  return t;
}

// R = V - sum_k f_k(z) A_k X  (FP64), R and X column-major n x l.
// R = V - id X - f_M M X in FP64 (the refinement residual), M an n x n column-major
// matrix (NULL: none). With two or more dense terms M is T(z_j) itself, assembled
// in FP64 once per node by the factor group (f_M = 1, id = 0), so that a sweep
// multiplies X by one matrix instead of one per term; with a single dense term M
// is that term's A_k.
__device__ void residual_fp64(const double2* __restrict__ X, double2* __restrict__ R, const NodeCtx& cx,
                              ResSmem& rs, const double2* __restrict__ M, double2 fM, double2 id) {
  const ProblemDev& P = cx.P;
  const int n = P.n, l = P.l;
  const int tid = gtid();
  const int tx = tid & 63, ty = tid >> 6;
  const int pr = tid % RT_ROWS, pk = tid / RT_ROWS;  // tile element (row, k) this thread fetches first
  const int xk = tid % RT_K, xc = tid / RT_K;        // X slice element (k, column)
  for (int c0 = 0; c0 < l; c0 += RT_COLS) {
    for (int r0 = 0; r0 < n; r0 += RT_ROWS) {
      double2 acc[RT_RI][4];
#pragma unroll
      for (int i = 0; i < RT_RI; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + tx + 64 * i, c = c0 + ty + 4 * q;
          double2 v = make_double2(0.0, 0.0);
          if (row < n && c < l) {
            v = P.V[(size_t)c * n + row];
            cfms(v, id, X[(size_t)c * n + row]);
          }
          acc[i][q] = v;
        }
      if (M) {
        // tiles of M stream through two shared buffers with cp.async: the copy
        // of the next tile is in flight while the current one is multiplied
        const double2* xcol = X + (size_t)(c0 + xc) * n;
        const bool xc_ok = c0 + xc < l;
        double2 px = (xk < n && xc_ok) ? xcol[xk] : make_double2(0.0, 0.0);
        gsync();  // both buffers are free
        res_tile_async(rs.As[0], M, n, r0, 0, pr, pk);
        cp_async_commit();
        int b = 0;
        for (int k0 = 0; k0 < n; k0 += RT_K, b ^= 1) {
          gsync();  // the previous step's multiplications are done
          rs.Xs[xk * RT_COLS + xc] = cmul(fM, px);
          if (k0 + RT_K < n) {
            res_tile_async(rs.As[b ^ 1], M, n, r0, k0 + RT_K, pr, pk);
            px = (k0 + RT_K + xk < n && xc_ok) ? xcol[k0 + RT_K + xk] : make_double2(0.0, 0.0);
          }
          cp_async_commit();
          cp_async_wait_prior();  // this tile's copies have landed (the next may be in flight)
          gsync();
          const double2* As = rs.As[b];
#pragma unroll 4
          for (int kk = 0; kk < RT_K; ++kk) {
            double2 av[RT_RI], xv[4];
#pragma unroll
            for (int i = 0; i < RT_RI; ++i) av[i] = As[kk * RT_ROWS + tx + 64 * i];
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] = rs.Xs[kk * RT_COLS + ty + 4 * q];
#pragma unroll
            for (int i = 0; i < RT_RI; ++i)
#pragma unroll
              for (int q = 0; q < 4; ++q) cfms(acc[i][q], av[i], xv[q]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RT_RI; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + tx + 64 * i, c = c0 + ty + 4 * q;
          if (row < n && c < l) R[(size_t)c * n + row] = acc[i][q];
        }
    }
  }
  cp_async_wait_all();
  gsync();
}

// The same for one column (l = 1), as a matrix-vector product: the tiled form
// above would multiply RT_COLS - 1 zero columns as well. Each thread owns four
// rows of a 4 x THREADS row block and streams the columns of M (coalesced over
// rows, several columns in flight); f_M x is staged in shared memory.
__device__ void residual_fp64_col(const double2* __restrict__ X, double2* __restrict__ R, const NodeCtx& cx,
                                  ResSmem& rs, const double2* __restrict__ M, double2 fM, double2 id) {
  const ProblemDev& P = cx.P;
  const int n = P.n;
  const int tid = gtid();
  constexpr int XCH = 2 * RT_K * RT_ROWS;  // f_M x entries per shared-memory chunk
  double2* xs = &rs.As[0][0];
  for (int r0 = 0; r0 < n; r0 += 4 * THREADS) {
    double2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = r0 + tid + i * THREADS;
      double2 v = make_double2(0.0, 0.0);
      if (row < n) {
        v = P.V[row];
        cfms(v, id, X[row]);
      }
      acc[i] = v;
    }
    if (M) {
      for (int c0 = 0; c0 < n; c0 += XCH) {
        const int cn = min(XCH, n - c0);
        gsync();  // the previous chunk is no longer read
        for (int e = tid; e < cn; e += THREADS) xs[e] = cmul(fM, X[c0 + e]);
        gsync();
#pragma unroll 4
        for (int c = 0; c < cn; ++c) {
          const double2 xv = xs[c];
          const double2* __restrict__ mc = M + (size_t)(c0 + c) * n;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int row = r0 + tid + i * THREADS;
            if (row < n) cfms(acc[i], mc[row], xv);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = r0 + tid + i * THREADS;
      if (row < n) R[row] = acc[i];
    }
  }
  gsync();
}

// T(z_j) in FP64 into T (n x n, column-major), the matrix of the refinement
// residuals, and rounded to complex64 into M32 (leading dimension n), the FP32
// LU's matrix: the dense terms in one pass over the elements, four elements per
// thread at a time so that their coefficient loads overlap, then a boundary-
// integral term (bie.cuh; a circulant one from its first column, formed in
// scratch, n values), then the identity terms on the diagonal. herm: T(z_j)^H
// instead (the coefficients read transposed, the sum conjugated; used by the
// certificates' bordered steps, which problems with a boundary-integral term do
// not take).
template <bool BIE>
__device__ void assemble_fp64(const NodeCtx& cx, double2* __restrict__ T, float2* __restrict__ M32, bool herm,
                              double2* __restrict__ scratch) {
  const ProblemDev& P = cx.P;
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  double2 id = make_double2(0.0, 0.0);
  for (int k = 0; k < P.K; ++k)
    if (!P.term[k].dense && P.term[k].kind != PMCIM_F_HELMHOLTZ_DLP) id = cadd(id, cmul(cx.fz[k], P.term[k].id));
  for (size_t e0 = gtid(); e0 < nn; e0 += 4 * (size_t)THREADS) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = make_double2(0.0, 0.0);
    for (int k = 0; k < P.K; ++k) {
      const TermDesc& t = P.term[k];
      if (!t.dense) continue;
      const double2* __restrict__ A = P.A + (size_t)t.mat_index * nn;
      double2 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t e = e0 + (size_t)u * THREADS;
        const size_t src = herm ? (e % n) * n + e / n : e;
        a[u] = e < nn ? A[src] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) cfma(v[u], cx.fz[k], a[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t e = e0 + (size_t)u * THREADS;
      if (e < nn) {
        if (herm) v[u].y = -v[u].y;
        T[e] = v[u];
        M32[e] = make_float2((float)v[u].x, (float)v[u].y);
      }
    }
  }
  gsync();
  if (BIE && P.bie && !herm) {
    int kb = 0;
    while (kb + 1 < P.K && P.term[kb].kind != PMCIM_F_HELMHOLTZ_DLP) ++kb;
    const double2 cb = P.term[kb].id, zb = cx.fz[kb];
    if (P.bie_circ) {
      for (int m = gtid(); m < n; m += THREADS) scratch[m] = bie::dlp_entry(P.bie, n, m, 0, zb);
      gsync();
    }
    for (int col = 0; col < n; ++col)
      for (int row = gtid(); row < n; row += THREADS) {
        const size_t e = (size_t)col * n + row;
        const double2 kv = P.bie_circ ? scratch[row >= col ? row - col : row - col + n]
                                      : bie::dlp_entry(P.bie, n, row, col, zb);
        double2 t = T[e];
        cfma(t, cb, kv);
        T[e] = t;
        M32[e] = make_float2((float)t.x, (float)t.y);
      }
    gsync();
  }
  if (herm) id.y = -id.y;
  for (int i = gtid(); i < n; i += THREADS) {
    const size_t e = (size_t)i * n + i;
    const double2 t = cadd(T[e], id);
    T[e] = t;
    M32[e] = make_float2((float)t.x, (float)t.y);
  }
  gsync();
}

// T(z_j) for the FP32 LU: FP32 arithmetic on the complex64 copy of the A_k
// (the LU only has to approximate T(z_j) to FP32 accuracy; the refinement
// residuals use the FP64 coefficients). It keeps the factor group off the FP64
// pipe. The flattened element index with eight elements per thread in flight
// keeps the loads of each term overlapped; the identity terms are added to the
// diagonal afterwards (a test per element would cost a 64-bit division).
__device__ void assemble32(const NodeCtx& cx, float2* __restrict__ M32) {
  const ProblemDev& P = cx.P;
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  constexpr int U = 8;
  const float2 fid = cx.fid32;
  for (size_t e0 = gtid(); e0 < nn; e0 += (size_t)U * THREADS) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = make_float2(0.f, 0.f);
    for (int k = 0; k < P.K; ++k) {
      const TermDesc& t = P.term[k];
      if (!t.dense) continue;
      const float2* __restrict__ A = P.A32 + (size_t)t.mat_index * nn;
      float2 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const size_t e = e0 + (size_t)u * THREADS;
        a[u] = e < nn ? A[e] : make_float2(0.f, 0.f);
      }
      const float2 f = cx.fz32[k];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        v[u].x = fmaf(f.x, a[u].x, fmaf(-f.y, a[u].y, v[u].x));
        v[u].y = fmaf(f.x, a[u].y, fmaf(f.y, a[u].x, v[u].y));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t e = e0 + (size_t)u * THREADS;
      if (e < nn) M32[e] = v[u];
    }
  }
  if (fid.x != 0.f || fid.y != 0.f) {
    gsync();
    for (int i = gtid(); i < n; i += THREADS) {
      float2& d = M32[(size_t)i * n + i];
      d.x += fid.x;
      d.y += fid.y;
    }
  }
}

// T(z_j) into the FP32 matrix (rounded) or, for the fallback, the FP64 matrix.
__device__ void assemble(const NodeCtx& cx, float2* M32, double2* M64) {
  const ProblemDev& P = cx.P;
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  for (int col = 0; col < n; ++col) {
    for (int row = gtid(); row < n; row += THREADS) {
      const size_t e = (size_t)col * n + row;
      double2 v = make_double2(0.0, 0.0);
      for (int k = 0; k < P.K; ++k) {
        const TermDesc& t = P.term[k];
        if (t.dense) cfma(v, cx.fz[k], P.A[(size_t)t.mat_index * nn + e]);
        else if (row == col) cfma(v, cx.fz[k], t.id);
      }
      if (M32) M32[e] = make_float2((float)v.x, (float)v.y);
      else M64[e] = v;
    }
  }
}

// Node item -> problem, node point and weight in the group's context.
__device__ void load_node(const NodeArgs& a, int idx, NodeCtx& c, RegionDev& rg, NodeItem& it) {
  it = a.items[idx];
  rg = a.regions[it.region];
  {
    const int* src = reinterpret_cast<const int*>(a.probs + rg.prob);
    int* dst = reinterpret_cast<int*>(&c.P);
    for (int i = gtid(); i < (int)(sizeof(ProblemDev) / sizeof(int)); i += THREADS) dst[i] = src[i];
  }
  gsync();
  double2 z, w;
  node_weight(rg.cre, rg.cim, rg.r, rg.N, it.j, &z, &w);
  if (gtid() < c.P.K) {
    const double2 f = eval_f(c.P.term[gtid()], z);
    c.fz[gtid()] = f;
    c.fz32[gtid()] = make_float2((float)f.x, (float)f.y);
  }
  gsync();
  if (gtid() == 0) {
    double2 id = make_double2(0.0, 0.0);
    for (int k = 0; k < c.P.K; ++k)
      if (!c.P.term[k].dense && c.P.term[k].kind != PMCIM_F_HELMHOLTZ_DLP)
        id = cadd(id, cmul(c.fz[k], c.P.term[k].id));
    c.fid32 = make_float2((float)id.x, (float)id.y);
  }
  gsync();
}

// True in every thread of the group when v is true in every thread (a group barrier).
__device__ __forceinline__ bool group_all(bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)v), "r"(1 + (int)(threadIdx.x / THREADS)), "n"(THREADS)
      : "memory");
  return r != 0;
}

// Bounded wait of the whole group on a hand-off barrier; the group agrees on
// the outcome, so that it never splits at a timeout.
__device__ bool handoff_wait(uint64_t* bar, uint32_t parity, int32_t* err, long long limit) {
  const bool ok = group_all(tcu::wait_parity(bar, parity, limit));
  if (!ok && gtid() == 0) atomicExch(err, 1);
  return ok;
}

constexpr uint32_t TMEM_ALL = 512;
constexpr uint32_t TMEM_REFINE = 256;  // first column of the refine group's accumulators
static_assert(tcu::TMEM_COLS <= TMEM_REFINE && TMEM_REFINE + ozk::TMEM_COLS <= TMEM_ALL, "TMEM split");

// Steps 1-2 for one node after another, into the CTA's slots in turn.
// BIE: the instantiation for launches with a boundary-integral term (bie.cuh); the
// other leaves its code out.
template <bool BIE>
__device__ void factor_group(const NodeArgs& a, MixedSmem& sm, tcu::Ctx& cx, PhaseClock& pc) {
  const int tid = gtid();
  NodeCtx& c = sm.f.c;
  for (int k = 0;; ++k) {
    const int s = k % SLOTS, use = k / SLOTS;
    // the slot is free again once the refine group has finished its previous node
    if (use > 0 && !handoff_wait(&sm.empty[s], (uint32_t)((use - 1) & 1), a.err, a.handoff_wait_cycles)) return;
    pc.mark(PH_FACTOR_WAIT);
    if (tid == 0) c.item = atomicAdd(a.counter, 1);
    gsync();
    const int idx = c.item;
    Slot& sl = sm.slot[s];
    if (idx >= a.n_items) {
      if (tid == 0) sl.item = -1;
      mbar_arrive(&sm.full[s]);
      return;
    }
    const size_t si = (size_t)blockIdx.x * SLOTS + s;
    char* slot = a.work + si * a.slot_bytes;
    float2* M32 = reinterpret_cast<float2*>(slot);
    int* piv = a.piv + si * a.max_n;
    NodeItem it;
    RegionDev rg;
    load_node(a, idx, c, rg, it);
    const ProblemDev& P = c.P;
    const int n = P.n, l = P.l, ncols = n + l;
    const size_t nn = (size_t)n * n, nl = (size_t)n * l;
    pc.mark(PH_SETUP);
    // T(z_j) in FP64 for the refine group's FP64 residual, and rounded; T(z_j)^H likewise;
    // always with a boundary-integral term (no stored coefficients to take residuals from)
    if (rg.herm || (P.n_dense >= 2 && !a.oz) || (BIE && P.bie))
      assemble_fp64<BIE>(c, a.t64 + si * a.t64_stride, M32, rg.herm != 0,
                         reinterpret_cast<double2*>(slot + mixed_residual_offset(n, l)));
    else
      assemble32(c, M32);
    for (size_t e = tid; e < nl; e += THREADS) M32[nn + e] = make_float2((float)P.V[e].x, (float)P.V[e].y);
    gsync();
    if (rg.border > 0) {  // the bordered matrix of a certificate: column s of T(z_j) replaced
      const double2* bc = a.border + rg.v_off;
      float2* col = M32 + (size_t)(rg.border - 1) * n;
      for (int i = tid; i < n; i += THREADS) col[i] = make_float2((float)bc[i].x, (float)bc[i].y);
      gsync();
    }
    pc.mark(PH_ASSEMBLE);
    const int bad_before = sm.tc_bad;
    int* lists = reinterpret_cast<int*>(slot + mixed_lists_offset(n, l));
    const int info = cta_lu32(M32, n, ncols, piv, lists, sm.f.u.lu32, cx, rg.lu_tc, pc);
    if (tid == 0) {
      sl.item = idx;
      sl.info = info;
      sl.tc_timeout = sm.tc_bad != bad_before;
    }
    mbar_arrive(&sm.full[s]);
  }
}

// Step 4: the node solved again by the FP64 LU in its slot. Kept out of line:
// it is rare, and its registers should not weigh on the refinement loop.
__device__ __noinline__ int fallback_fp64(const NodeCtx& c, double2* M64, int* piv, double2* X,
                                          LuSmemT<double2>& lu, const double2* __restrict__ T64) {
  const ProblemDev& P = c.P;
  const int n = P.n, l = P.l;
  const size_t nn = (size_t)n * n, nl = (size_t)n * l;
  gsync();
  if (T64)  // T(z_j) as the factor group assembled it in FP64 (a boundary-integral term)
    for (size_t e = gtid(); e < nn; e += THREADS) M64[e] = T64[e];
  else
    assemble(c, nullptr, M64);
  for (size_t e = gtid(); e < nl; e += THREADS) M64[nn + e] = P.V[e];
  gsync();
  const int info = cta_lu(M64, n, n + l, piv, lu);
  cta_back_blocked(M64, n, l, lu);
  for (size_t e = gtid(); e < nl; e += THREADS) X[e] = M64[nn + e];
  gsync();
  return info;
}

// Steps 3-4 for the nodes the factor group hands over, in the same order.
template <bool BIE>
__device__ void refine_group(const NodeArgs& a, MixedSmem& sm, PhaseClock& pc) {
  const int tid = gtid();
  NodeCtx& c = sm.r.c;
  for (int k = 0;; ++k) {
    const int s = k % SLOTS, use = k / SLOTS;
    if (!handoff_wait(&sm.full[s], (uint32_t)(use & 1), a.err, a.handoff_wait_cycles)) return;
    pc.mark(PH_REFINE_WAIT);
    const Slot sl = sm.slot[s];
    if (sl.item < 0) return;
    const size_t si = (size_t)blockIdx.x * SLOTS + s;
    char* slot = a.work + si * a.slot_bytes;
    float2* M32 = reinterpret_cast<float2*>(slot);
    double2* M64 = reinterpret_cast<double2*>(slot);  // fallback only; aliases M32
    int* piv = a.piv + si * a.max_n;
    NodeItem it;
    RegionDev rg;
    load_node(a, sl.item, c, rg, it);
    const ProblemDev& P = c.P;
    const int n = P.n, l = P.l;
    const size_t nn = (size_t)n * n, nl = (size_t)n * l;
    double2* R = reinterpret_cast<double2*>(slot + mixed_residual_offset(n, l));
    const int* lists = reinterpret_cast<const int*>(slot + mixed_lists_offset(n, l));
    double2* X = a.X + rg.x_off + (size_t)it.j * nl;
    int info = sl.info;
    bool ok = (info == 0);
    // the first solve, X_0 = U^-1 (L^-1 P V) in FP32 (the factor group eliminated V
    // with the LU), here so that the factor group can start the next node
    double xm = 0.0;
    if (ok) {
      cta_back_blocked(M32, n, l, sm.r.u.lu32);
      for (size_t e = tid; e < nl; e += THREADS) {
        const float2 y = M32[nn + e];
        const double2 x = make_double2((double)y.x, (double)y.y);
        X[e] = x;
        xm = fmax(xm, fmax(fabs(x.x), fabs(x.y)));
      }
      xm = block_max(xm, c.red);
    }
    pc.mark(PH_FIRST_SOLVE);
    bool tc_lost = sl.tc_timeout != 0;
    int sweeps = 0;
    // residuals on the tensor cores (exact digit products), unless a wait of that
    // path ran out earlier in this CTA; then the node is solved in FP64 below
    const bool bie = BIE && P.bie;
    const bool use_oz = a.oz && P.Adig != nullptr && !rg.herm && !bie;
    if (use_oz && sm.ozb.bad) {
      ok = false;
      tc_lost = true;
    }
    // max_sweeps == 0: the FP32 solve alone (a direction for a certificate), no refinement
    // and no FP64 re-solve
    const bool refine = a.max_sweeps > 0;
    if (ok && refine) {
      // the matrix each residual multiplies: T(z_j) assembled once, or the one dense term
      const double2* M = nullptr;
      double2 fM = make_double2(0.0, 0.0), id = make_double2(0.0, 0.0);
      if (use_oz) {
        // every dense term through the digit products; nothing to set up here
      } else if (P.n_dense >= 2 || rg.herm || bie) {  // assembled by the factor group with the slot
        M = a.t64 + si * a.t64_stride;
        fM = make_double2(1.0, 0.0);
      } else {
        for (int k = 0; k < P.K; ++k) {
          const TermDesc& t = P.term[k];
          if (t.dense) {
            M = P.A + (size_t)t.mat_index * nn;
            fM = c.fz[k];
          } else {
            id = cadd(id, cmul(c.fz[k], t.id));
          }
        }
      }
      double dprev = xm;
      bool conv = false;
      for (int sw = 1; sw <= a.max_sweeps && ok; ++sw) {
        if (use_oz) {
          if (!ozk::residual(P, c.fz, X, R, sm.r.u.oz, sm.ozb, a.ysl + si * a.ysl_stride,
                             sm.tmem_base + TMEM_REFINE, sm.r.ozg, sm.r.ozred, a.tc_wait_cycles)) {
            ok = false;
            tc_lost = true;
            break;
          }
        } else {
          if (l == 1) residual_fp64_col(X, R, c, sm.r.u.res, M, fM, id);
          else residual_fp64(X, R, c, sm.r.u.res, M, fM, id);
        }
        if (rg.border > 0) {
          // bordered system M u = b, M = T(z_j) + (c - T(z_j) e_s) e_s^T with b = -T(z_j) e_s:
          // R = b - T X - (c + b) X_s (l = 1)
          const double2 xs = X[rg.border - 1];
          const double2* bc = a.border + rg.v_off;
          for (size_t e = tid; e < nl; e += THREADS) cfms(R[e], cadd(bc[e], P.V[e]), xs);
        }
        pc.mark(PH_RESIDUAL);
        double rm = 0.0;
        for (size_t e = tid; e < nl; e += THREADS) rm = fmax(rm, fmax(fabs(R[e].x), fabs(R[e].y)));
        rm = block_max(rm, c.red);
        if (rm == 0.0) {
          conv = true;
          break;
        }
        const double inv = 1.0 / rm;
        // right-hand side R / |R|max; the forward solve applies the row interchanges
        for (size_t e = tid; e < nl; e += THREADS) {
          const double2 rv = R[e];
          M32[nn + e] = make_float2((float)(rv.x * inv), (float)(rv.y * inv));
        }
        gsync();
        cta_fwd_blocked_lp(M32, n, l, sm.r.u.lu32, lists);
        cta_back_blocked(M32, n, l, sm.r.u.lu32);
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
        dm = block_max(dm, c.red);
        xmx = block_max(xmx, c.red);
        pc.mark(PH_CORRECTION);
        sweeps = sw;
        if (!(dm < dprev) && sw > 1) {  // no contraction
          ok = false;
          break;
        }
        if (dm * dm <= a.tol_ir * xmx * dprev) {
          conv = true;
          break;
        }
        dprev = dm;
      }
      if (!conv) ok = false;
    }
    if (!ok && refine && rg.border == 0) {
      info = fallback_fp64(c, M64, piv, X, sm.r.u.lu64, bie ? a.t64 + si * a.t64_stride : nullptr);
      pc.mark(PH_FALLBACK);
    }
    if (rg.border > 0) {
      // the certificate's vector y = e_s + (u - u_s e_s): T(z_j) y = -u_s c
      gsync();
      if (tid == 0) X[rg.border - 1] = make_double2(1.0, 0.0);
    }
    if (tid == 0)
      a.node_info[rg.node_off + it.j] =
          info | (sweeps << 24) | (tc_lost ? (1 << 29) : 0) | (ok ? 0 : (1 << 30));
    gsync();
    mbar_arrive(&sm.empty[s]);
  }
}

template <bool BIE>
__global__ void __launch_bounds__(CTA_THREADS, 1) k_factor_solve_mixed(NodeArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  MixedSmem& sm = *reinterpret_cast<MixedSmem*>(smem_raw);
  const int tid = threadIdx.x;
  PhaseClock pc(a.phase ? a.phase + (size_t)blockIdx.x * PMCIM_PHASES : nullptr);
  unsigned long long t_start = 0;
  if (a.phase && tid == 0) t_start = global_ns();

  // tensor memory (all of it: one CTA per SM) and the barriers, for the whole persistent CTA
  if (tid < 32) tcu::tmem_alloc_cols(&sm.tmem_base, TMEM_ALL);
  if (tid == 0) {
    ozk::init_bars(sm.ozb);
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init_count(&sm.full[s], THREADS);
      mbar_init_count(&sm.empty[s], THREADS);
    }
    tcu::mbar_init(&sm.mbar_tc[0]);
    tcu::mbar_init(&sm.mbar_tc[1]);
    sm.tc_bad = 0;
  }
  tcu::fence_async_smem();
  tcu::fence_before();
  __syncthreads();
  tcu::fence_after();

  if (tid < THREADS) {
    tcu::Ctx cx{sm.f.u.tc + offsetof(LuSmemT<float2>, Ls), sm.mbar_tc, sm.tmem_base, {0u, 0u}, &sm.tc_bad,
                a.tc_wait_cycles};
    factor_group<BIE>(a, sm, cx, pc);
    // a commit whose wait ran out may still be in flight: wait once more, with the
    // default limit whatever the update's own limit was, before the columns are given back
    if (sm.tc_bad) {
      // returns at once for a barrier with no commit outstanding
      tcu::wait_parity(&sm.mbar_tc[0], cx.phase[0] ^ 1u, tcu::WAIT_CYCLES);
      tcu::wait_parity(&sm.mbar_tc[1], cx.phase[1] ^ 1u, tcu::WAIT_CYCLES);
    }
  } else {
    refine_group<BIE>(a, sm, pc);
  }
  // both groups are done with tensor memory before it is given back
  tcu::fence_before();
  __syncthreads();
  tcu::fence_after();
  if (tid < 32) tcu::tmem_dealloc_cols(sm.tmem_base, TMEM_ALL);
  if (a.phase && tid == 0)  // the CTA's lifetime, for cycles per ns
    a.phase[(size_t)blockIdx.x * PMCIM_PHASES + PH_CTA_WALL_NS] += global_ns() - t_start;
}

}  // namespace

// Slot layout: [FP32 matrix n x (n + l)] [FP64 residual n x l] [the panels' row
// permutations, SWAP_LIST_INTS ints each], or, after a fallback, the FP64 matrix
// n x (n + l) over the whole slot.
size_t mixed_slot_bytes(int n, int l) {
  const size_t fp64 = (size_t)n * (n + l) * sizeof(double2);
  const size_t mixed = mixed_lists_offset(n, l) + (size_t)((n + NB - 1) / NB) * SWAP_LIST_INTS * sizeof(int);
  const size_t b = fp64 > mixed ? fp64 : mixed;
  return (b + 255) & ~(size_t)255;
}

static_assert(sizeof(MixedSmem) + 1024 <= 227 * 1024, "one CTA per SM");

cudaError_t prepare_factor_mixed() {
  cudaError_t e = cudaFuncSetAttribute(k_factor_solve_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(MixedSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_factor_solve_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(MixedSmem));
}

int mixed_slots_per_cta() { return SLOTS; }

namespace {
__global__ void k_round_c64(const double2* __restrict__ src, float2* __restrict__ dst, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}
}  // namespace

cudaError_t round_coefficients_c64(const double2* src, float2* dst, size_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const size_t blocks = (count + 255) / 256;
  k_round_c64<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

// Launch only; prepare_factor_mixed() must have set the shared-memory limit.
// One CTA per a.slots / SLOTS workspace slots.
cudaError_t launch_factor_solve_mixed(const NodeArgs& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  const size_t smem = sizeof(MixedSmem);
  int grid = a.slots / SLOTS;
  if (grid > a.n_items) grid = a.n_items;
  if (grid < 1) return cudaErrorInvalidValue;
  if (a.bie) k_factor_solve_mixed<true><<<grid, CTA_THREADS, smem, s>>>(a);
  else k_factor_solve_mixed<false><<<grid, CTA_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}
