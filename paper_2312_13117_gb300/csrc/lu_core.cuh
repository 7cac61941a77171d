// CTA-level dense complex LU with partial pivoting and triangular solves,
// templated on the complex element type (double2 for FP64, float2 for FP32).
//
// Blocked right-looking factorisation of the n x n leading block of a
// column-major matrix with ncols >= n columns (extra columns receive the same
// row swaps and elimination, which performs P and L^-1 on appended right-hand
// sides). Panels of NB = 32 columns are factored column by column (pivot =
// row maximising |Re| + |Im|, lowest index on ties); U12 = L11^-1 A12 is solved
// one warp per column; the trailing update runs over 64 x 64 tiles staged in
// shared memory with a 4 x 4 complex register block per thread.
#pragma once

#include "pmcim_internal.cuh"

namespace lucore {

constexpr int THREADS = 256;

// Thread groups. Every routine below runs on one group of THREADS threads and
// synchronises only that group, through named barrier 1 + group: a CTA of
// THREADS threads is one group (the barrier then spans the whole CTA), and the
// precision-form kernel runs two groups side by side in one CTA.
__device__ __forceinline__ int gtid() { return (int)(threadIdx.x & (THREADS - 1)); }
__device__ __forceinline__ void gsync() {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / THREADS)), "n"(THREADS) : "memory");
}
// True in every thread of the group when v is true in every thread (a group barrier).
__device__ __forceinline__ bool group_all_sync(bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)v), "r"(1 + (int)(threadIdx.x / THREADS)), "n"(THREADS)
      : "memory");
  return r != 0;
}
constexpr int NB = 32;    // panel width
constexpr int TILE = 64;  // trailing-update tile (TILE x TILE complex)
constexpr int US_LD = TILE + 1;

template <typename T2>
struct LuSmemT {
  T2 prow[NB];             // pivot row of the panel
  double red_v[THREADS / 32];
  int red_i[THREADS / 32];
  T2 bcast[PMCIM_MAX_L];
  double2 fz[PMCIM_MAX_TERMS];
  int piv_sh;
  int info_sh;
  // the tile buffers come last: a tensor-core update may stage its operands
  // from here on, over the end of the struct
  alignas(128) T2 Ls[NB * TILE];  // L21 tile, [kk][row]; reused for L11 during the TRSM
  T2 Us[NB * US_LD];              // U12 tile, [kk][col], padded
};
using LuSmem = LuSmemT<double2>;

template <typename R>
__device__ __forceinline__ void warp_argmax(R& v, int& i) {
  for (int o = 16; o > 0; o >>= 1) {
    R ov = __shfl_down_sync(0xffffffffu, v, o);
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
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = gtid() & 31, wid = gtid() >> 5;
  v = warp_sum(v);
  gsync();
  if (lane == 0) red[wid] = v;
  gsync();
  double t = 0.0;
  for (int k = 0; k < THREADS / 32; ++k) t += red[k];
  return t;
}

// Block sum of a complex value; every thread gets the result.
__device__ __forceinline__ double2 block_sum2(double2 v, double2* red2) {
  const int lane = gtid() & 31, wid = gtid() >> 5;
  v = warp_sum2(v);
  gsync();
  if (lane == 0) red2[wid] = v;
  gsync();
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
// Panel factorisation of columns k0..k0+kb-1 (rows k0..n-1), with the row swaps
// applied across columns c_first..ncols-1 (0: all columns, LAPACK's order; k0:
// not to the L columns left of the panel, LINPACK's order).
template <typename T2>
__device__ void cta_lu_panel(T2* __restrict__ M, int n, int ncols, int k0, int kb, int* __restrict__ piv,
                             LuSmemT<T2>& sm, int c_first = 0) {
  const int tid = gtid();
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  // ---- panel factorisation, columns k0..kend-1 ----
  using R = decltype(l1abs(T2{}));  // pivot magnitudes in the matrix's own precision
  // rows and columns a thread handles per batch: all loads of a batch are issued
  // before its stores, so that each batch costs one memory round trip
  constexpr int RB = sizeof(T2) == 8 ? 4 : 2, CB = RB;
  for (int j = k0; j < kend; ++j) {
    T2* colj = M + (size_t)j * ld;
    R bv = R(-1);
    int bi = n;
    for (int i = j + tid; i < n; i += THREADS) {
      const R v = l1abs(colj[i]);
      if (v > bv) { bv = v; bi = i; }
    }
    warp_argmax(bv, bi);
    if ((tid & 31) == 0) { sm.red_v[tid >> 5] = (double)bv; sm.red_i[tid >> 5] = bi; }
    gsync();
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
    gsync();
    const int p = sm.piv_sh;
    if (p != j) {
      for (int c0 = c_first + tid; c0 < ncols; c0 += THREADS * RB) {
        T2 a[RB], b[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const int c = c0 + u * THREADS;
          if (c < ncols) {
            a[u] = M[(size_t)c * ld + j];
            b[u] = M[(size_t)c * ld + p];
          }
        }
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const int c = c0 + u * THREADS;
          if (c < ncols) {
            M[(size_t)c * ld + j] = b[u];
            M[(size_t)c * ld + p] = a[u];
          }
        }
      }
    }
    gsync();
    for (int c = j + 1 + tid; c < kend; c += THREADS) sm.prow[c - k0] = M[(size_t)c * ld + j];
    const T2 pv = colj[j];
    const bool zero = cis_zero(pv);
    if (zero && tid == 0 && sm.info_sh == 0) sm.info_sh = j + 1;
    gsync();
    if (!zero) {
      const T2 rp = crecip(pv);
      for (int i0 = j + 1 + tid; i0 < n; i0 += THREADS * RB) {
        T2 lv[RB];  // multipliers l_ij of this thread's rows
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int i = i0 + r * THREADS;
          lv[r] = i < n ? colj[i] : czero<T2>();
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int i = i0 + r * THREADS;
          lv[r] = cmul(lv[r], rp);
          if (i < n) colj[i] = lv[r];
        }
        for (int c = j + 1; c < kend; c += CB) {
          T2 mv[CB][RB];
#pragma unroll
          for (int q = 0; q < CB; ++q)
#pragma unroll
            for (int r = 0; r < RB; ++r) {
              const int i = i0 + r * THREADS;
              mv[q][r] = (c + q < kend && i < n) ? M[(size_t)(c + q) * ld + i] : czero<T2>();
            }
#pragma unroll
          for (int q = 0; q < CB; ++q)
#pragma unroll
            for (int r = 0; r < RB; ++r) {
              const int i = i0 + r * THREADS;
              if (c + q < kend && i < n) {
                cfms(mv[q][r], lv[r], sm.prow[c + q - k0]);
                M[(size_t)(c + q) * ld + i] = mv[q][r];
              }
            }
        }
      }
    }
    gsync();
  }
}

// The same panel factorisation (same pivots, same arithmetic up to the order of
// the updates of each element) in sub-panels of SB <= 8 columns held in shared
// memory: each sub-panel is loaded once, factored column by column in shared
// memory, written back, and then applied to the rest of the panel (its row
// swaps as one gather, the unit lower triangular solve for its U rows, and one
// rank-SB update). The row swaps of the columns outside the panel (and of the
// panel's earlier sub-panels) are applied after the panel (cta_panel_swaps_lp,
// with the sub-panel width this returns).
// scratch: shared memory of scratch_elems elements, at least (n - k0) + 8 NB + 40
// (then SB = 1).
template <typename T2>
__device__ __noinline__ int cta_lu_panel_sub(T2* __restrict__ M, int n, int ncols, int k0, int kb, int* __restrict__ piv,
                                 LuSmemT<T2>& sm, T2* __restrict__ scratch, int scratch_elems) {
  const int tid = gtid();
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  using R = decltype(l1abs(T2{}));
  constexpr int SBMAX = 8, CHUNK = 8;
  const int m0 = n - k0;
  int SB = SBMAX;
  while (SB > 1 && (size_t)m0 * SB + (size_t)NB * SBMAX + 40 > (size_t)scratch_elems) SB >>= 1;
  T2* sp = scratch;                                  // sub-panel, rows p0..n-1, leading dimension m
  T2* us = scratch + (size_t)m0 * SB;                // its U rows for the rest of the panel, [col][t]
  int* mp = reinterpret_cast<int*>(us + NB * SBMAX);  // composed swaps: count, dst[2 SBMAX], src[2 SBMAX]
  for (int p0 = k0; p0 < kend; p0 += SB) {
    const int sb = min(SB, kend - p0);
    const int m = n - p0;
    // 1. load (many loads in flight per thread: one round trip per 16 elements)
#pragma unroll 16
    for (int e = tid; e < m * sb; e += THREADS) {
      const int r = e % m, c = e / m;
      sp[(size_t)c * m + r] = M[(size_t)(p0 + c) * ld + p0 + r];
    }
    gsync();
    // 2. factor in shared memory
    for (int j = 0; j < sb; ++j) {
      R bv = R(-1);
      int bi = m;
      for (int r = j + tid; r < m; r += THREADS) {
        const R v = l1abs(sp[(size_t)j * m + r]);
        if (v > bv) { bv = v; bi = r; }
      }
      warp_argmax(bv, bi);
      if ((tid & 31) == 0) { sm.red_v[tid >> 5] = (double)bv; sm.red_i[tid >> 5] = bi; }
      gsync();
      if (tid == 0) {
        double v = sm.red_v[0];
        int ii = sm.red_i[0];
        for (int w = 1; w < THREADS / 32; ++w)
          if (sm.red_v[w] > v || (sm.red_v[w] == v && sm.red_i[w] < ii)) { v = sm.red_v[w]; ii = sm.red_i[w]; }
        if (ii >= m) ii = j;
        sm.piv_sh = ii;
        piv[p0 + j] = p0 + ii;
      }
      gsync();
      const int pr = sm.piv_sh;
      if (pr != j && tid < sb) {
        const T2 t = sp[(size_t)tid * m + j];
        sp[(size_t)tid * m + j] = sp[(size_t)tid * m + pr];
        sp[(size_t)tid * m + pr] = t;
      }
      gsync();
      const T2 pv = sp[(size_t)j * m + j];
      const bool zero = cis_zero(pv);
      if (zero && tid == 0 && sm.info_sh == 0) sm.info_sh = p0 + j + 1;
      if (!zero) {
        const T2 rp = crecip(pv);
        for (int r = j + 1 + tid; r < m; r += THREADS) {
          const T2 lv = cmul(sp[(size_t)j * m + r], rp);
          sp[(size_t)j * m + r] = lv;
          for (int c = j + 1; c < sb; ++c) cfms(sp[(size_t)c * m + r], lv, sp[(size_t)c * m + j]);
        }
      }
      gsync();
    }
    // 3. write back
#pragma unroll 4
    for (int e = tid; e < m * sb; e += THREADS) {
      const int r = e % m, c = e / m;
      M[(size_t)(p0 + c) * ld + p0 + r] = sp[(size_t)c * m + r];
    }
    const int c1 = p0 + sb, nr = kend - c1;  // the rest of the panel
    if (nr > 0) {
      // the sub-panel's swaps composed: row dst[i] receives the old row src[i]
      if (tid == 0) {
        int cnt = 0;
        int* dst = mp + 1;
        int* src = mp + 1 + 2 * SBMAX;
        for (int j = 0; j < sb; ++j) {
          const int a = p0 + j, b = piv[p0 + j];
          if (a == b) continue;
          int ia = -1, ib = -1;
          for (int i = 0; i < cnt; ++i) {
            if (dst[i] == a) ia = i;
            if (dst[i] == b) ib = i;
          }
          if (ia < 0) { ia = cnt; dst[cnt] = a; src[cnt] = a; ++cnt; }
          if (ib < 0) { ib = cnt; dst[cnt] = b; src[cnt] = b; ++cnt; }
          const int t = src[ia];
          src[ia] = src[ib];
          src[ib] = t;
        }
        mp[0] = cnt;
      }
      gsync();
      {
        const int cnt = mp[0];
        const int* dst = mp + 1;
        const int* src = mp + 1 + 2 * SBMAX;
        constexpr int GU = (2 * SBMAX * NB + THREADS - 1) / THREADS;  // gather elements per thread
        T2 tmp[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
          const int e = tid + u * THREADS;
          if (e < cnt * nr) tmp[u] = M[(size_t)(c1 + e / cnt) * ld + src[e % cnt]];
        }
        gsync();
#pragma unroll
        for (int u = 0; u < GU; ++u) {
          const int e = tid + u * THREADS;
          if (e < cnt * nr) M[(size_t)(c1 + e / cnt) * ld + dst[e % cnt]] = tmp[u];
        }
      }
      gsync();
      // U rows p0..p0+sb-1 of the rest: unit lower triangular solve with L11 (one thread per column)
      for (int c = tid; c < nr; c += THREADS) {
        T2 u[SBMAX];
#pragma unroll
        for (int t = 0; t < SBMAX; ++t)
          if (t < sb) u[t] = M[(size_t)(c1 + c) * ld + p0 + t];
#pragma unroll
        for (int t = 1; t < SBMAX; ++t)
#pragma unroll
          for (int q = 0; q < SBMAX; ++q)
            if (t < sb && q < t) cfms(u[t], sp[(size_t)q * m + t], u[q]);
#pragma unroll
        for (int t = 0; t < SBMAX; ++t)
          if (t < sb) {
            M[(size_t)(c1 + c) * ld + p0 + t] = u[t];
            us[c * SBMAX + t] = u[t];
          }
      }
      gsync();
      // rank-sb update of rows p0+sb..n-1 of the rest, CHUNK columns in flight per row
      for (int r = sb + tid; r < m; r += THREADS) {
        T2 lr[SBMAX];
#pragma unroll
        for (int t = 0; t < SBMAX; ++t) lr[t] = t < sb ? sp[(size_t)t * m + r] : czero<T2>();
        for (int cc = 0; cc < nr; cc += CHUNK) {
          T2 v[CHUNK];
#pragma unroll
          for (int q = 0; q < CHUNK; ++q)
            if (cc + q < nr) v[q] = M[(size_t)(c1 + cc + q) * ld + p0 + r];
#pragma unroll
          for (int q = 0; q < CHUNK; ++q)
            if (cc + q < nr) {
#pragma unroll
              for (int t = 0; t < SBMAX; ++t)
                if (t < sb) cfms(v[q], lr[t], us[(cc + q) * SBMAX + t]);
              M[(size_t)(c1 + cc + q) * ld + p0 + r] = v[q];
            }
        }
      }
    }
    gsync();
  }
  return SB;
}

// ---------------------------------------------------------------------------
// Row interchanges in LINPACK's order (the precision form's FP32 LU): a panel's
// swaps reach the panel's own columns and the columns right of it, never the L
// columns left of it, so a forward solve applies each panel's swaps to the
// right-hand side just before that panel's columns of L. A panel's swaps are
// handled as one permutation of at most 2 NB rows.
// ---------------------------------------------------------------------------
constexpr int SWAP_LIST_INTS = 1 + 4 * NB;  // [cnt, dst[2 NB], src[2 NB]]

// The swaps piv[a..b-1] (row j with row piv[j], in that order) as one permutation:
// row dst[i] receives the old row src[i], i < cnt. One thread.
__device__ inline void compose_swaps(const int* __restrict__ piv, int a, int b, int* __restrict__ list) {
  int cnt = 0;
  int* dst = list + 1;
  int* src = list + 1 + 2 * NB;
  for (int j = a; j < b; ++j) {
    const int p = piv[j];
    if (p == j) continue;
    int ia = -1, ib = -1;
    for (int i = 0; i < cnt; ++i) {
      if (dst[i] == j) ia = i;
      if (dst[i] == p) ib = i;
    }
    if (ia < 0) { ia = cnt; dst[cnt] = j; src[cnt] = j; ++cnt; }
    if (ib < 0) { ib = cnt; dst[cnt] = p; src[cnt] = p; ++cnt; }
    const int t = src[ia];
    src[ia] = src[ib];
    src[ib] = t;
  }
  list[0] = cnt;
}

// The permutation in list (shared memory, complete before the call) on columns
// c_lo..c_hi-1 of M, staged through stage (stage_elems elements of shared memory):
// all of a chunk's rows are read before any is written. All threads; returns with
// the group synchronised.
template <typename T2>
__device__ void apply_row_perm(T2* __restrict__ M, size_t ld, int c_lo, int c_hi, const int* __restrict__ list,
                               T2* __restrict__ stage, int stage_elems) {
  const int cnt = list[0];
  if (cnt > 0 && c_hi > c_lo) {
    const int* dst = list + 1;
    const int* src = list + 1 + 2 * NB;
    const int per = max(1, stage_elems / cnt);
    for (int c0 = c_lo; c0 < c_hi; c0 += per) {
      const int tot = min(per, c_hi - c0) * cnt;
#pragma unroll 8
      for (int e = gtid(); e < tot; e += THREADS) stage[e] = M[(size_t)(c0 + e / cnt) * ld + src[e % cnt]];
      gsync();
#pragma unroll 8
      for (int e = gtid(); e < tot; e += THREADS) M[(size_t)(c0 + e / cnt) * ld + dst[e % cnt]] = stage[e];
      gsync();
    }
  }
  gsync();
}

// After cta_lu_panel_sub (sub-panels of SB columns), in LINPACK's order: the
// panel's swaps on the columns right of it, and on each sub-panel's columns the
// swaps of the later sub-panels (a sub-panel's own swaps and those before it are
// already in its columns). The panel's whole permutation is also written to
// list_out (global memory) for the forward solves. scratch: shared memory of
// scratch_bytes bytes, of which the last SWAP_LIST_INTS ints hold a list.
template <typename T2>
__device__ void cta_panel_swaps_lp(T2* __restrict__ M, int n, int ncols, int k0, int kb, const int* __restrict__ piv,
                                   int SB, int* __restrict__ list_out, unsigned char* scratch, int scratch_bytes) {
  const int tid = gtid();
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  int* ls = reinterpret_cast<int*>(scratch + scratch_bytes) - SWAP_LIST_INTS;
  T2* stage = reinterpret_cast<T2*>(scratch);
  const int elems = (int)((reinterpret_cast<unsigned char*>(ls) - scratch) / sizeof(T2));
  gsync();
  if (tid == 0) compose_swaps(piv, k0, kend, ls);
  gsync();
  for (int i = tid; i < SWAP_LIST_INTS; i += THREADS) list_out[i] = ls[i];
  apply_row_perm(M, ld, kend, ncols, ls, stage, elems);
  for (int q0 = k0; q0 + SB < kend; q0 += SB) {
    if (tid == 0) compose_swaps(piv, q0 + SB, kend, ls);
    gsync();
    apply_row_perm(M, ld, q0, q0 + SB, ls, stage, elems);
  }
}

// U12 = L11^{-1} A12 for rows k0..k0+kb-1, columns k0+kb..ncols-1.
template <typename T2>
__device__ void cta_lu_trsm(T2* __restrict__ M, int n, int ncols, int k0, int kb, LuSmemT<T2>& sm) {
  const int tid = gtid();
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  // ---- U12 = L11^{-1} A12 (rows k0..kend-1, columns kend..ncols-1) ----
  for (int e = tid; e < kb * kb; e += THREADS) {
    int r = e % kb, c = e / kb;
    sm.Ls[c * NB + r] = M[(size_t)(k0 + c) * ld + k0 + r];  // Ls[t*NB + i] = L11[i][t]
  }
  gsync();
  {
    // a warp takes CW columns at a time, lane i holds row k0+i of each (NB == warp
    // size); the CW substitutions are independent, so their shuffle chains overlap
    constexpr int CW = 4;
    constexpr int STRIDE = (THREADS / 32) * CW;
    const int lane = tid & 31, wid = tid >> 5;
    // the loads of a warp's next column group are issued before this group's
    // substitution, so that their latency overlaps it
    T2 xn[CW];
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      const int c = kend + wid * CW + q;
      xn[q] = (lane < kb && c < ncols) ? M[(size_t)c * ld + k0 + lane] : czero<T2>();
    }
    for (int c0 = kend + wid * CW; c0 < ncols; c0 += STRIDE) {
      T2 x[CW];
#pragma unroll
      for (int q = 0; q < CW; ++q) {
        x[q] = xn[q];
        const int c = c0 + STRIDE + q;
        xn[q] = (lane < kb && c < ncols) ? M[(size_t)c * ld + k0 + lane] : czero<T2>();
      }
      for (int t = 0; t < kb - 1; ++t) {
        const T2 lt = sm.Ls[t * NB + lane];
#pragma unroll
        for (int q = 0; q < CW; ++q) {
          T2 xt;
          xt.x = __shfl_sync(0xffffffffu, x[q].x, t);
          xt.y = __shfl_sync(0xffffffffu, x[q].y, t);
          if (lane > t && lane < kb) cfms(x[q], lt, xt);
        }
      }
#pragma unroll
      for (int q = 0; q < CW; ++q)
        if (lane < kb && c0 + q < ncols) M[(size_t)(c0 + q) * ld + k0 + lane] = x[q];
    }
  }
  gsync();
}

// Trailing update A22 -= L21 U12 (rows and columns from k0+kb on), FMA pipes.
// RI x RI register block per thread on a 16 x 16 thread grid: tiles of 16 RI x 16 RI
// (RI = 4: 64 x 64, the default; RI = 2: 32 x 32, less padding on small matrices,
// chosen by the autotuner per problem size).
template <typename T2, int RI = 4>
__device__ void cta_lu_update_simt(T2* __restrict__ M, int n, int ncols, int k0, int kb, LuSmemT<T2>& sm) {
  constexpr int TT = 16 * RI;
  static_assert(TT <= TILE, "the shared tiles are sized for TILE");
  const int tid = gtid();
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  // ---- trailing update A22 -= L21 U12 over TT x TT tiles ----
  const int m_rows = n - kend, m_cols = ncols - kend;
  const int mt = (m_rows + TT - 1) / TT, nt = (m_cols + TT - 1) / TT;
  const int tx = tid & 15, ty = tid >> 4;
  for (int ti = 0; ti < mt; ++ti) {
    const int r0 = kend + ti * TT;
    static_assert((NB * TT) % THREADS == 0, "tile staging mapping");
#pragma unroll
    for (int u = 0; u < NB * TT / THREADS; ++u) {  // unrolled: all loads in flight at once
      const int e = tid + u * THREADS;
      int r = e % TT, kk = e / TT;
      T2 v = czero<T2>();
      if (kk < kb && r0 + r < n) v = M[(size_t)(k0 + kk) * ld + r0 + r];
      sm.Ls[kk * TT + r] = v;
    }
    for (int tj = 0; tj < nt; ++tj) {
      const int c0 = kend + tj * TT;
#pragma unroll
      for (int u = 0; u < NB * TT / THREADS; ++u) {
        const int e = tid + u * THREADS;
        int kk = e % NB, c = e / NB;
        T2 v = czero<T2>();
        if (kk < kb && c0 + c < ncols) v = M[(size_t)(c0 + c) * ld + k0 + kk];
        sm.Us[kk * US_LD + c] = v;
      }
      gsync();
      T2 acc[RI][RI];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int q = 0; q < RI; ++q) {
          int r = r0 + tx + 16 * i, c = c0 + ty + 16 * q;
          acc[i][q] = (r < n && c < ncols) ? M[(size_t)c * ld + r] : czero<T2>();
        }
      // a thread whose rows (tx + 16 i) or columns (ty + 16 q) all lie past the matrix has
      // nothing to update: on the ragged last tiles (most of each tile when n is small) it skips
      // the multiply instead of running it on padding
      if (r0 + tx < n && c0 + ty < ncols) {
        for (int kk = 0; kk < kb; ++kk) {
          T2 a[RI], b[RI];
#pragma unroll
          for (int i = 0; i < RI; ++i) a[i] = sm.Ls[kk * TT + tx + 16 * i];
#pragma unroll
          for (int q = 0; q < RI; ++q) b[q] = sm.Us[kk * US_LD + ty + 16 * q];
#pragma unroll
          for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int q = 0; q < RI; ++q) cfms(acc[i][q], a[i], b[q]);
        }
      }
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int q = 0; q < RI; ++q) {
          int r = r0 + tx + 16 * i, c = c0 + ty + 16 * q;
          if (r < n && c < ncols) M[(size_t)c * ld + r] = acc[i][q];
        }
      gsync();
    }
  }
}

template <typename T2, int RI = 4>
__device__ int cta_lu(T2* __restrict__ M, int n, int ncols, int* __restrict__ piv, LuSmemT<T2>& sm) {
  if (gtid() == 0) sm.info_sh = 0;
  gsync();
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    const int kend = k0 + kb;
    cta_lu_panel(M, n, ncols, k0, kb, piv, sm);
    if (kend >= ncols) continue;
    cta_lu_trsm(M, n, ncols, k0, kb, sm);
    if (kend >= n) continue;
    cta_lu_update_simt<T2, RI>(M, n, ncols, k0, kb, sm);
  }
  gsync();
  return sm.info_sh;
}

// Back substitution U X = Y for the l columns n..n+l-1 of M, in place.
template <typename T2>
__device__ void cta_back_subst(T2* __restrict__ M, int n, int l, LuSmemT<T2>& sm) {
  const int tid = gtid();
  const size_t ld = (size_t)n;
  T2* Y = M + (size_t)n * ld;
  for (int j = n - 1; j >= 0; --j) {
    if (tid < l) {
      T2 x = cdiv(Y[(size_t)tid * ld + j], M[(size_t)j * ld + j]);
      Y[(size_t)tid * ld + j] = x;
      sm.bcast[tid] = x;
    }
    gsync();
    const T2* uj = M + (size_t)j * ld;
    for (int i = tid; i < j; i += THREADS) {
      const T2 u = uj[i];
      for (int c = 0; c < l; ++c) cfms(Y[(size_t)c * ld + i], u, sm.bcast[c]);
    }
    gsync();
  }
}

// ---------------------------------------------------------------------------
// Blocked triangular solves on the l columns n..n+l-1 of M (32-row blocks):
// the 32 x 32 diagonal block is solved one warp per column (lane = row), then
// the rows outside the block are updated by all threads (coalesced over rows).
// Two barriers per block instead of two per row.
// ---------------------------------------------------------------------------

// Y[i, :] -= M[i, k0:k0+kb] * S where S (kb x l) sits in sm.Us ([t][c]).
// Columns in register chunks (16 complex64 or 8 complex128), so M is read once
// per chunk; the M elements of 8 steps are loaded before they are used, so that
// their memory latencies overlap instead of adding up.
template <typename T2>
__device__ __forceinline__ void block_update_row(const T2* __restrict__ M, T2* __restrict__ Y, size_t ld, int i,
                                                 int k0, int kb, int l, LuSmemT<T2>& sm) {
  constexpr int CH = sizeof(T2) == 8 ? 16 : 8;
  for (int c0 = 0; c0 < l; c0 += CH) {
    T2 acc[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) acc[q] = (c0 + q < l) ? Y[(size_t)(c0 + q) * ld + i] : czero<T2>();
    for (int t0 = 0; t0 < kb; t0 += 8) {
      T2 m[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) m[u] = (t0 + u < kb) ? M[(size_t)(k0 + t0 + u) * ld + i] : czero<T2>();
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t0 + u < kb) {  // rows of S past kb hold stale values
#pragma unroll
          for (int q = 0; q < CH; ++q) cfms(acc[q], m[u], sm.Us[(t0 + u) * US_LD + c0 + q]);
        }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (c0 + q < l) Y[(size_t)(c0 + q) * ld + i] = acc[q];
  }
}


// U x = y, U upper with its diagonal.
template <typename T2>
__device__ void cta_back_blocked(T2* __restrict__ M, int n, int l, LuSmemT<T2>& sm) {
  const int tid = gtid(), lane = tid & 31, wid = tid >> 5;
  const size_t ld = (size_t)n;
  T2* Y = M + (size_t)n * ld;
  const int nblk = (n + NB - 1) / NB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * NB;
    const int kb = min(NB, n - k0);
    for (int e = tid; e < kb * kb; e += THREADS) {
      const int r = e % kb, c = e / kb;
      sm.Ls[c * NB + r] = M[(size_t)(k0 + c) * ld + k0 + r];  // Ls[t*NB + i] = U[k0+i][k0+t]
    }
    gsync();
    for (int c = wid; c < l; c += THREADS / 32) {
      T2* yc = Y + (size_t)c * ld + k0;
      T2 y = (lane < kb) ? yc[lane] : czero<T2>();
      for (int t = kb - 1; t >= 0; --t) {
        if (lane == t) y = cdiv(y, sm.Ls[t * NB + t]);
        T2 xt;
        xt.x = __shfl_sync(0xffffffffu, y.x, t);
        xt.y = __shfl_sync(0xffffffffu, y.y, t);
        if (lane < t) cfms(y, sm.Ls[t * NB + lane], xt);
      }
      if (lane < kb) yc[lane] = y;
      if (lane < kb) sm.Us[lane * US_LD + c] = y;
    }
    gsync();
    for (int i = tid; i < k0; i += THREADS) block_update_row(M, Y, ld, i, k0, kb, l, sm);
    gsync();
  }
}

// L y = b for the l columns after the n x n block of M, with L from an LU whose
// row interchanges are in LINPACK's order: before panel p's columns of L, its
// permutation (lists + p SWAP_LIST_INTS, global memory) is applied to y.
template <typename T2>
__device__ void cta_fwd_blocked_lp(T2* __restrict__ M, int n, int l, LuSmemT<T2>& sm, const int* __restrict__ lists) {
  const int tid = gtid(), lane = tid & 31, wid = tid >> 5;
  const size_t ld = (size_t)n;
  T2* Y = M + (size_t)n * ld;
  constexpr int GU = 4;  // permuted elements per thread and round
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    {
      const int* L = lists + (size_t)(k0 / NB) * SWAP_LIST_INTS;
      const int cnt = L[0];
      const int* dst = L + 1;
      const int* src = L + 1 + 2 * NB;
      // whole columns per round, so that a column's rows are all read before any is written
      const int per = cnt > 0 ? max(1, GU * THREADS / cnt) : l;
      for (int c0 = 0; c0 < l && cnt > 0; c0 += per) {
        const int tot = min(per, l - c0) * cnt;
        T2 v[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
          const int e = tid + u * THREADS;
          if (e < tot) v[u] = Y[(size_t)(c0 + e / cnt) * ld + src[e % cnt]];
        }
        gsync();
#pragma unroll
        for (int u = 0; u < GU; ++u) {
          const int e = tid + u * THREADS;
          if (e < tot) Y[(size_t)(c0 + e / cnt) * ld + dst[e % cnt]] = v[u];
        }
        gsync();
      }
    }
    for (int e = tid; e < kb * kb; e += THREADS) {
      const int r = e % kb, c = e / kb;
      sm.Ls[c * NB + r] = M[(size_t)(k0 + c) * ld + k0 + r];  // Ls[t*NB + i] = L[k0+i][k0+t]
    }
    gsync();
    for (int c = wid; c < l; c += THREADS / 32) {
      T2* yc = Y + (size_t)c * ld + k0;
      T2 y = (lane < kb) ? yc[lane] : czero<T2>();
      for (int t = 0; t < kb - 1; ++t) {
        T2 yt;
        yt.x = __shfl_sync(0xffffffffu, y.x, t);
        yt.y = __shfl_sync(0xffffffffu, y.y, t);
        if (lane > t && lane < kb) cfms(y, sm.Ls[t * NB + lane], yt);
      }
      if (lane < kb) yc[lane] = y;
      if (lane < kb) sm.Us[lane * US_LD + c] = y;  // solved block rows, [t][c]
    }
    gsync();
    for (int i = k0 + kb + tid; i < n; i += THREADS) block_update_row(M, Y, ld, i, k0, kb, l, sm);
    gsync();
  }
}


}  // namespace lucore
