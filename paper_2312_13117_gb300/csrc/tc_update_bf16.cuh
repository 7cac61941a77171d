// Trailing update of the FP32 LU on the tensor cores in BF16, with complex
// products in the 3M form (the third precision form, PMCIM_PREC_BF16X3_IR).
//
// A22 -= L21 U12 for one 32-column panel, in 128-row x 32-column tiles:
//
//   * 3M: with P1 = Lr Ur, P2 = Li Ui and P3 = (Lr + Li)(Ur + Ui), the complex
//     product is D_re = P1 - P2, D_im = P3 - P1 - P2: three real products instead
//     of four. The sums Lr + Li and Ur + Ui are formed in FP32;
//   * each FP32 operand x is split into three BF16 parts, x0 = bf16(x),
//     x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (round to nearest even), so that
//     x - x0 - x1 - x2 is below 2^-24 |x|; a real product keeps the six part
//     products x_s y_t with s + t <= 2 (the dropped ones are below 2^-26 |x||y|),
//     accumulated in FP32 by tcgen05.mma of kind::f16 (M = 128, N = 32, K = 16).
//     The update is then accurate to FP32 level, as the FP64 refinement around the
//     LU assumes; 3M adds the cancellation of P3 - P1 - P2, an absolute error of
//     the order of 2^-24 (|Lr| + |Li|)(|Ur| + |Ui|);
//   * per tile the three products sit in three 32-column TMEM accumulators; two
//     tiles' accumulators (192 of the factor group's 256 columns) alternate, so the
//     epilogue of tile t runs while the tensor cores multiply tile t+1;
//   * the operand stage holds the nine BF16 planes of L21 (3 operands x 3 parts,
//     128 x 32 each, 72 KB) and the nine of one U12 tile (18 KB), in the canonical
//     K-major no-swizzle layout (8-row x 16-byte core matrices, LBO 128 B, SBO
//     512 B). One U12 set only (the stage is the 96 KB that the 3xTF32 form uses):
//     tile t+1's U12 is staged after tile t's products have read the set.
//
// Thread 0 issues the MMAs and commits them to an mbarrier; every wait on it is
// bounded, with the same fallback as the 3xTF32 form (tc_update.cuh).
#pragma once
#include <cstddef>
#include <cstdint>

#include "tc_update.cuh"

namespace tcb {

constexpr int TM = 128, TN = 32, TK = 32;
constexpr int PLANE_A = TM * TK * 2;         // one BF16 plane of L21: 8 KB
constexpr int PLANE_B = TN * TK * 2;         // one BF16 plane of U12: 2 KB
constexpr int PARTS = 3;
constexpr int A_BYTES = 3 * PARTS * PLANE_A;  // [Lr, Li, Lr + Li] x 3 parts: 72 KB
constexpr int B_BYTES = 3 * PARTS * PLANE_B;  // [Ur, Ui, Ur + Ui] x 3 parts: 18 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t ACC_COLS = 3 * TN;         // P1, P2, P3 of one tile
static_assert(STAGE_BYTES <= tcu::STAGE_BYTES, "the operands fit the 3xTF32 form's stage");
static_assert(2 * ACC_COLS <= 256, "two tiles' accumulators in the factor group's TMEM columns");
static_assert(TK == lucore::NB, "the tensor-core tile is one panel deep");

// Byte offset of element (row r, inner index k) in a K-major BF16 plane of 32 inner indices.
__device__ __forceinline__ int off(int r, int k) { return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         (1ull << 46);
}

// kind::f16: F32 accumulator, BF16 A and B, both K-major, N = TN, M = TM.
__device__ __forceinline__ uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(da), "l"(db), "r"(id), "r"(acc));
}

// One 8-column load of this warp's 32 TMEM lanes, and the wait for it.
__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(addr)
      : "memory");
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ uint16_t bf16_rn(float x) {
  uint16_t h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
  return h;
}
__device__ __forceinline__ float bf16_val(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// The three BF16 parts of x.
__device__ __forceinline__ void split3(float x, uint16_t& p0, uint16_t& p1, uint16_t& p2) {
  p0 = bf16_rn(x);
  const float r1 = x - bf16_val(p0);
  p1 = bf16_rn(r1);
  p2 = bf16_rn(r1 - bf16_val(p1));
}

// Stage L21 rows r0..r0+127 (panel columns k0..k0+kb-1) as nine planes. Thread t
// takes row t % 128 and the k-octets t / 128 and t / 128 + 2: 16 values, all loads
// in flight before the first store.
__device__ __forceinline__ void stage_L(const float2* __restrict__ M, size_t ld, int n, int r0, int k0, int kb,
                                        unsigned char* st) {
  const int tid = lucore::gtid();
  const int r = tid & (TM - 1);
  const bool row_ok = r0 + r < n;
  float2 v[2][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = 8 * ((tid >> 7) + 2 * i) + t;
      v[i][t] = (row_ok && k < kb) ? M[(size_t)(k0 + k) * ld + r0 + r] : make_float2(0.f, 0.f);
    }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int o = off(r, 8 * ((tid >> 7) + 2 * i));
    uint32_t w[3][PARTS][4];  // [operand][part][packed pairs]
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      uint16_t a[3][PARTS], b[3][PARTS];
      split3(v[i][t].x, a[0][0], a[0][1], a[0][2]);
      split3(v[i][t].y, a[1][0], a[1][1], a[1][2]);
      split3(v[i][t].x + v[i][t].y, a[2][0], a[2][1], a[2][2]);
      split3(v[i][t + 1].x, b[0][0], b[0][1], b[0][2]);
      split3(v[i][t + 1].y, b[1][0], b[1][1], b[1][2]);
      split3(v[i][t + 1].x + v[i][t + 1].y, b[2][0], b[2][1], b[2][2]);
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int p = 0; p < PARTS; ++p) w[q][p][t / 2] = (uint32_t)a[q][p] | ((uint32_t)b[q][p] << 16);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int p = 0; p < PARTS; ++p)
        *reinterpret_cast<uint4*>(st + (q * PARTS + p) * PLANE_A + o) =
            make_uint4(w[q][p][0], w[q][p][1], w[q][p][2], w[q][p][3]);
  }
}

// Stage U12 rows k0..k0+kb-1 of columns c0..c0+31 (bounded by ncols) as nine
// planes at bset. Thread t takes column t % 32 and the four values 4 (t / 32) ..
// 4 (t / 32) + 3 of it.
__device__ __forceinline__ void stage_U(const float2* __restrict__ M, size_t ld, int ncols, int c0, int k0, int kb,
                                        unsigned char* bset) {
  const int tid = lucore::gtid();
  const int c = tid & (TN - 1), q4 = tid >> 5;
  const bool col_ok = c0 + c < ncols;
  float2 v[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int k = 4 * q4 + t;
    v[t] = (col_ok && k < kb) ? M[(size_t)(c0 + c) * ld + k0 + k] : make_float2(0.f, 0.f);
  }
  uint32_t w[3][PARTS][2];
#pragma unroll
  for (int t = 0; t < 4; t += 2) {
    uint16_t a[3][PARTS], b[3][PARTS];
    split3(v[t].x, a[0][0], a[0][1], a[0][2]);
    split3(v[t].y, a[1][0], a[1][1], a[1][2]);
    split3(v[t].x + v[t].y, a[2][0], a[2][1], a[2][2]);
    split3(v[t + 1].x, b[0][0], b[0][1], b[0][2]);
    split3(v[t + 1].y, b[1][0], b[1][1], b[1][2]);
    split3(v[t + 1].x + v[t + 1].y, b[2][0], b[2][1], b[2][2]);
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int p = 0; p < PARTS; ++p) w[q][p][t / 2] = (uint32_t)a[q][p] | ((uint32_t)b[q][p] << 16);
  }
  const int o = off(c, 4 * q4);
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int p = 0; p < PARTS; ++p)
      *reinterpret_cast<uint2*>(bset + (q * PARTS + p) * PLANE_B + o) = make_uint2(w[q][p][0], w[q][p][1]);
}

// Thread 0: the 36 MMAs of one tile (3 products x 6 part pairs x 2 K-steps of 16)
// into accumulator set b, then the commit to barrier b.
__device__ __forceinline__ void issue_tile_3m(const tcu::Ctx& cx, int b) {
  const uint32_t sa = tcu::smem_u32(cx.stage), sb = sa + A_BYTES;
  const uint32_t id = idesc();
  const int ps[6] = {0, 0, 1, 0, 1, 2}, pt[6] = {0, 1, 0, 2, 1, 0};  // part pairs s + t <= 2
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const uint32_t d = cx.tmem + (uint32_t)b * ACC_COLS + (uint32_t)(q * TN);
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const uint32_t a = sa + (uint32_t)((q * PARTS + ps[j]) * PLANE_A);
      const uint32_t bb = sb + (uint32_t)((q * PARTS + pt[j]) * PLANE_B);
#pragma unroll
      for (int ks = 0; ks < TK / 16; ++ks) {
        const uint32_t o = (uint32_t)(ks * 256);  // 16 BF16 = two core matrices along K
        mma(d, desc(a + o), desc(bb + o), id, acc);
        acc = 1u;
      }
    }
  }
  tcu::commit(cx.mbar + b);
}

// A22 -= L21 U12 for the panel k0..k0+kb-1. All threads of the group call it; it
// returns with the group synchronised and no MMA in flight, unless a wait ran out
// (then *cx.bad is set and the rest of the panel's update is skipped).
__device__ inline void update(float2* __restrict__ M, int n, int ncols, int k0, int kb, tcu::Ctx& cx) {
  const int tid = lucore::gtid(), warp = tid >> 5, lane = tid & 31;
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32*quad.., tile columns 16*half..
  const uint32_t lane_base = cx.tmem + ((uint32_t)(32 * quad) << 16);
  unsigned char* bset = cx.stage + A_BYTES;
  const int T = (ncols - kend + TN - 1) / TN;  // column tiles of a row block
  for (int r0 = kend; r0 < n; r0 += TM) {
    stage_L(M, ld, n, r0, k0, kb, cx.stage);
    stage_U(M, ld, ncols, kend, k0, kb, bset);
    tcu::stage_barrier();
    if (tid == 0) issue_tile_3m(cx, 0);
    const int row = r0 + 32 * quad + lane;
    for (int t = 0; t < T; ++t) {
      const int b = t & 1;
      const int c0 = kend + t * TN;
      if (t + 2 < T) tcu::prefetch_tile(M, ld, n, ncols, k0, kend, r0, t + 2);
      else if (r0 + TM < n && t + 2 - T < T) tcu::prefetch_tile(M, ld, n, ncols, k0, kend, r0 + TM, t + 2 - T);
      if (t + 3 == T && r0 + TM < n) tcu::prefetch_L(M, ld, n, k0, kend, r0 + TM);
      float2 cv[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = c0 + 16 * half + c;
        cv[c] = (row < n && col < ncols) ? M[(size_t)col * ld + row] : make_float2(0.f, 0.f);
      }
      const bool ok = tcu::wait_parity(cx.mbar + b, cx.phase[b], cx.wait_cycles);
      cx.phase[b] ^= 1u;
      if (!ok) atomicExch(cx.bad, 1);
      tcu::fence_after();
      lucore::gsync();  // tile t's products are done: the U12 set is free
      if (*cx.bad) return;
      if (t + 1 < T) {
        stage_U(M, ld, ncols, c0 + TN, k0, kb, bset);
        tcu::stage_barrier();
        if (tid == 0) issue_tile_3m(cx, b ^ 1);
      }
      const uint32_t acc = lane_base + (uint32_t)b * ACC_COLS + (uint32_t)(16 * half);
#pragma unroll
      for (int h = 0; h < 16; h += 8) {
        float p1[8], p2[8], p3[8];
        tmem_ld8(acc + (uint32_t)h, p1);
        tmem_ld8(acc + (uint32_t)(TN + h), p2);
        tmem_ld8(acc + (uint32_t)(2 * TN + h), p3);
        if (row < n) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int col = c0 + 16 * half + h + c;
            if (col < ncols)
              M[(size_t)col * ld + row] =
                  make_float2(cv[h + c].x - (p1[c] - p2[c]), cv[h + c].y - (p3[c] - p1[c] - p2[c]));
          }
        }
      }
      tcu::fence_before();  // this accumulator read is ordered before the next barrier
    }
    lucore::gsync();  // every epilogue store of the row block done before the next staging
  }
}

}  // namespace tcb
