// Trailing update of the FP32 LU on the 5th-generation tensor cores.
//
// In the right-looking blocked LU (the factorisation step of every node solve,
// Eq. 2.4) almost all arithmetic is the update A22 -= L21 U12 after each
// 32-column panel. Here it runs as tcgen05.mma of kind::tf32 with the
// accumulators in tensor memory (TMEM):
//
//   * a complex product is four real ones, D_re = Lr Ur - Li Ui and
//     D_im = Li Ur + Lr Ui; the minus sign is the MMA's negate-A bit;
//   * each FP32 operand x is split into x_big = tf32(x) and
//     x_small = tf32(x - x_big) ("3xTF32"), and every real product is
//     big*big + big*small + small*big, accumulated in FP32. The dropped
//     small*small term is below 2^-22 |x||y|, so the update has FP32-level
//     accuracy, which is what the FP64 refinement around the LU assumes;
//   * one tile is 128 rows (the MMA's M, one TMEM lane per row) by 32 columns;
//     D_re sits in TMEM columns 0..31 and D_im in 32..63 of one of two
//     accumulator buffers. The L21 tile is staged once per 128-row block and
//     reused across its column tiles;
//   * the column tiles of a row block are software-pipelined over two U12
//     buffers and two accumulators: while the tensor cores multiply tile t+1,
//     the threads stage the operands of tile t+2 and subtract tile t from C;
//     the C values of a tile are loaded before its MMAs are waited for;
//   * operands are K-major in the canonical no-swizzle layout: 8-row x 16-byte
//     core matrices, element (r, k) at (r/8)*SBO + (k/4)*LBO + (r%8)*16 + (k%4)*4
//     with LBO = 128 and SBO = 1024 bytes (32 TF32 values per row).
//
// Thread 0 issues the MMAs and commits them to an mbarrier; every wait on it is
// bounded. A wait that runs out sets the caller's flag and the rest of that
// panel's update is skipped; the CTA's later panels use the FMA pipes. The LU is
// then inexact, which the FP64 refinement around it either absorbs (it only
// needs an approximate inverse) or answers by solving the node again in FP64.
#pragma once
#include <cstddef>
#include <cstdint>

#include "lu_core.cuh"

namespace tcu {

constexpr int TM = 128;                  // tile rows = MMA M = TMEM lanes
constexpr int TN = 32;                   // tile columns = MMA N
constexpr int TK = 32;                   // panel width (complex) = lucore::NB
constexpr int LBO = 128;                 // bytes between core matrices along K
constexpr int SBO = (TK / 4) * 128;      // bytes between 8-row groups
constexpr int A_BYTES = TM * TK * 4;     // one real TF32 operand of L21: 16 KB
constexpr int B_BYTES = TN * TK * 4;     // one real TF32 operand of U12: 4 KB
constexpr int B_SET = 4 * B_BYTES;       // [Ur_big][Ui_big][Ur_small][Ui_small]
// [Lr_big][Li_big][Lr_small][Li_small] [U12 set 0] [U12 set 1]
constexpr int STAGE_BYTES = 4 * A_BYTES + 2 * B_SET;  // 96 KB
constexpr uint32_t ACC_COLS = 2 * TN;    // D_re, D_im of one tile
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;  // two accumulators
constexpr long long WAIT_CYCLES = 1ll << 30;  // about half a second at 2 GHz

static_assert(TK == lucore::NB, "the tensor-core tile is one panel deep");
static_assert(lucore::THREADS == 256, "staging and epilogue assume 8 warps");

struct Ctx {
  unsigned char* stage;  // STAGE_BYTES of shared memory, 128-byte aligned
  uint64_t* mbar;        // two shared mbarriers (one per accumulator), count 1
  uint32_t tmem;         // TMEM address of the TMEM_COLS allocated columns
  uint32_t phase[2];     // parity of each barrier's next commit (the same in every thread)
  int* bad;              // shared flag: a wait ran out
  long long wait_cycles; // limit of one completion wait inside update()
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, LBO, SBO, descriptor version 1,
// base offset 0, no swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both
// K-major, N = TN, M = TM, optional negation of A.
__device__ __forceinline__ uint32_t idesc(uint32_t neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (neg_a << 13) | ((uint32_t)(TN >> 3) << 17) |
         ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split(float x, uint32_t& big, uint32_t& small) {
  big = tf32_bits(x);
  small = tf32_bits(x - __uint_as_float(big));
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(da), "l"(db), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity, long long limit = WAIT_CYCLES) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Two 16-column loads of this warp's 32 TMEM lanes (the real and the imaginary
// part of 16 tile columns) and the wait for them, in one statement so that no
// use of the registers can move above the wait.
__device__ __forceinline__ void tmem_ld_pair(uint32_t a_re, uint32_t a_im, float (&re)[16], float (&im)[16]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(a_re), "r"(a_im)
      : "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    re[c] = __uint_as_float(r[c]);
    im[c] = __uint_as_float(r[16 + c]);
  }
}

// Allocation, by one whole warp, before a barrier that the warps using the
// columns also pass. The column count is a power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// The same for a given column count (a power of two, 32..512).
__device__ __forceinline__ void tmem_alloc_cols(uint32_t* dst_smem, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_cols(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Core-matrix offset (bytes) of the 16-byte group holding elements (r, 4q..4q+3).
__device__ __forceinline__ int core_off(int r, int q) { return (r >> 3) * SBO + q * LBO + (r & 7) * 16; }

__device__ __forceinline__ void st_v4(unsigned char* base, int off, const uint32_t (&v)[4]) {
  *reinterpret_cast<uint4*>(base + off) = make_uint4(v[0], v[1], v[2], v[3]);
}

// Stage L21 rows r0..r0+127 (columns k0..k0+kb-1) of the column-major matrix M
// (leading dimension ld, n rows). Thread t takes row t % 128 and the k-quads
// q = t / 128 + 2 i: a warp reads 32 consecutive rows of one column at a time.
__device__ __forceinline__ void stage_L(const float2* __restrict__ M, size_t ld, int n, int r0, int k0, int kb,
                                        unsigned char* st) {
  const int tid = lucore::gtid();
  const int r = tid & (TM - 1);
  const bool row_ok = r0 + r < n;
  float2 v[4][4];  // all 16 loads in flight before the first shared store
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int k = 4 * ((tid >> 7) + 2 * i) + t;
      v[i][t] = (row_ok && k < kb) ? M[(size_t)(k0 + k) * ld + r0 + r] : make_float2(0.f, 0.f);
    }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = (tid >> 7) + 2 * i;
    uint32_t rb[4], ib[4], rs[4], is[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      split(v[i][t].x, rb[t], rs[t]);
      split(v[i][t].y, ib[t], is[t]);
    }
    const int off = core_off(r, q);
    st_v4(st + 0 * A_BYTES, off, rb);
    st_v4(st + 1 * A_BYTES, off, ib);
    st_v4(st + 2 * A_BYTES, off, rs);
    st_v4(st + 3 * A_BYTES, off, is);
  }
}

// Stage U12 rows k0..k0+kb-1 of columns c0..c0+31 (bounded by ncols) into the
// U12 set at bset. Thread t takes column t % 32 and k-quad t / 32: four
// consecutive values of a column.
__device__ __forceinline__ void stage_U(const float2* __restrict__ M, size_t ld, int ncols, int c0, int k0, int kb,
                                        unsigned char* bset) {
  const int tid = lucore::gtid();
  const int c = tid & (TN - 1), q = tid >> 5;
  const bool col_ok = c0 + c < ncols;
  float2 v[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int k = 4 * q + t;
    v[t] = (col_ok && k < kb) ? M[(size_t)(c0 + c) * ld + k0 + k] : make_float2(0.f, 0.f);
  }
  uint32_t rb[4], ib[4], rs[4], is[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    split(v[t].x, rb[t], rs[t]);
    split(v[t].y, ib[t], is[t]);
  }
  const int off = core_off(c, q);
  st_v4(bset + 0 * B_BYTES, off, rb);
  st_v4(bset + 1 * B_BYTES, off, ib);
  st_v4(bset + 2 * B_BYTES, off, rs);
  st_v4(bset + 3 * B_BYTES, off, is);
}

// Thread 0: the 48 MMAs of one tile (3 split pairs x 4 real products x 4 K-steps
// of 8) from the L21 stage and U12 set b into accumulator b, then the commit
// to barrier b.
__device__ __forceinline__ void issue_tile(const Ctx& cx, int b) {
  const uint32_t sa = smem_u32(cx.stage), sb = sa + 4 * A_BYTES + (uint32_t)(b * B_SET);
  const uint32_t id_p = idesc(0), id_n = idesc(1);
  const uint32_t d_re = cx.tmem + (uint32_t)b * ACC_COLS, d_im = d_re + (uint32_t)TN;
  // (A split, B split): big*big, big*small, small*big
  const int pa[3] = {0, 0, 2}, pb[3] = {0, 2, 0};
  uint32_t acc = 0;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const uint32_t ar = sa + (pa[p] + 0) * A_BYTES, ai = sa + (pa[p] + 1) * A_BYTES;
    const uint32_t br = sb + (pb[p] + 0) * B_BYTES, bi = sb + (pb[p] + 1) * B_BYTES;
#pragma unroll
    for (int ks = 0; ks < TK / 8; ++ks) {
      const uint32_t o = (uint32_t)(ks * 2 * LBO);  // 8 TF32 = two core matrices along K
      mma(d_re, desc(ar + o), desc(br + o), id_p, acc);
      mma(d_re, desc(ai + o), desc(bi + o), id_n, 1u);
      mma(d_im, desc(ai + o), desc(br + o), id_p, acc);
      mma(d_im, desc(ar + o), desc(bi + o), id_p, 1u);
      acc = 1u;
    }
  }
  commit(cx.mbar + b);
}

// Shared-memory writes of the staging threads made visible to the tensor cores,
// and the group synchronised (tcgen05 ordering on both sides of the barrier).
__device__ __forceinline__ void stage_barrier() {
  fence_async_smem();
  fence_before();
  lucore::gsync();
  fence_after();
}

// Hint to bring the 128-byte line holding p into L2 (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of what tile tt of the row block at r0 will load: its C values (32
// columns x 128 rows: one line per thread) and its U12 operand (32 columns x 32
// rows: two lines per column). Only addresses inside the matrix are touched.
__device__ __forceinline__ void prefetch_tile(const float2* M, size_t ld, int n, int ncols, int k0, int kend,
                                              int r0, int tt) {
  const int tid = lucore::gtid();
  const int c0 = kend + tt * TN;
  const int col = c0 + (tid >> 3), row = r0 + 16 * (tid & 7);
  if (col < ncols && row < n) prefetch_l2(M + (size_t)col * ld + row);
  if (tid < 2 * TN) {
    const int uc = c0 + (tid >> 1), ur = k0 + 16 * (tid & 1);
    if (uc < ncols && ur < kend) prefetch_l2(M + (size_t)uc * ld + ur);
  }
}

// L2 prefetch of the L21 rows r0..r0+127 of panel columns k0..k0+31 (one line per thread).
__device__ __forceinline__ void prefetch_L(const float2* M, size_t ld, int n, int k0, int kend, int r0) {
  const int tid = lucore::gtid();
  const int col = k0 + (tid >> 3), row = r0 + 16 * (tid & 7);
  if (col < kend && row < n) prefetch_l2(M + (size_t)col * ld + row);
}

// A22 -= L21 U12 for the panel k0..k0+kb-1 on the tensor cores. All threads of
// the group call it; it returns with the group synchronised and no MMA in
// flight, unless a wait ran out (then *cx.bad is set and the rest of the
// panel's update is skipped).
__device__ inline void update(float2* __restrict__ M, int n, int ncols, int k0, int kb, Ctx& cx) {
  const int tid = lucore::gtid(), warp = tid >> 5, lane = tid & 31;
  const size_t ld = (size_t)n;
  const int kend = k0 + kb;
  const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32*quad.., tile columns 16*half..
  const uint32_t lane_base = cx.tmem + ((uint32_t)(32 * quad) << 16);
  unsigned char* bset0 = cx.stage + 4 * A_BYTES;
  const int T = (ncols - kend + TN - 1) / TN;  // column tiles of a row block
  for (int r0 = kend; r0 < n; r0 += TM) {
    stage_L(M, ld, n, r0, k0, kb, cx.stage);
    stage_U(M, ld, ncols, kend, k0, kb, bset0);
    stage_barrier();
    if (tid == 0) issue_tile(cx, 0);
    const int row = r0 + 32 * quad + lane;
    for (int t = 0; t < T; ++t) {
      const int b = t & 1;
      const int c0 = kend + t * TN;
      // the lines of the tile two steps ahead (in this row block or the next) into L2
      if (t + 2 < T) prefetch_tile(M, ld, n, ncols, k0, kend, r0, t + 2);
      else if (r0 + TM < n && t + 2 - T < T) prefetch_tile(M, ld, n, ncols, k0, kend, r0 + TM, t + 2 - T);
      if (t + 3 == T && r0 + TM < n) prefetch_L(M, ld, n, k0, kend, r0 + TM);
      // this tile's C values, loaded while its MMAs run; issued first, so that their
      // latency overlaps that of the U12 loads below
      float2 cv[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = c0 + 16 * half + c;
        cv[c] = (row < n && col < ncols) ? M[(size_t)col * ld + row] : make_float2(0.f, 0.f);
      }
      // operands of tile t+1: its U12 set was last read by tile t-1's MMAs, complete
      if (t + 1 < T) stage_U(M, ld, ncols, c0 + TN, k0, kb, bset0 + (b ^ 1) * B_SET);
      const bool ok = wait_parity(cx.mbar + b, cx.phase[b], cx.wait_cycles);
      cx.phase[b] ^= 1u;
      if (!ok) atomicExch(cx.bad, 1);
      stage_barrier();  // tile t+1 staged; tile t-1's accumulator read by every thread
      if (*cx.bad) return;
      if (t + 1 < T && tid == 0) issue_tile(cx, b ^ 1);
      float re[16], im[16];
      const uint32_t acc = lane_base + (uint32_t)b * ACC_COLS;
      tmem_ld_pair(acc + (uint32_t)(16 * half), acc + (uint32_t)(TN + 16 * half), re, im);
      if (row < n) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = c0 + 16 * half + c;
          if (col < ncols) M[(size_t)col * ld + row] = make_float2(cv[c].x - re[c], cv[c].y - im[c]);
        }
      }
      fence_before();  // this accumulator read is ordered before the next barrier
    }
    lucore::gsync();  // every epilogue store of the row block done before the next staging
  }
}

}  // namespace tcu
