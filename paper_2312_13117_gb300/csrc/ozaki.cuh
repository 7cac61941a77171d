// FP64-accurate products of the refinement residual on the tensor cores.
//
// The precision form refines every node solve with residuals
// R = V - T(z_j) X = V - id X - sum_d f_d(z_j) A_d X (Eq. 2.4 solved to FP64
// accuracy). GB300's FP64 pipe issues 2 DFMA per SM per clock, so these
// products are formed instead from exact integer pieces on the BF16 tensor
// cores, in the manner of the error-free splitting of Ozaki, Ogita, Oishi and
// Rump (Numer. Algorithms 59, 2012):
//
//   * every row i of a coefficient A_d is scaled by 2^-e_i (e_i: the smallest
//     exponent with max_j max(|Re a_ij|, |Im a_ij|) <= 2^e_i), rounded to the
//     integer N = rint(a 2^(48 - e_i)) and written as S = 7 balanced base-128
//     digits, a^(1..7) in [-64, 64]; every column c of Y = f_d X likewise with
//     its own exponent g_c. Digits are exact BF16 values;
//   * a y ~ 2^(e_i + g_c - 96) sum_{s,t} a^(s) y^(t) 2^(7 (14 - s - t)); the
//     pairs with s + t <= QMAX = 9 are kept (34 of 49; the dropped ones are
//     below 2^-53 of |a||y| each), grouped by q = s + t into one TMEM
//     accumulator each (8 x 32 columns);
//   * a product of two digits is an integer of magnitude <= 2^12 and a group
//     holds at most 7 pairs, so over K = 256 inner indices and the two real
//     products of a complex one every partial sum is an integer below 2^24:
//     the FP32 accumulation of the tensor cores is exact. After every 256
//     inner indices the 8 accumulators are read (tcgen05.ld) and combined by
//     Horner's rule, H = sum_q acc_q 2^(7 (9 - q)), in double-float FP32
//     arithmetic (Dekker/Knuth error-free sums, about 48 bits), and the scaled
//     result is subtracted from R in FP64.
//
// Complex products use N = 32 accumulator columns: D = [Re | Im] of
// A Y = Ar [Yr | Yi] + Ai [-Yi | Yr], two MMAs (M = 128, N = 32, K = 16) per
// digit pair and K-step. Operands are K-major in the canonical no-swizzle
// layout (8-row x 16-byte core matrices; LBO 128 B along K, SBO 512 B between
// 8-row groups, 32 K values per tile row), pre-arranged in global memory so
// that every stage is one contiguous bulk copy: coefficient digits once per
// problem, Y digits per node and sweep into a per-slot scratch.
//
// One thread of the calling group issues the bulk copies (cp.async.bulk with
// mbarrier completion) and the MMAs; the whole group drains the accumulators.
// Every wait is bounded; a wait that runs out makes the call return false
// after the copies and products in flight have completed (bounded again).
#pragma once
#include <cstdint>

#include "tc_update.cuh"

namespace ozk {

constexpr int THREADS_PER_GROUP = lucore::THREADS;
constexpr int S = 7;                  // digits per operand
constexpr int QMAX = 9;               // digit pairs with s + t <= QMAX are multiplied
constexpr int NQ = QMAX - 1;          // accumulators, q = 2..QMAX
constexpr int TM = 128;               // MMA M: rows of a block, TMEM lanes
constexpr int TN = 32;                // MMA N: 16 real + 16 imaginary columns
constexpr int LC = 16;                // solution columns per column block
constexpr int KC = 32;                // inner indices per stage
constexpr int KD = 256;               // inner indices between drains
constexpr int A_TILE = TM * KC * 2;   // one part (re or im) of one digit of a 128 x 32 block: 8 KB
constexpr int B_TILE = TN * KC * 2;   // [Yr|Yi] or [-Yi|Yr] of one digit, 32 inner indices: 2 KB
constexpr int A_STAGE = 2 * A_TILE;   // re and im of digit s: 16 KB
constexpr int B_STAGE = 2 * S * B_TILE;  // both operands of every digit t: 28 KB
constexpr int NA = 3;                 // A stages in the ring
constexpr int NBUF = 2;               // B stages in the ring
constexpr uint32_t TMEM_COLS = NQ * TN;  // 256
constexpr int DIGIT_SHIFT = 48;       // N = rint(x 2^(48 - exponent)), |N| <= 2^48
constexpr int DRAIN_SCALE = 61;       // H 2^(e + g - 61) is the block's product (96 - 35)

// exactness of the FP32 accumulation (pairs per group x 2 real products x KD x 64^2)
static_assert(7 * 2 * KD * 64 * 64 < (1 << 24), "tensor-core partial sums must stay exact in FP32");
static_assert(KD % KC == 0, "drains fall on stage boundaries");

struct Smem {
  alignas(1024) unsigned char a[NA][A_STAGE];
  alignas(1024) unsigned char b[NBUF][B_STAGE];
};

// Barriers and ring counters; they live outside any union and keep their phases
// from call to call.
struct Bars {
  uint64_t a_full[NA], a_empty[NA], b_full[NBUF], b_empty[NBUF], acc;
  uint32_t a_issue, a_use, b_issue, b_use, acc_n;
  int bad;  // a wait ran out: the products are abandoned for good in this CTA
};

__device__ __forceinline__ void init_bars(Bars& b) {
  for (int i = 0; i < NA; ++i) {
    tcu::mbar_init(&b.a_full[i]);
    tcu::mbar_init(&b.a_empty[i]);
  }
  for (int i = 0; i < NBUF; ++i) {
    tcu::mbar_init(&b.b_full[i]);
    tcu::mbar_init(&b.b_empty[i]);
  }
  tcu::mbar_init(&b.acc);
  b.a_issue = b.a_use = b.b_issue = b.b_use = b.acc_n = 0;
  b.bad = 0;
}

// Shared-memory descriptor of a BF16 K-major tile with 32 inner indices per row.
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, K-major, N = 32, M = 128.
__device__ __forceinline__ uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(da), "l"(db), "r"(id), "r"(acc));
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tcu::smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completing on the barrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tcu::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(tcu::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// One 8-column load of this warp's 32 TMEM lanes and the wait for it.
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

// Exponent e with |x| <= 2^e for the largest |x| m >= 0 (0 for m = 0).
__device__ __forceinline__ int exponent_of(double m) {
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// Digit t (0 = most significant) when the digits are taken from the least
// significant end: for t > 0 the balanced remainder of N modulo 128 (N becomes
// the quotient), for t = 0 what is left of N.
__device__ __forceinline__ int next_digit(long long& N, int t) {
  if (t == 0) return (int)N;
  const long long d = ((N + 64) & 127) - 64;
  N = (N - d) >> 7;
  return (int)d;
}

// BF16 bits of a small integer (|v| <= 256 has at most 8 significant bits, so the
// upper half of its FP32 representation is exact).
__device__ __forceinline__ uint16_t bf16_of_int(int v) { return (uint16_t)(__float_as_uint((float)v) >> 16); }

// Byte offset of element (row r, inner index k) in a K-major tile of 32 inner indices.
__device__ __forceinline__ int tile_off(int r, int k) { return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// ---- double-float arithmetic (Dekker 1971; Knuth's TwoSum) -----------------
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_add_f(DF a, float b) {  // a + b, b exact
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b - bb);
  const float lo = a.lo + e;
  const float h = s + lo;
  return DF{h, lo - (h - s)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = a.lo + b.lo + e;
  const float h = s + lo;
  return DF{h, lo - (h - s)};
}

// Number of column blocks and stage counts of a problem of order n.
__host__ __device__ inline int row_blocks(int n) { return (n + TM - 1) / TM; }
__host__ __device__ inline int k_chunks(int n) { return (n + KC - 1) / KC; }
// Bytes of the coefficient digits of n_dense terms, and of one slot's Y digits.
__host__ __device__ inline size_t coeff_digit_bytes(int n, int n_dense) {
  return (size_t)n_dense * row_blocks(n) * k_chunks(n) * S * (size_t)A_STAGE;
}
__host__ __device__ inline size_t y_digit_bytes(int n, int n_dense) {
  return (size_t)n_dense * k_chunks(n) * (size_t)B_STAGE;
}

// ---------------------------------------------------------------------------
// Group routines (one group of lucore::THREADS = 256 threads)
// ---------------------------------------------------------------------------

// Digits of the block Y = f X[:, c0 .. c0 + 15] (X n x l, column-major) into the
// tiles [kc][t][form] at dst (form 0 = [Yr | Yi], 1 = [-Yi | Yr]); the column
// exponents into g[16]. Rows >= n and columns >= l are zero. red: 256 doubles.
__device__ inline void y_digits(const double2* __restrict__ X, int n, int l, int c0, double2 f,
                         unsigned char* __restrict__ dst, int* g, double* red) {
  const int tid = lucore::gtid();
  {
    const int c = tid & (LC - 1), r0 = tid >> 4;
    double m = 0.0;
    if (c0 + c < l) {
      const double2* xc = X + (size_t)(c0 + c) * n;
      for (int j = r0; j < n; j += THREADS_PER_GROUP / LC) {
        const double2 y = cmul(f, xc[j]);
        m = fmax(m, fmax(fabs(y.x), fabs(y.y)));
      }
    }
    red[tid] = m;
    lucore::gsync();
    if (tid < LC) {
      double mm = 0.0;
      for (int k = 0; k < THREADS_PER_GROUP / LC; ++k) mm = fmax(mm, red[tid + LC * k]);
      g[tid] = exponent_of(mm);
    }
    lucore::gsync();
  }
  const int rows = k_chunks(n) * KC;
  const int tasks = LC * (rows / 8);
  for (int task = tid; task < tasks; task += THREADS_PER_GROUP) {
    const int c = task & (LC - 1), j0 = (task >> 4) * 8;
    const int kc = j0 / KC, k0 = j0 % KC;
    const bool col_ok = c0 + c < l;
    const int e = g[c];
    long long Nr[8], Ni[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u;
      double2 y = make_double2(0.0, 0.0);
      if (col_ok && j < n) y = cmul(f, X[(size_t)(c0 + c) * n + j]);
      Nr[u] = __double2ll_rn(scalbn(y.x, DIGIT_SHIFT - e));
      Ni[u] = __double2ll_rn(scalbn(y.y, DIGIT_SHIFT - e));
    }
    unsigned char* tiles = dst + (size_t)kc * B_STAGE;
    const int off_lo = tile_off(c, k0), off_hi = tile_off(LC + c, k0);
#pragma unroll 1
    for (int t = S - 1; t >= 0; --t) {
      uint32_t pr[4], pi[4], nr[4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const int dr0 = next_digit(Nr[u], t), dr1 = next_digit(Nr[u + 1], t);
        const int di0 = next_digit(Ni[u], t), di1 = next_digit(Ni[u + 1], t);
        pr[u / 2] = (uint32_t)bf16_of_int(dr0) | ((uint32_t)bf16_of_int(dr1) << 16);
        pi[u / 2] = (uint32_t)bf16_of_int(di0) | ((uint32_t)bf16_of_int(di1) << 16);
        nr[u / 2] = (uint32_t)bf16_of_int(-di0) | ((uint32_t)bf16_of_int(-di1) << 16);
      }
      unsigned char* b0 = tiles + (size_t)(t * 2 + 0) * B_TILE;  // [Yr | Yi]
      unsigned char* b1 = tiles + (size_t)(t * 2 + 1) * B_TILE;  // [-Yi | Yr]
      *reinterpret_cast<uint4*>(b0 + off_lo) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(b0 + off_hi) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
      *reinterpret_cast<uint4*>(b1 + off_lo) = make_uint4(nr[0], nr[1], nr[2], nr[3]);
      *reinterpret_cast<uint4*>(b1 + off_hi) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
    }
  }
}

// The issuing thread's view of one product sequence (row block rb, term d):
// A stages u = kc S + s, B stages kc.
struct Seq {
  const unsigned char* a_src;  // digits of (d, rb): KCN * S stages of A_STAGE bytes
  const unsigned char* b_src;  // Y digits of d: KCN stages of B_STAGE bytes
  int n_a, n_b;                // stages in the sequence
  int next_a, next_b;          // next stage to copy
};

__device__ __forceinline__ bool issue_a(Smem& st, Bars& bb, Seq& q, long long limit) {
  const uint32_t buf = bb.a_issue % NA, k = bb.a_issue / NA;
  if (k > 0 && !tcu::wait_parity(&bb.a_empty[buf], (k - 1) & 1u, limit)) return false;
  expect_tx(&bb.a_full[buf], A_STAGE);
  bulk_g2s(st.a[buf], q.a_src + (size_t)q.next_a * A_STAGE, A_STAGE, &bb.a_full[buf]);
  ++bb.a_issue;
  ++q.next_a;
  return true;
}

__device__ __forceinline__ bool issue_b(Smem& st, Bars& bb, Seq& q, long long limit) {
  const uint32_t buf = bb.b_issue % NBUF, k = bb.b_issue / NBUF;
  if (k > 0 && !tcu::wait_parity(&bb.b_empty[buf], (k - 1) & 1u, limit)) return false;
  expect_tx(&bb.b_full[buf], B_STAGE);
  bulk_g2s(st.b[buf], q.b_src + (size_t)q.next_b * B_STAGE, B_STAGE, &bb.b_full[buf]);
  ++bb.b_issue;
  ++q.next_b;
  return true;
}

// Issuing thread: the MMAs of stages [u0, u1) of the sequence (with the copies of
// later stages kept in flight), then one commit to bb.acc. On a wait that runs
// out it stops issuing, sets bb.bad and still commits.
__device__ inline void issue_block(Smem& st, Bars& bb, Seq& q, uint32_t tmem, int u0, int u1, long long limit) {
  const uint32_t id = idesc();
  uint32_t used = 0;  // accumulators written since the last drain
  for (int u = u0; u < u1 && !bb.bad; ++u) {
    const int s = u % S;
    if (s == 0 && !tcu::wait_parity(&bb.b_full[bb.b_use % NBUF], (bb.b_use / NBUF) & 1u, limit)) {
      bb.bad = 1;
      break;
    }
    if (!tcu::wait_parity(&bb.a_full[bb.a_use % NA], (bb.a_use / NA) & 1u, limit)) {
      bb.bad = 1;
      break;
    }
    tcu::fence_after();
    const uint32_t ab = tcu::smem_u32(st.a[bb.a_use % NA]), bbase = tcu::smem_u32(st.b[bb.b_use % NBUF]);
    for (int t = 0; t + s + 2 <= QMAX && t < S; ++t) {
      const int qi = s + t;  // q - 2
      const uint32_t d = tmem + (uint32_t)(qi * TN);
      const uint32_t b0 = bbase + (uint32_t)((t * 2 + 0) * B_TILE), b1 = bbase + (uint32_t)((t * 2 + 1) * B_TILE);
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        const uint32_t o = (uint32_t)(ks * 256);  // 16 BF16 = two core matrices along K
        mma(d, desc(ab + o), desc(b0 + o), id, (used >> qi) & 1u);
        mma(d, desc(ab + A_TILE + o), desc(b1 + o), id, 1u);
        used |= 1u << qi;
      }
    }
    tcu::commit(&bb.a_empty[bb.a_use % NA]);
    ++bb.a_use;
    if (q.next_a < q.n_a && !issue_a(st, bb, q, limit)) {
      bb.bad = 1;
      break;
    }
    if (s == 0 && q.next_b < q.n_b && !issue_b(st, bb, q, limit)) {
      bb.bad = 1;
      break;
    }
    if (s == S - 1) {
      tcu::commit(&bb.b_empty[bb.b_use % NBUF]);
      ++bb.b_use;
    }
  }
  tcu::commit(&bb.acc);
}

// After a wait ran out: let every issued copy land and the products committed
// last complete (each wait bounded by the default limit, whatever the caller's),
// so that nothing asynchronous touches shared or tensor memory after the caller
// reuses it.
__device__ inline void settle(Bars& bb, uint32_t acc_n) {
  while (bb.a_use < bb.a_issue) {
    tcu::wait_parity(&bb.a_full[bb.a_use % NA], (bb.a_use / NA) & 1u, tcu::WAIT_CYCLES);
    ++bb.a_use;
  }
  while (bb.b_use < bb.b_issue) {
    tcu::wait_parity(&bb.b_full[bb.b_use % NBUF], (bb.b_use / NBUF) & 1u, tcu::WAIT_CYCLES);
    ++bb.b_use;
  }
  if (acc_n > 0) tcu::wait_parity(&bb.acc, (acc_n - 1) & 1u, tcu::WAIT_CYCLES);
}

// R = V - id X - sum_d f_d A_d X for one node solution X (n x l, column-major,
// global), R (the same layout) written in FP64. fz: f_k(z_j) per term; ysl: the
// slot's Y-digit scratch; tmem: TMEM_COLS accumulator columns; g: LC * terms
// ints and red: 256 doubles of shared memory. Every thread of the group calls it;
// returns false (the same in every thread) when a wait ran out.
__device__ inline bool residual(const ProblemDev& P, const double2* fz, const double2* __restrict__ X,
                         double2* __restrict__ R, Smem& st, Bars& bb, unsigned char* ysl, uint32_t tmem, int* g,
                         double* red, long long limit) {
  const int tid = lucore::gtid(), warp = tid >> 5, lane = tid & 31;
  const int n = P.n, l = P.l;
  const int RB = row_blocks(n), KCN = k_chunks(n);
  double2 id = make_double2(0.0, 0.0);
  for (int k = 0; k < P.K; ++k)
    if (!P.term[k].dense) id = cadd(id, cmul(fz[k], P.term[k].id));
  for (size_t e = tid; e < (size_t)n * l; e += THREADS_PER_GROUP) {
    double2 v = P.V[e];
    cfms(v, id, X[e]);
    R[e] = v;
  }
  const int quad = warp & 3, half = warp >> 2;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(16 * half);
  uint32_t acc_n = bb.acc_n;
  bool ok = !bb.bad;
  for (int c0 = 0; c0 < l && ok; c0 += LC) {
    // Y digits of every dense term for this column block
    int dd = 0;
    for (int k = 0; k < P.K; ++k) {
      if (!P.term[k].dense) continue;
      y_digits(X, n, l, c0, fz[k], ysl + (size_t)dd * KCN * B_STAGE, g + LC * dd, red);
      ++dd;
    }
    fence_proxy_async_all();  // the digits written above are read by bulk copies
    lucore::gsync();
    for (int rb = 0; rb < RB && ok; ++rb) {
      const int row = rb * TM + 32 * quad + lane;
      dd = 0;
      for (int k = 0; k < P.K && ok; ++k) {
        if (!P.term[k].dense) continue;
        Seq q;
        q.a_src = P.Adig + ((size_t)P.term[k].mat_index * RB + rb) * KCN * S * A_STAGE;
        q.b_src = ysl + (size_t)dd * KCN * B_STAGE;
        q.n_a = KCN * S;
        q.n_b = KCN;
        q.next_a = 0;
        q.next_b = 0;
        if (tid == 0) {
          for (int i = 0; i < NA - 1 && q.next_a < q.n_a && !bb.bad; ++i)
            if (!issue_a(st, bb, q, limit)) bb.bad = 1;
          if (!bb.bad && !issue_b(st, bb, q, limit)) bb.bad = 1;
        }
        const int er = row < n ? P.Aexp[(size_t)P.term[k].mat_index * RB * TM + row] : 0;
        for (int kc0 = 0; kc0 < KCN; kc0 += KD / KC) {
          const int kc1 = min(KCN, kc0 + KD / KC);
          if (tid == 0) issue_block(st, bb, q, tmem, kc0 * S, kc1 * S, limit);
          lucore::gsync();  // the block's products are issued and committed
          const bool done = tcu::wait_parity(&bb.acc, acc_n & 1u, limit);
          ++acc_n;
          if (!lucore::group_all_sync(done && !bb.bad)) {
            ok = false;
            break;
          }
          tcu::fence_after();
          __syncwarp();
          // Horner's rule over the accumulators, q = 2 .. QMAX, in double-float,
          // eight columns at a time; the block's product leaves R in FP64
#pragma unroll 1
          for (int c8 = 0; c8 < LC; c8 += 8) {
            DF H[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) H[c] = DF{0.f, 0.f};
#pragma unroll 1
            for (int qi = 0; qi < NQ; ++qi) {
              float v[8];
              tmem_ld8(lane_base + (uint32_t)(qi * TN + c8), v);
#pragma unroll
              for (int c = 0; c < 8; ++c) H[c] = df_add_f(DF{H[c].hi * 128.f, H[c].lo * 128.f}, v[c]);
            }
            if (row < n) {
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                const int col = c0 + c8 + c;
                if (col < l) {
                  const double sc = scalbn(1.0, er + g[LC * dd + c8 + c] - DRAIN_SCALE);
                  double* r = reinterpret_cast<double*>(R + (size_t)col * n + row) + half;
                  *r = fma(-sc, (double)H[c].hi, fma(-sc, (double)H[c].lo, *r));
                }
              }
            }
          }
          tcu::fence_before();
          lucore::gsync();  // every accumulator is read before the next block's products
        }
        ++dd;
      }
    }
  }
  if (tid == 0) {
    if (!ok) settle(bb, acc_n);
    bb.acc_n = acc_n;
  }
  lucore::gsync();
  return ok;
}

}  // namespace ozk
