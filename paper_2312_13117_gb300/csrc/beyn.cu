// Beyn's extraction on the device, FP64 (Eq. 2.8; pmCIMb steps 2.c-2.f).
//
// One CTA per disk of a level; disks the indicator gate rules out return at once:
//   1. one-sided (Hestenes) Jacobi SVD of C0 (n x l): columns of C0 W are
//      orthogonalised by complex plane rotations; sigma_k are their norms,
//      sorted descending; V0 = normalised columns, W0 = W's columns;
//   2. p = #{sigma_k > tol_svd} (absolute threshold, Sec. 3.2);
//   3. D = V0^H C1 W0 Sigma0^{-1} (p x p);
//   4. eig(D): Householder reduction to Hessenberg form, then single-shift
//      complex QR with Wilkinson shifts and deflation to Schur form T = Z^H D Z;
//      eigenvectors of T by back substitution, s = Z y;
//   5. eigenvectors v = V0 s, unit 2-norm, largest-modulus entry real positive;
//   6. square filter: keep c - h <= Re, Im < c + h with h = r / sqrt(2).
// Steps 1, 3 and 5 are spread over the CTA; step 4 (p <= 64) runs on one thread.
// With K > 1 moment pairs the same steps run on the block Hankel matrices of the
// scaled moments M_p (reduce.cu): C0 -> B0 = [M_{i+j}], C1 -> B1 = [M_{i+j+1}]
// (i, j < K; K n x K l); eig(D) then gives mu = (lambda - c) / r, and an
// eigenvector is the first n-block of V0 s (B0's left factor has block rows
// v, v mu, ..., v mu^{K-1}).
#include "pmcim_internal.cuh"

namespace {

constexpr int BT = 256;
constexpr double EPS = 2.220446049250313e-16;

struct BeynSmem {
  int rotated;  // a Jacobi rotation happened in this sweep
  double red[4][BT / 32];
  int red_i[BT / 32];
  double sig[PMCIM_MAX_L];
  int perm[PMCIM_MAX_L];
  double2 lam[PMCIM_MAX_L];
  double2 gc_s[PMCIM_MAX_L];  // Givens s of one QR sweep
  double gc_c[PMCIM_MAX_L];   // Givens c
  double bcast[4];
  int flag;
  int p;
  int status;
};

__device__ __forceinline__ void block_sum4(double v[4], BeynSmem& sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) sm.red[q][wid] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double t = 0.0;
    for (int k = 0; k < BT / 32; ++k) t += sm.red[q][k];
    v[q] = t;
  }
}

// principal complex square root
__device__ double2 csqrt_(double2 z) {
  double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  double a = sqrt(0.5 * (r + fabs(z.x)));
  double b = 0.5 * z.y / a;
  if (z.x >= 0.0) return make_double2(a, b);
  return make_double2(fabs(b), copysign(a, z.y));
}

// ---------------------------------------------------------------------------
// Single-thread dense complex eigen-solver for small p (column-major, ld = p).
// H is overwritten by the Schur form, Z by the Schur vectors, Y by the
// eigenvectors of the input (columns, unnormalised). Returns 0 or 1 when the
// QR iteration hit its limit.
// ---------------------------------------------------------------------------
__device__ int small_eig(double2* H, double2* Z, double2* Y, int p, double2* lam, BeynSmem& sm) {
#define Hm(i, j) H[(size_t)(j) * p + (i)]
#define Zm(i, j) Z[(size_t)(j) * p + (i)]
#define Ym(i, j) Y[(size_t)(j) * p + (i)]
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) Zm(i, j) = make_double2(i == j ? 1.0 : 0.0, 0.0);
  double hnorm = 0.0;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) hnorm = fmax(hnorm, l1abs(Hm(i, j)));

  // Householder reduction to upper Hessenberg form
  for (int k = 0; k + 2 < p; ++k) {
    double xn2 = 0.0;
    for (int i = k + 1; i < p; ++i) xn2 += cabs2(Hm(i, k));
    const double xn = sqrt(xn2);
    if (xn == 0.0) continue;
    const double2 x0 = Hm(k + 1, k);
    const double ax0 = hypot(x0.x, x0.y);
    const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
    const double2 alpha = cscale(ph, -xn);  // H[k+1,k] becomes alpha
    // v = x - alpha e1, stored in lam[] temporarily (p <= 64)
    double2* v = sm.gc_s;
    double vn2 = 0.0;
    for (int i = k + 1; i < p; ++i) {
      double2 vi = Hm(i, k);
      if (i == k + 1) vi = csub(vi, alpha);
      v[i] = vi;
      vn2 += cabs2(vi);
    }
    if (vn2 == 0.0) continue;
    const double inv = 1.0 / sqrt(vn2);
    for (int i = k + 1; i < p; ++i) v[i] = cscale(v[i], inv);
    // left: H[k+1:, k:] -= 2 v (v^H H[k+1:, k:])
    for (int j = k; j < p; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = k + 1; i < p; ++i) cfma_conj(s, v[i], Hm(i, j));
      s = cscale(s, 2.0);
      for (int i = k + 1; i < p; ++i) cfms(Hm(i, j), v[i], s);
    }
    // right: H[:, k+1:] -= 2 (H[:, k+1:] v) v^H, same for Z
    for (int i = 0; i < p; ++i) {
      double2 s = make_double2(0.0, 0.0), t = s;
      for (int j = k + 1; j < p; ++j) { cfma(s, Hm(i, j), v[j]); cfma(t, Zm(i, j), v[j]); }
      s = cscale(s, 2.0);
      t = cscale(t, 2.0);
      for (int j = k + 1; j < p; ++j) { cfms(Hm(i, j), s, cconj(v[j])); cfms(Zm(i, j), t, cconj(v[j])); }
    }
    for (int i = k + 2; i < p; ++i) Hm(i, k) = make_double2(0.0, 0.0);
  }

  // shifted QR iteration on the Hessenberg matrix
  int fail = 0;
  int hi = p - 1, its = 0, total = 0;
  const double small = fmax(hnorm, 1e-300) * EPS;
  while (hi > 0) {
    int lo = hi;
    for (; lo > 0; --lo) {
      double s = l1abs(Hm(lo - 1, lo - 1)) + l1abs(Hm(lo, lo));
      if (s == 0.0) s = hnorm;
      if (l1abs(Hm(lo, lo - 1)) <= EPS * s || l1abs(Hm(lo, lo - 1)) < 1e-300) {
        Hm(lo, lo - 1) = make_double2(0.0, 0.0);
        break;
      }
    }
    if (lo == hi) { --hi; its = 0; continue; }
    if (total > 60 * p) { fail = 1; break; }
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to H[hi,hi]
    const double2 a = Hm(hi - 1, hi - 1), b = Hm(hi - 1, hi), c = Hm(hi, hi - 1), d = Hm(hi, hi);
    double2 mu;
    if (its > 0 && its % 10 == 0) {
      mu = cadd(d, make_double2(1.5 * l1abs(c), 0.0));  // exceptional shift
    } else {
      const double2 m = cscale(cadd(a, d), 0.5);
      const double2 hdif = cscale(csub(a, d), 0.5);
      const double2 disc = csqrt_(cadd(cmul(hdif, hdif), cmul(b, c)));
      const double2 m1 = cadd(m, disc), m2 = csub(m, disc);
      mu = (cabs2(csub(m1, d)) <= cabs2(csub(m2, d))) ? m1 : m2;
    }
    // explicit shifted QR step on rows/cols lo..hi: H - mu I = G^H R, H <- R G^H + mu I
    for (int k = lo; k <= hi; ++k) Hm(k, k) = csub(Hm(k, k), mu);
    for (int k = lo; k < hi; ++k) {
      const double2 x = Hm(k, k), y = Hm(k + 1, k);
      const double ax = hypot(x.x, x.y), ay = hypot(y.x, y.y);
      const double rr = hypot(ax, ay);
      double cc;
      double2 ss;
      if (rr == 0.0) { cc = 1.0; ss = make_double2(0.0, 0.0); }
      else if (ax == 0.0) { cc = 0.0; ss = make_double2(y.x / ay, -y.y / ay); }
      else {
        cc = ax / rr;
        const double2 ph = make_double2(x.x / ax, x.y / ax);
        ss = cscale(cmul(ph, cconj(y)), 1.0 / rr);
      }
      sm.gc_c[k] = cc;
      sm.gc_s[k] = ss;
      for (int j = k; j < p; ++j) {
        const double2 u = Hm(k, j), w = Hm(k + 1, j);
        Hm(k, j) = cadd(cscale(u, cc), cmul(ss, w));
        Hm(k + 1, j) = csub(cscale(w, cc), cmul(cconj(ss), u));
      }
      Hm(k + 1, k) = make_double2(0.0, 0.0);
    }
    for (int k = lo; k < hi; ++k) {
      const double cc = sm.gc_c[k];
      const double2 ss = sm.gc_s[k];
      const int rmax = min(k + 2, hi);
      for (int i = 0; i <= rmax; ++i) {
        const double2 u = Hm(i, k), w = Hm(i, k + 1);
        Hm(i, k) = cadd(cscale(u, cc), cmul(cconj(ss), w));
        Hm(i, k + 1) = csub(cscale(w, cc), cmul(ss, u));
      }
      for (int i = 0; i < p; ++i) {
        const double2 u = Zm(i, k), w = Zm(i, k + 1);
        Zm(i, k) = cadd(cscale(u, cc), cmul(cconj(ss), w));
        Zm(i, k + 1) = csub(cscale(w, cc), cmul(ss, u));
      }
    }
    for (int k = lo; k <= hi; ++k) Hm(k, k) = cadd(Hm(k, k), mu);
    ++its;
    ++total;
  }
  for (int k = 0; k < p; ++k) lam[k] = Hm(k, k);

  // eigenvectors of the triangular T, then Y = Z y
  for (int k = 0; k < p; ++k) {
    double2* yk = sm.gc_s;  // scratch p-vector
    for (int i = 0; i < p; ++i) yk[i] = make_double2(0.0, 0.0);
    yk[k] = make_double2(1.0, 0.0);
    const double2 tk = Hm(k, k);
    for (int i = k - 1; i >= 0; --i) {
      double2 s = make_double2(0.0, 0.0);
      for (int m = i + 1; m <= k; ++m) cfma(s, Hm(i, m), yk[m]);
      double2 den = csub(Hm(i, i), tk);
      if (l1abs(den) < small) den = make_double2(small, 0.0);
      yk[i] = cdiv(make_double2(-s.x, -s.y), den);
    }
    for (int i = 0; i < p; ++i) {
      double2 s = make_double2(0.0, 0.0);
      for (int m = 0; m <= k; ++m) cfma(s, Zm(i, m), yk[m]);
      Ym(i, k) = s;
    }
  }
#undef Hm
#undef Zm
#undef Ym
  return fail;
}

__global__ void __launch_bounds__(BT, 1) k_beyn(LevelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BeynSmem& sm = *reinterpret_cast<BeynSmem*>(smem_raw);
  const int g = blockIdx.x;
  const int tid = threadIdx.x;
  const RegionDev rg = a.regions[g];
  const size_t ol = (size_t)g * PMCIM_MAX_L;  // per-disk slot of sigma, lam, kept
  if (rg.gate && !a.cand[g]) {                // gated out: no Beyn step for this disk
    if (tid == 0) {
      a.p[g] = -1;
      a.status[g] = 0;
    }
    return;
  }
  const int nv = a.probs[rg.prob].n, lp = a.probs[rg.prob].l;  // eigenvector length, probes
  const int K = a.K;
  const int n = K * nv, l = K * lp;  // rows and columns of the matrix the SVD runs on
  const size_t nl = (size_t)n * l;
  // per-disk scratch: Acol (n x l) | B (n x l) | W (l x l) | H | Z | Y (p x p each, p <= l),
  // then, for K > 1, B1 (n x l)
  double2* Ac = a.bwork + rg.w_off;
  double2* B = Ac + nl;
  double2* W = B + nl;
  double2* H = W + (size_t)l * l;
  double2* Z = H + (size_t)l * l;
  double2* Y = Z + (size_t)l * l;
  const double2* C1;
  if (K == 1) {
    const double2* C0 = a.C0 + rg.c_off;
    C1 = a.C1 + rg.c_off;
    for (size_t e = tid; e < nl; e += BT) Ac[e] = C0[e];
  } else {
    double2* B1 = Y + (size_t)l * l;
    const double2* Mm = a.Cm + (size_t)2 * K * rg.c_off;
    const size_t blk = (size_t)nv * lp;
    for (size_t e = tid; e < nl; e += BT) {
      const int row = (int)(e % n), col = (int)(e / n);
      const int ib = row / nv, ir = row % nv, jb = col / lp, jc = col % lp;
      Ac[e] = Mm[(size_t)(ib + jb) * blk + (size_t)jc * nv + ir];
      B1[e] = Mm[(size_t)(ib + jb + 1) * blk + (size_t)jc * nv + ir];
    }
    C1 = B1;
  }
  for (int e = tid; e < l * l; e += BT) W[e] = make_double2((e % l) == (e / l) ? 1.0 : 0.0, 0.0);
  __syncthreads();

  // ---- 1. one-sided Jacobi, round-robin ordering ----
  // The columns are paired by the circle method: l' = l rounded up to even players,
  // player 0 fixed and the others rotating, so every round holds l'/2 disjoint pairs
  // and every pair meets once per sweep. The warps take the pairs of a round in turn
  // (warp-shuffle reductions, one CTA barrier per round).
  const double tol_rot = EPS * sqrt((double)n) * 4.0;
  const int lp2 = l + (l & 1), lane = tid & 31, warp = tid >> 5;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) sm.rotated = 0;
    __syncthreads();
    for (int round = 0; round < lp2 - 1; ++round) {
      for (int k = warp; k < lp2 / 2; k += BT / 32) {
        int pc, qc;
        if (k == 0) {
          pc = 0;
          qc = round % (lp2 - 1) + 1;
        } else {
          pc = (round + k) % (lp2 - 1) + 1;
          qc = (round - k + lp2 - 1) % (lp2 - 1) + 1;
        }
        if (pc > qc) { const int t = pc; pc = qc; qc = t; }
        if (qc >= l) continue;  // the padding player
        double2* ap = Ac + (size_t)pc * n;
        double2* aq = Ac + (size_t)qc * n;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double2 x = ap[i], y = aq[i];
          v0 += cabs2(x);
          v1 += cabs2(y);
          v2 += x.x * y.x + x.y * y.y;  // conj(x) y
          v3 += x.x * y.y - x.y * y.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
          v0 += __shfl_xor_sync(0xffffffffu, v0, o);
          v1 += __shfl_xor_sync(0xffffffffu, v1, o);
          v2 += __shfl_xor_sync(0xffffffffu, v2, o);
          v3 += __shfl_xor_sync(0xffffffffu, v3, o);
        }
        const double al = v0, be = v1;
        const double gabs = hypot(v2, v3);
        if (al == 0.0 || be == 0.0 || gabs <= tol_rot * sqrt(al) * sqrt(be)) continue;
        if (lane == 0) sm.rotated = 1;
        const double zeta = (be - al) / (2.0 * gabs);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t);
        const double sn = cs * t;
        const double2 e = make_double2(v2 / gabs, v3 / gabs);  // e^{i phi}
        // a_p' = c a_p - s e^{-i phi} a_q ;  a_q' = s e^{i phi} a_p + c a_q
        const double2 sem = cscale(cconj(e), sn), sep = cscale(e, sn);
        for (int i = lane; i < n; i += 32) {
          const double2 x = ap[i], y = aq[i];
          ap[i] = csub(cscale(x, cs), cmul(sem, y));
          aq[i] = cadd(cmul(sep, x), cscale(y, cs));
        }
        double2* wp = W + (size_t)pc * l;
        double2* wq = W + (size_t)qc * l;
        for (int i = lane; i < l; i += 32) {
          const double2 x = wp[i], y = wq[i];
          wp[i] = csub(cscale(x, cs), cmul(sem, y));
          wq[i] = cadd(cmul(sep, x), cscale(y, cs));
        }
      }
      __syncthreads();
    }
    if (!sm.rotated) break;
  }

  // ---- 2. singular values, order, rank ----
  for (int k = 0; k < l; ++k) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const double2* ak = Ac + (size_t)k * n;
    for (int i = tid; i < n; i += BT) v[0] += cabs2(ak[i]);
    block_sum4(v, sm);
    if (tid == 0) sm.sig[k] = sqrt(v[0]);
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < l; ++k) sm.perm[k] = k;
    for (int k = 1; k < l; ++k) {  // stable insertion sort, descending
      int pk = sm.perm[k];
      int q = k - 1;
      while (q >= 0 && sm.sig[sm.perm[q]] < sm.sig[pk]) { sm.perm[q + 1] = sm.perm[q]; --q; }
      sm.perm[q + 1] = pk;
    }
    int p = 0;
    for (int k = 0; k < l; ++k) {
      const double s = sm.sig[sm.perm[k]];
      a.sigma[ol + k] = s;
      if (s > a.tol_svd) ++p;
    }
    sm.p = p;
    int st = 0;
    if (p >= min(n, l)) st |= PMCIM_RS_SATURATED;
    sm.status = st;
    a.p[g] = p;
  }
  __syncthreads();
  const int p = sm.p;

  // ---- 3. V0 (normalise in place), B = C1 W0, D = V0^H B Sigma0^{-1} ----
  for (int k = 0; k < p; ++k) {
    const int src = sm.perm[k];
    const double inv = 1.0 / sm.sig[src];
    const double2* ak = Ac + (size_t)src * n;
    double2* bk = B + (size_t)k * n;  // B's column k temporarily holds u_k
    for (int i = tid; i < n; i += BT) bk[i] = cscale(ak[i], inv);
  }
  __syncthreads();
  // move u_k into Ac's first p columns (ordered), then B = C1 W0
  for (int k = 0; k < p; ++k) {
    const double2* bk = B + (size_t)k * n;
    double2* ak = Ac + (size_t)k * n;
    for (int i = tid; i < n; i += BT) ak[i] = bk[i];
  }
  __syncthreads();
  for (int i = tid; i < n; i += BT) {
    for (int k = 0; k < p; ++k) {
      const double2* wk = W + (size_t)sm.perm[k] * l;
      double2 s = make_double2(0.0, 0.0);
      for (int m = 0; m < l; ++m) cfma(s, C1[(size_t)m * n + i], wk[m]);
      B[(size_t)k * n + i] = s;
    }
  }
  __syncthreads();
  {
    const int lane = tid & 31, wid = tid >> 5;
    for (int pair = wid; pair < p * p; pair += BT / 32) {
      const int r = pair % p, k = pair / p;
      const double2* ur = Ac + (size_t)r * n;
      const double2* bk = B + (size_t)k * n;
      double2 s = make_double2(0.0, 0.0);
      for (int i = lane; i < n; i += 32) cfma_conj(s, ur[i], bk[i]);
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) H[(size_t)k * p + r] = cscale(s, 1.0 / sm.sig[sm.perm[k]]);
    }
  }
  __syncthreads();

  // ---- 4. eig(D) ----
  if (tid == 0 && p > 0) {
    int fail = small_eig(H, Z, Y, p, sm.lam, sm);
    (void)fail;
    if (K > 1)  // mu = (lambda - c) / r
      for (int k = 0; k < p; ++k) sm.lam[k] = make_double2(rg.cre + rg.r * sm.lam[k].x, rg.cim + rg.r * sm.lam[k].y);
  }
  __syncthreads();

  // ---- 5. eigenvectors v = V0 s, normalised ----
  for (int k = 0; k < p; ++k) {
    double2* vk = a.vecs + rg.v_off + (size_t)k * nv;
    const double2* sk = Y + (size_t)k * p;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    double best = -1.0;
    int bi = nv;
    for (int i = tid; i < nv; i += BT) {
      double2 s = make_double2(0.0, 0.0);
      for (int m = 0; m < p; ++m) cfma(s, Ac[(size_t)m * n + i], sk[m]);
      vk[i] = s;
      v[0] += cabs2(s);
      const double mg = cabs2(s);
      if (mg > best) { best = mg; bi = i; }
    }
    // argmax of |v_i| with lowest index on ties
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    __syncthreads();
    if ((tid & 31) == 0) { sm.red[1][tid >> 5] = best; sm.red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bb = sm.red[1][0];
      int ii = sm.red_i[0];
      for (int w = 1; w < BT / 32; ++w) {
        double ob = sm.red[1][w];
        int oi = sm.red_i[w];
        if (ob > bb || (ob == bb && oi < ii)) { bb = ob; ii = oi; }
      }
      sm.flag = ii;
    }
    block_sum4(v, sm);
    const double nrm = sqrt(v[0]);
    const double2 big = vk[sm.flag];
    const double ab = hypot(big.x, big.y);
    // multiply by conj(big)/|big| / nrm
    const double2 rot = ab > 0.0 ? make_double2(big.x / (ab * nrm), -big.y / (ab * nrm))
                                 : make_double2(1.0 / nrm, 0.0);
    __syncthreads();
    for (int i = tid; i < nv; i += BT) vk[i] = cmul(vk[i], rot);
    __syncthreads();
  }

  // ---- 6. square filter and outputs ----
  if (tid == 0) {
    const double h = rg.r / sqrt(2.0);
    int kept_any = 0;
    for (int k = 0; k < l; ++k) {
      uint8_t keep = 0;
      double2 lm = make_double2(0.0, 0.0);
      if (k < p) {
        lm = sm.lam[k];
        keep = (lm.x >= rg.cre - h && lm.x < rg.cre + h && lm.y >= rg.cim - h && lm.y < rg.cim + h) ? 1 : 0;
      }
      a.lam[ol + k] = lm;
      a.kept[ol + k] = keep;
      kept_any |= keep;
    }
    int st = sm.status;
    if (!kept_any) st |= PMCIM_RS_NO_EIG;
    a.status[g] = st;
  }
}

}  // namespace

cudaError_t launch_beyn(const LevelArgs& a, cudaStream_t s) {
  if (a.R <= 0) return cudaSuccess;
  const size_t smem = sizeof(BeynSmem);
  k_beyn<<<a.R, BT, smem, s>>>(a);
  return cudaGetLastError();
}
