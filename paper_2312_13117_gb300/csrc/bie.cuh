// Boundary-integral terms: the Nystrom matrix of the 2-D Helmholtz double-layer
// operator of the scattering-pole problem (Sec. 4.2), formed entry by entry on
// the device, and the Bessel functions of complex argument it needs.
//
// K(kappa) phi(x) = 2 int_C d/dnu(y) Phi(x, y) phi(y) ds(y), Phi = (i/4) H_0^(1)(kappa |x - y|).
// With the curve x(t) sampled at t_j = 2 pi j / n (n = 2 n'), n(t) = (x2', -x1'),
// r = |x(t_i) - x(t_j)| and q = n(t_j).(x(t_i) - x(t_j)), Kress's rule for kernels
// with a logarithmic singularity (R. Kress, Linear Integral Equations, Sec. 12.3)
// gives the matrix entry
//   K_ij = h L_ij + (R_m - h log(4 sin^2(pi m / n))) L1_ij,   m = (i - j) mod n, h = 2 pi / n,
//   L  = (i kappa / 2) q H_1^(1)(kappa r) / r,   L1 = -(kappa / (2 pi)) q J_1(kappa r) / r,
//   K_jj = h n(t_j).x''(t_j) / (2 pi |x'(t_j)|^2),
//   R_m = -(2 pi / n') sum_{k=1}^{n'-1} cos(k m pi / n') / k - (pi / n'^2) cos(m pi).
// The host folds R_m - h log(4 sin^2(pi m / n)) into one table of n values.
//
// Everything here is plain arithmetic on double2 and compiles for the host too.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#if defined(__CUDACC__)
#define BIE_HD __host__ __device__ __forceinline__
// the entry is a call: inlined into the assembly loops it would raise their register
// pressure on every path, also where a problem has no boundary-integral term
#define BIE_ENTRY static __host__ __device__ __noinline__
#else
#define BIE_HD inline
#define BIE_ENTRY inline
#endif

namespace bie {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;
constexpr double kSeriesMax = 13.0;  // |w| at or below: ascending series; above: Hankel's expansion
constexpr int kSeriesTerms = 96, kAsymTerms = 64;

// The series' coefficients, made at compile time in the order the loops below would
// compute them (so the results are those of dividing in the loop), and read from the
// constant cache on the device instead of two FP64 divisions per term:
//   inv_kk1[k] = 1 / (k (k+1)),  psi2[k] = psi(k+1) + psi(k+2) = 2 (H_k - gamma) + 1/(k+1),
//   ak[k] = prod_{j=1..k} (4 - (2j-1)^2) / (8 j)  (Hankel's a_k for order 1).
struct SeriesTables {
  double inv_kk1[kSeriesTerms];
  double psi2[kSeriesTerms];
  double ak[kAsymTerms];
};
constexpr SeriesTables make_series_tables() {
  SeriesTables T{};
  double Hk = 0.0;
  T.inv_kk1[0] = 0.0;
  T.psi2[0] = 1.0 - 2.0 * kEulerGamma;
  for (int k = 1; k < kSeriesTerms; ++k) {
    T.inv_kk1[k] = 1.0 / ((double)k * (double)(k + 1));
    Hk += 1.0 / (double)k;
    T.psi2[k] = 2.0 * (Hk - kEulerGamma) + 1.0 / (double)(k + 1);
  }
  double a = 1.0;
  T.ak[0] = 1.0;
  for (int k = 1; k < kAsymTerms; ++k) {
    a *= (4.0 - (double)(2 * k - 1) * (double)(2 * k - 1)) / (8.0 * (double)k);
    T.ak[k] = a;
  }
  return T;
}
#if defined(__CUDACC__)
static __constant__ SeriesTables kSeriesDev = make_series_tables();
#endif
static const SeriesTables kSeriesHost = make_series_tables();
#if defined(__CUDA_ARCH__)
#define BIE_TABLES kSeriesDev
#else
#define BIE_TABLES kSeriesHost
#endif

BIE_HD double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
BIE_HD double2 ca(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
BIE_HD double2 cs(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
BIE_HD double2 ci(double2 a) { return make_double2(-a.y, a.x); }  // i a
BIE_HD double2 crec(double2 b) {                                    // 1 / b (Smith's scaling)
  if (fabs(b.x) >= fabs(b.y)) {
    const double t = b.y / b.x, d = b.x + b.y * t;
    return make_double2(1.0 / d, -t / d);
  }
  const double t = b.x / b.y, d = b.x * t + b.y;
  return make_double2(t / d, -1.0 / d);
}

// J_1(w) and H_1^(1)(w) for Re w > 0.
//  |w| <= 13: the ascending series J_1(w) = sum_k (-1)^k (w/2)^{2k+1} / (k! (k+1)!) and
//    Y_1(w) = -2 / (pi w) + (2/pi) log(w/2) J_1(w)
//             - (1/pi) sum_k (psi(k+1) + psi(k+2)) (-1)^k (w/2)^{2k+1} / (k! (k+1)!)
//    (DLMF 10.2.2 and 10.8.1; psi(k+1) = -gamma + H_k with H_k the harmonic number),
//    H_1^(1) = J_1 + i Y_1 (DLMF 10.4.3). Summed until a term falls below 1e-17 of the
//    largest one.
//  |w| > 13: Hankel's expansions (DLMF 10.17.5, 10.17.6)
//    H_1^(1,2)(w) ~ sqrt(2 / (pi w)) e^{+-i (w - 3 pi / 4)} sum_k (+-i)^k a_k / w^k,
//    a_k = prod_{j=1..k} (4 - (2j - 1)^2) / (k! 8^k), truncated before the smallest term
//    grows again, and J_1 = (H_1^(1) + H_1^(2)) / 2 (DLMF 10.4.4).
BIE_HD void j1_h1(double2 w, double2* J, double2* H) {
  const double aw = hypot(w.x, w.y);
  if (aw <= kSeriesMax) {
    const double2 h = cs(w, 0.5);
    const double2 hh = cm(h, h);
    const double2 u = make_double2(-hh.x, -hh.y);  // -(w/2)^2
    const SeriesTables& TB = BIE_TABLES;
    double2 t = h;                                 // k = 0 term
    double2 Js = t;
    double2 S = cs(t, TB.psi2[0]);                 // psi(1) + psi(2)
    double tmax = fabs(t.x) + fabs(t.y);
    const double au = hypot(u.x, u.y);
    for (int k = 1; k < kSeriesTerms; ++k) {
      t = cs(cm(t, u), TB.inv_kk1[k]);
      Js = ca(Js, t);
      S = ca(S, cs(t, TB.psi2[k]));
      const double at = fabs(t.x) + fabs(t.y);
      tmax = fmax(tmax, at);
      if ((double)k * (double)(k + 1) > au && at <= 1e-17 * tmax) break;
    }
    // log(w/2) = log|w/2| + i arg(w)
    const double2 lg = make_double2(log(0.5 * aw), atan2(w.y, w.x));
    const double2 iw = crec(w);
    double2 Y = cs(iw, -2.0 / kPi);
    Y = ca(Y, cs(cm(lg, Js), 2.0 / kPi));
    Y = ca(Y, cs(S, -1.0 / kPi));
    *J = Js;
    *H = ca(Js, ci(Y));
    return;
  }
  const SeriesTables& TB = BIE_TABLES;
  const double2 iw = crec(w);
  double2 p = make_double2(1.0, 0.0);   // 1 / w^k
  double2 s1 = p, s2 = p;               // sums with (+i)^k and (-i)^k
  double prev = 1.0;
  for (int k = 1; k < kAsymTerms; ++k) {
    p = cm(p, iw);
    const double2 tk = cs(p, TB.ak[k]);
    const double mag = fabs(tk.x) + fabs(tk.y);
    if (mag > prev) break;  // past the smallest term
    // (+i)^k tk and (-i)^k tk
    double2 t1, t2;
    switch (k & 3) {
      case 0: t1 = tk; t2 = tk; break;
      case 1: t1 = ci(tk); t2 = make_double2(tk.y, -tk.x); break;
      case 2: t1 = make_double2(-tk.x, -tk.y); t2 = t1; break;
      default: t1 = make_double2(tk.y, -tk.x); t2 = ci(tk); break;
    }
    s1 = ca(s1, t1);
    s2 = ca(s2, t2);
    prev = mag;
    if (mag < 1e-17) break;
  }
  // sqrt(2 / (pi w)) = sqrt(2 / pi) |w|^{-1/2} e^{-i arg(w) / 2}
  const double ph = -0.5 * atan2(w.y, w.x);
  double sp, cp;
  sincos(ph, &sp, &cp);
  const double mod = sqrt(2.0 / (kPi * aw));
  const double2 pref = make_double2(mod * cp, mod * sp);
  double so, co;
  sincos(w.x - 0.75 * kPi, &so, &co);
  const double eu = exp(-w.y), ed = exp(w.y);
  const double2 e1 = make_double2(eu * co, eu * so);   // e^{+i (w - 3 pi / 4)}
  const double2 e2 = make_double2(ed * co, -ed * so);  // e^{-i (w - 3 pi / 4)}
  const double2 h1 = cm(pref, cm(e1, s1));
  const double2 h2 = cm(pref, cm(e2, s2));
  *H = h1;
  *J = cs(ca(h1, h2), 0.5);
}

// Entry (i, j) of K_n(kappa). G: the device geometry of the term (n >= 4, even),
//   G[5 j + 0..4] = x1, x2, n1 = x2', n2 = -x1', d = n.x'' / (2 pi |x'|^2) at t_j,
//   G[5 n + m]    = R_m - (2 pi / n) log(4 sin^2(pi m / n))  (m = 1..n-1; m = 0 unused),
//   G[6 n]        = 1 when the sampled curve is invariant under the shift j -> j + 1 (a
//                   circle), so that K_n is circulant: K_ij = K_{(i-j) mod n, 0}; else 0.
BIE_ENTRY double2 dlp_entry(const double* G, int n, int i, int j, double2 kappa) {
  const double h = 2.0 * kPi / (double)n;
  const double* pj = G + 5 * (size_t)j;
  if (i == j) return make_double2(h * pj[4], 0.0);
  const double* pi_ = G + 5 * (size_t)i;
  const double ex = pi_[0] - pj[0], ey = pi_[1] - pj[1];
  const double r = hypot(ex, ey);
  const double qr = (pj[2] * ex + pj[3] * ey) / r;  // n(t_j).(x_i - x_j) / r
  double2 J1, H1;
  j1_h1(cs(kappa, r), &J1, &H1);
  const double2 kq = cs(kappa, qr);
  const double2 L = ci(cs(cm(kq, H1), 0.5));             // (i kappa / 2) q H_1 / r
  const double2 L1 = cs(cm(kq, J1), -1.0 / (2.0 * kPi));  // -(kappa / 2 pi) q J_1 / r
  int m = i - j;
  if (m < 0) m += n;
  return ca(cs(L, h), cs(L1, G[5 * (size_t)n + m]));
}

constexpr int kCirculantMaxN = 8192;  // the shift-invariance test is O(n^2)

// Host: the device geometry G (6 n + 1 doubles) of a curve given by its samples
// s = [x1 | x2 | x1' | x2' | x1'' | x2''] (six rows of n values at t_j = 2 pi j / n).
// Returns false when n is odd or below 4, a sample is not finite, x'(t_j) = 0, or
// two sample points coincide.
inline bool build_geometry(const double* s, int n, double* G) {
  if (n < 4 || (n & 1)) return false;
  for (int j = 0; j < n; ++j) {
    const double x1 = s[j], x2 = s[n + j], d1 = s[2 * n + j], d2 = s[3 * n + j];
    const double dd1 = s[4 * n + j], dd2 = s[5 * n + j];
    const double sp2 = d1 * d1 + d2 * d2;
    if (!(isfinite(x1) && isfinite(x2) && isfinite(d1) && isfinite(d2) && isfinite(dd1) && isfinite(dd2)) ||
        !(sp2 > 0.0))
      return false;
    G[5 * j + 0] = x1;
    G[5 * j + 1] = x2;
    G[5 * j + 2] = d2;
    G[5 * j + 3] = -d1;
    G[5 * j + 4] = (d2 * dd1 - d1 * dd2) / (2.0 * kPi * sp2);
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (s[i] == s[j] && s[n + i] == s[n + j]) return false;
  const int np = n / 2;
  const double h = 2.0 * kPi / (double)n;
  // cos(k m pi / n') through the index k m mod 2 n'
  double* ct = new double[2 * np];
  for (int q = 0; q < 2 * np; ++q) ct[q] = cos(kPi * (double)q / (double)np);
  G[5 * (size_t)n] = 0.0;
  for (int m = 1; m < n; ++m) {
    double R = -(kPi / ((double)np * (double)np)) * ((m & 1) ? -1.0 : 1.0);
    double acc = 0.0;
    for (int k = 1; k < np; ++k) acc += ct[(int)(((long long)k * m) % (2 * np))] / (double)k;
    R -= (2.0 * kPi / (double)np) * acc;
    const double sn = sin(kPi * (double)m / (double)n);
    G[5 * (size_t)n + m] = R - h * log(4.0 * sn * sn);
  }
  delete[] ct;
  // circulant when every entry's geometry (r, n(t_j).(x_i - x_j), and the diagonal term)
  // depends on i - j only, to a few rounding units of the curve's size
  bool circ = n <= kCirculantMaxN;
  double scale = 0.0, dmax = 0.0;
  for (int j = 0; j < n; ++j) {
    scale = fmax(scale, fmax(fabs(G[5 * j]), fabs(G[5 * j + 1])));
    scale = fmax(scale, fmax(fabs(G[5 * j + 2]), fabs(G[5 * j + 3])));
    dmax = fmax(dmax, fabs(G[5 * j + 4]));
  }
  const double tol = 8e-15 * scale, tq = 8e-15 * scale * scale;
  for (int j = 1; j < n && circ; ++j) circ = fabs(G[5 * j + 4] - G[4]) <= 8e-15 * dmax;
  for (int m = 1; m < n && circ; ++m) {
    const double ex0 = G[5 * m] - G[0], ey0 = G[5 * m + 1] - G[1];
    const double r0 = hypot(ex0, ey0), q0 = G[2] * ex0 + G[3] * ey0;
    for (int j = 1; j < n; ++j) {
      const int i = (j + m) % n;
      const double ex = G[5 * i] - G[5 * j], ey = G[5 * i + 1] - G[5 * j + 1];
      if (fabs(hypot(ex, ey) - r0) > tol || fabs(G[5 * j + 2] * ex + G[5 * j + 3] * ey - q0) > tq) {
        circ = false;
        break;
      }
    }
  }
  G[6 * (size_t)n] = circ ? 1.0 : 0.0;
  return true;
}

}  // namespace bie
