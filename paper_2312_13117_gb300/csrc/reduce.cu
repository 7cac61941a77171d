// Segmented quadrature reduction and the ratio indicator.
//
// For each disk g with nodes z_j, weights w_j (Eq. 3.2), and solutions X_j:
//   C0 = sum_j w_j X_j, C1 = sum_j w_j z_j X_j                  (Eq. 3.2-3.3)
//   P f|_N = C0[:,0],  P f|_{N/2} = sum_{j odd} 2 w_j X_j[:,0]  (Eq. 3.1; the
//   1-based even nodes x_2, x_4, ..., x_N are the 0-based odd ones)
//   I = || P f|_N ./ P f|_{N/2} ||_2 / sqrt(n)                  (Eq. 3.1)
// With K > 1 moment pairs it also forms the scaled moments of the block Hankel
// form of Beyn's step, M_p = sum_j w_j ((z_j - c)/r)^p X_j, p < 2K; on the nodes
// ((z_j - c)/r)^p = e^{i p theta_j}, taken from the integer phase p j mod N.
// Nodes are summed in index order by one thread per output element, so the
// result is deterministic. The kernel streams X once: it is HBM-bound.
#include "pmcim_internal.cuh"

namespace {

constexpr int RT = 256;

__global__ void __launch_bounds__(RT) k_reduce_moments(LevelArgs a) {
  const int g = blockIdx.y;
  const RegionDev rg = a.regions[g];
  const ProblemDev* P = a.probs + rg.prob;
  const int n = P->n, l = P->l;
  const int nl = n * l;
  const int e = blockIdx.x * RT + threadIdx.x;
  if (e >= nl) return;
  const bool first_col = e < n;
  double2 c0 = make_double2(0.0, 0.0), c1 = c0, ph = c0;
  double pa = 0.0;
  const double2* Xg = a.X + rg.x_off + e;
  for (int j = 0; j < rg.N; ++j) {
    double2 z, w;
    node_weight(rg.cre, rg.cim, rg.r, rg.N, j, &z, &w);
    const double2 x = Xg[(size_t)j * nl];
    cfma(c0, w, x);
    cfma(c1, cmul(w, z), x);
    if (first_col) {
      if (j & 1) cfma(ph, cscale(w, 2.0), x);
      pa += hypot(w.x, w.y) * hypot(x.x, x.y);
    }
  }
  a.C0[rg.c_off + e] = c0;
  a.C1[rg.c_off + e] = c1;
  if (a.K > 1) {
    // M_0 = C0; M_p for 1 <= p < 2K, all p in one pass over the nodes
    double2 m[2 * PMCIM_MAX_BEYN_K - 1];
#pragma unroll
    for (int q = 0; q < 2 * PMCIM_MAX_BEYN_K - 1; ++q) m[q] = make_double2(0.0, 0.0);
    const double wr = rg.r / rg.N;
    for (int j = 0; j < rg.N; ++j) {
      const double2 x = Xg[(size_t)j * nl];
#pragma unroll
      for (int q = 0; q < 2 * PMCIM_MAX_BEYN_K - 1; ++q) {
        if (q + 1 < 2 * a.K) {
          // w_j e^{i (q+1) theta_j} = (r / N) e^{i (q+2) theta_j}
          const int ph = (int)(((long long)(q + 2) * j) % rg.N);
          double sn, cs;
          sincospi(2.0 * ph / rg.N, &sn, &cs);
          cfma(m[q], make_double2(wr * cs, wr * sn), x);
        }
      }
    }
    double2* Cm = a.Cm + (size_t)2 * a.K * rg.c_off + e;
    Cm[0] = c0;
#pragma unroll
    for (int q = 0; q < 2 * PMCIM_MAX_BEYN_K - 1; ++q)
      if (q + 1 < 2 * a.K) Cm[(size_t)(q + 1) * nl] = m[q];
  }
  if (first_col) {
    a.pf_half[rg.p_off + e] = ph;
    a.pf_abs[rg.p_off + e] = pa;
  }
}

__global__ void __launch_bounds__(RT) k_indicator(LevelArgs a) {
  __shared__ double red[2][RT / 32];
  const int g = blockIdx.x;
  const RegionDev rg = a.regions[g];
  const int n = a.probs[rg.prob].n;
  const double2* pfN = a.C0 + rg.c_off;  // column 0 of C0
  const double2* pfh = a.pf_half + rg.p_off;
  const double* pab = a.pf_abs + rg.p_off;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // pass 1: ||P f|_N||^2 and the size of the summed terms ||sum_j |w_j| |x_j|||^2
  double s_norm = 0.0, s_abs = 0.0;
  for (int i = threadIdx.x; i < n; i += RT) {
    s_norm += cabs2(pfN[i]);
    s_abs += pab[i] * pab[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s_norm += __shfl_down_sync(0xffffffffu, s_norm, o);
    s_abs += __shfl_down_sync(0xffffffffu, s_abs, o);
  }
  if (lane == 0) { red[0][wid] = s_norm; red[1][wid] = s_abs; }
  __syncthreads();
  double t1 = 0.0, t2 = 0.0;
  for (int k = 0; k < RT / 32; ++k) { t1 += red[0][k]; t2 += red[1][k]; }
  __syncthreads();
  // pass 2: Eq. 3.1 componentwise; a component whose |P f|_{N/2}| is at or below the
  // rounding level kPfFloor ||sum_j |w_j| |x_j||| has no determined ratio and is left out
  // (the root mean square runs over the components with a determined ratio)
  const double floor2 = kPfFloor * kPfFloor * t2;
  double s_ratio = 0.0, s_kept = 0.0;
  for (int i = threadIdx.x; i < n; i += RT) {
    const double den = cabs2(pfh[i]);
    if (den > floor2) {
      s_ratio += cabs2(pfN[i]) / den;
      s_kept += 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s_ratio += __shfl_down_sync(0xffffffffu, s_ratio, o);
    s_kept += __shfl_down_sync(0xffffffffu, s_kept, o);
  }
  if (lane == 0) { red[0][wid] = s_ratio; red[1][wid] = s_kept; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, tk = 0.0;
    for (int k = 0; k < RT / 32; ++k) { t0 += red[0][k]; tk += red[1][k]; }
    // P f = 0 when the disk holds no eigenvalue (Sec. 2.1): at rounding level the
    // ratio of Eq. 3.1 is 0/0, and the indicator is taken as 0
    const double I = (sqrt(t1) <= kPfFloor * sqrt(t2) || tk == 0.0) ? 0.0 : sqrt(t0 / tk);
    a.ind[g] = I;
    a.pf_norm[g] = sqrt(t1);
    a.pf_scale[g] = sqrt(t2);
    a.cand[g] = (I > a.tol_ind) ? 1 : 0;
  }
}

__global__ void k_gather_vecs(const double2* __restrict__ src, double2* __restrict__ dst,
                              const VecItem* __restrict__ items) {
  const VecItem it = items[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= it.n) return;
  dst[it.dst + i] = src[it.src + i];
}

// The data of a certificate's bordered inverse step, one value per CTA (values
// with off[m] < 0 are skipped). T is T(lambda), or T(lambda)^H when a.herm. With
// c the value's start vector: s = the index of the largest |c_i| (the smallest
// such index), written to regions[m].border as s + 1; at out + off[m] the
// right-hand side b = -T e_s (n values; for T^H the conjugate of row s of
// T(lambda)) and then the replacement column alpha c, alpha = ||T e_s|| / ||c||
// (1 when either norm is zero), so that it is on the scale of the columns it
// stands among.
__global__ void __launch_bounds__(RT) k_border_rhs(ValueArgs a, const int64_t* __restrict__ off,
                                                   double2* __restrict__ out, RegionDev* __restrict__ regions) {
  __shared__ ProblemDev P;
  __shared__ double2 fz[PMCIM_MAX_TERMS];
  __shared__ double rq[RT / 32], rc[RT / 32];
  __shared__ int ri[RT / 32];
  __shared__ double alpha;
  __shared__ int s_col;
  const int m = blockIdx.x;
  if (off[m] < 0) return;
  load_problem(&P, a.probs + a.prob_of[m]);
  __syncthreads();
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  const double2* c = a.vecs + a.vec_off[m];
  double2* b = out + off[m];
  if (threadIdx.x < P.K) fz[threadIdx.x] = eval_f(P.term[threadIdx.x], a.lam[m]);
  // argmax |c_i| (each thread scans increasing i, so a tie keeps the smaller index) and ||c||^2
  double best = -1.0, cc = 0.0;
  int bi = 0;
  for (int i = threadIdx.x; i < n; i += RT) {
    const double q = cabs2(c[i]);
    cc += q;
    if (q > best) {
      best = q;
      bi = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    cc += __shfl_down_sync(0xffffffffu, cc, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    rq[threadIdx.x >> 5] = best;
    ri[threadIdx.x >> 5] = bi;
    rc[threadIdx.x >> 5] = cc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bq = rq[0];
    int bs = ri[0];
    for (int k = 1; k < RT / 32; ++k)
      if (rq[k] > bq || (rq[k] == bq && ri[k] < bs)) {
        bq = rq[k];
        bs = ri[k];
      }
    s_col = bs;
  }
  __syncthreads();
  const int sc = s_col;
  // b = -(column s of T) and its squared norm
  double tt = 0.0;
  for (int i = threadIdx.x; i < n; i += RT) {
    double2 t = make_double2(0.0, 0.0);
    const size_t e = a.herm ? (size_t)i * n + sc : (size_t)sc * n + i;  // element (i, s) or (s, i) of T(lambda)
    for (int k = 0; k < P.K; ++k) {
      const TermDesc& tk = P.term[k];
      if (tk.dense) cfma(t, fz[k], P.A[(size_t)tk.mat_index * nn + e]);
      else if (i == sc) cfma(t, fz[k], tk.id);
    }
    tt += cabs2(t);
    b[i] = a.herm ? make_double2(-t.x, t.y) : make_double2(-t.x, -t.y);
  }
  for (int o = 16; o > 0; o >>= 1) tt += __shfl_down_sync(0xffffffffu, tt, o);
  __syncthreads();  // rq is reused
  if ((threadIdx.x & 31) == 0) rq[threadIdx.x >> 5] = tt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0, c2 = 0.0;
    for (int k = 0; k < RT / 32; ++k) {
      t2 += rq[k];
      c2 += rc[k];
    }
    alpha = (t2 > 0.0 && c2 > 0.0 && isfinite(t2) && isfinite(c2)) ? sqrt(t2) / sqrt(c2) : 1.0;
    regions[m].border = sc + 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RT) b[n + i] = cscale(c[i], alpha);
}

// Verification certificate (pmCIMb step 3): for a candidate lambda and a vector
// v != 0, sigma_min(T(lambda)) <= ||T(lambda) v|| / ||v||, and likewise with
// T(lambda)^H (a.herm), whose smallest singular value is the same. One CTA per
// value forms T(lambda) element by element (never stored), accumulating
// r = T v (or T^H v) and ||T(lambda)||_F^2, all in FP64.
template <bool BIE>
__global__ void __launch_bounds__(RT) k_certify(ValueArgs a) {
  constexpr int kCircMax = 2048;  // circulant boundary-integral matrices up to this n: first column in smem
  __shared__ ProblemDev P;
  __shared__ double2 fz[PMCIM_MAX_TERMS];
  __shared__ double red[2][RT / 32];
  __shared__ double2 ccol[BIE ? kCircMax : 1];
  const int m = blockIdx.x;
  load_problem(&P, a.probs + a.prob_of[m]);
  __syncthreads();
  const int n = P.n;
  const size_t nn = (size_t)n * n;
  const double2 lam = a.lam[m];
  const double2* v = a.vecs + a.vec_off[m];
  if (threadIdx.x < P.K) fz[threadIdx.x] = eval_f(P.term[threadIdx.x], lam);
  const bool circ = BIE && P.bie_circ && n <= kCircMax;
  if (circ)
    for (int q = threadIdx.x; q < n; q += RT) ccol[q] = bie::dlp_entry(P.bie, n, q, 0, lam);
  __syncthreads();
  double r2 = 0.0, f2 = 0.0;
  for (int row = threadIdx.x; row < n; row += RT) {
    double2 r = make_double2(0.0, 0.0);
    for (int col = 0; col < n; ++col) {
      double2 t = make_double2(0.0, 0.0);
      // element (row, col) of T(lambda), or for T^H the conjugate of element (col, row)
      const size_t e = a.herm ? (size_t)row * n + col : (size_t)col * n + row;
      for (int k = 0; k < P.K; ++k) {
        const TermDesc& tk = P.term[k];
        if (tk.dense) cfma(t, fz[k], P.A[(size_t)tk.mat_index * nn + e]);
        else if (BIE && tk.kind == PMCIM_F_HELMHOLTZ_DLP) {  // T^H: entry (col, row), conjugated below
          const int i = a.herm ? col : row, j = a.herm ? row : col;
          cfma(t, tk.id, circ ? ccol[i >= j ? i - j : i - j + n] : bie::dlp_entry(P.bie, n, i, j, fz[k]));
        }
        else if (row == col) cfma(t, fz[k], tk.id);
      }
      if (a.herm) t.y = -t.y;
      cfma(r, t, v[col]);
      f2 += cabs2(t);
    }
    r2 += cabs2(r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
    f2 += __shfl_down_sync(0xffffffffu, f2, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = r2; red[1][threadIdx.x >> 5] = f2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, tf = 0.0, vv = 0.0;
    for (int k = 0; k < RT / 32; ++k) { tr += red[0][k]; tf += red[1][k]; }
    for (int i = 0; i < n; ++i) vv += cabs2(v[i]);
    const double cert = sqrt(tr) / sqrt(vv);
    a.sigma[m] = cert;
    a.accept[m] = (cert <= a.tol_verify * fmax(1.0, sqrt(tf) / sqrt((double)n))) ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// Certificates of many values of one problem from coefficient products: with
// T(lambda) = sum_d f_d(lambda) A_d + g(lambda) I (d over the dense terms, g the
// identity terms), T(lambda_i) v_i = sum_d f_d(lambda_i) (A_d v_i) + g(lambda_i) v_i,
// and the products W_d = A_d [v_1 .. v_m] read each A_d once for all m values
// instead of once per value. ||T(lambda)||_F^2 comes from the Gram data of the
// coefficients: sum_{d,e} f_d conj(f_e) <A_d, A_e> + 2 Re(conj(g) sum_d f_d tr A_d)
// + n |g|^2, with <X, Y> = sum_ij X_ij conj(Y_ij). All in FP64.
// ---------------------------------------------------------------------------
constexpr int GT_R = 64, GT_C = 16, GT_K = 32;  // product tile: rows x values, inner chunk

// W[(d m + i) n + row] = (A_d v_i)[row]: grid (row tiles, value tiles, dense terms).
__global__ void __launch_bounds__(RT) k_apply_dense(const ProblemDev* __restrict__ prob, const double2* __restrict__ vecs,
                                                    const int64_t* __restrict__ vec_off, int m,
                                                    double2* __restrict__ W) {
  __shared__ double2 As[GT_K][GT_R];
  __shared__ double2 Bs[GT_K][GT_C];
  __shared__ int mat;
  const int n = prob->n;
  const int r0 = blockIdx.x * GT_R, c0 = blockIdx.y * GT_C, d = blockIdx.z;
  if (threadIdx.x == 0) {
    int dd = -1;
    for (int k = 0; k < prob->K; ++k)
      if (prob->term[k].dense && ++dd == d) mat = prob->term[k].mat_index;
  }
  __syncthreads();
  const double2* A = prob->A + (size_t)mat * n * n;
  const int tx = threadIdx.x % GT_R, ty = threadIdx.x / GT_R;  // a row, and 4 values
  double2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < n; k0 += GT_K) {
#pragma unroll
    for (int u = 0; u < GT_K * GT_R / RT; ++u) {
      const int e = threadIdx.x + u * RT, k = e / GT_R, r = e % GT_R;
      As[k][r] = (r0 + r < n && k0 + k < n) ? A[(size_t)(k0 + k) * n + r0 + r] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < GT_K * GT_C / RT; ++u) {
      const int e = threadIdx.x + u * RT, c = e / GT_K, k = e % GT_K;
      Bs[k][c] = (c0 + c < m && k0 + k < n) ? vecs[vec_off[c0 + c] + k0 + k] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GT_K; ++k) {
      const double2 av = As[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) cfma(acc[q], av, Bs[k][4 * ty + q]);
    }
    __syncthreads();
  }
  if (r0 + tx < n)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c0 + 4 * ty + q < m) W[((size_t)d * m + c0 + 4 * ty + q) * n + r0 + tx] = acc[q];
}

// Gram data of one problem's dense coefficients, first pass: per CTA, the partial
// sums of <A_d, A_e> (d <= e, at most GRAM_MAX_DENSE dense terms) over its share of
// the elements, into partial[blockIdx][pair]. The second pass adds them in CTA
// order (deterministic) and the traces.
constexpr int GRAM_MAX_DENSE = 4;
constexpr int GRAM_PAIRS = GRAM_MAX_DENSE * (GRAM_MAX_DENSE + 1) / 2;
__global__ void __launch_bounds__(RT) k_gram_partial(const ProblemDev* __restrict__ prob, double2* __restrict__ partial) {
  __shared__ double red[2][RT / 32];
  __shared__ int mats[GRAM_MAX_DENSE];
  __shared__ int nd;
  const int n = prob->n;
  const size_t nn = (size_t)n * n;
  if (threadIdx.x == 0) {
    int dd = 0;
    for (int k = 0; k < prob->K; ++k)
      if (prob->term[k].dense && dd < GRAM_MAX_DENSE) mats[dd++] = prob->term[k].mat_index;
    nd = dd;
  }
  __syncthreads();
  double2 acc[GRAM_PAIRS];
#pragma unroll
  for (int q = 0; q < GRAM_PAIRS; ++q) acc[q] = make_double2(0.0, 0.0);
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < nn; e += (size_t)gridDim.x * RT) {
    double2 v[GRAM_MAX_DENSE];
#pragma unroll
    for (int d = 0; d < GRAM_MAX_DENSE; ++d) v[d] = d < nd ? prob->A[(size_t)mats[d] * nn + e] : make_double2(0.0, 0.0);
    int q = 0;
#pragma unroll
    for (int d = 0; d < GRAM_MAX_DENSE; ++d)
#pragma unroll
      for (int f = d; f < GRAM_MAX_DENSE; ++f, ++q) cfma_conj(acc[q], v[f], v[d]);  // v_d conj(v_f)
  }
#pragma unroll
  for (int q = 0; q < GRAM_PAIRS; ++q) {
    double x = acc[q].x, y = acc[q].y;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = x; red[1][threadIdx.x >> 5] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sx = 0.0, sy = 0.0;
      for (int w = 0; w < RT / 32; ++w) { sx += red[0][w]; sy += red[1][w]; }
      partial[(size_t)blockIdx.x * GRAM_PAIRS + q] = make_double2(sx, sy);
    }
  }
}

// Second pass: gram[pair] = the sum of the partials in CTA order; gram[GRAM_PAIRS + d]
// = tr A_d.
__global__ void __launch_bounds__(32) k_gram_final(const ProblemDev* __restrict__ prob,
                                                   const double2* __restrict__ partial, int parts,
                                                   double2* __restrict__ gram) {
  const int n = prob->n;
  const int q = threadIdx.x;
  if (q < GRAM_PAIRS) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < parts; ++b) s = cadd(s, partial[(size_t)b * GRAM_PAIRS + q]);
    gram[q] = s;
  }
  if (q < GRAM_MAX_DENSE) {
    int dd = -1, mat = -1;
    for (int k = 0; k < prob->K; ++k)
      if (prob->term[k].dense && ++dd == q) mat = prob->term[k].mat_index;
    double2 t = make_double2(0.0, 0.0);
    if (mat >= 0)
      for (int i = 0; i < n; ++i) t = cadd(t, prob->A[(size_t)mat * n * n + (size_t)i * n + i]);
    gram[GRAM_PAIRS + q] = t;
  }
}

// Per value (one CTA each): r = sum_d f_d W_d[:, i] + g v_i, the certificate ||r|| / ||v||,
// ||T(lambda)||_F from the Gram data, and the acceptance as in k_certify.
__global__ void __launch_bounds__(RT) k_certify_products(ValueArgs a, const double2* __restrict__ W,
                                                         const int64_t* __restrict__ w_col,
                                                         const int32_t* __restrict__ w_m, const double2* gram) {
  __shared__ ProblemDev P;
  __shared__ double2 fz[PMCIM_MAX_TERMS];
  __shared__ double red[2][RT / 32];
  const int m = blockIdx.x;
  load_problem(&P, a.probs + a.prob_of[m]);
  __syncthreads();
  const int n = P.n;
  const double2 lam = a.lam[m];
  const double2* v = a.vecs + a.vec_off[m];
  if (threadIdx.x < P.K) fz[threadIdx.x] = eval_f(P.term[threadIdx.x], lam);
  __syncthreads();
  double2 g = make_double2(0.0, 0.0), fd[GRAM_MAX_DENSE];
  int nd = 0;
  for (int k = 0; k < P.K; ++k) {
    if (P.term[k].dense) {
      if (nd < GRAM_MAX_DENSE) fd[nd] = fz[k];
      ++nd;
    } else {
      cfma(g, fz[k], P.term[k].id);
    }
  }
  gram += (size_t)a.prob_of[m] * (GRAM_PAIRS + GRAM_MAX_DENSE);  // this value's problem
  const double2* w0 = W + w_col[m];  // term d's column at w0 + d * w_m[m] * n
  const size_t dstride = (size_t)w_m[m] * n;
  double r2 = 0.0, v2 = 0.0;
  for (int row = threadIdx.x; row < n; row += RT) {
    const double2 vr = v[row];
    double2 r = cmul(g, vr);
    for (int d = 0; d < nd && d < GRAM_MAX_DENSE; ++d) cfma(r, fd[d], w0[(size_t)d * dstride + row]);
    r2 += cabs2(r);
    v2 += cabs2(vr);
  }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = r2; red[1][threadIdx.x >> 5] = v2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, tv = 0.0;
    for (int k = 0; k < RT / 32; ++k) { tr += red[0][k]; tv += red[1][k]; }
    // ||T||_F^2 from the Gram data (pairs d <= e in row order)
    double f2 = (double)n * cabs2(g);
    int q = 0;
    for (int d = 0; d < GRAM_MAX_DENSE; ++d)
      for (int e = d; e < GRAM_MAX_DENSE; ++e, ++q) {
        if (d >= nd || e >= nd) continue;
        // f_d conj(f_e) <A_d, A_e>, and for d != e its conjugate partner
        const double2 t = cmul(cmul(fd[d], cconj(fd[e])), gram[q]);
        f2 += (d == e) ? t.x : 2.0 * t.x;
      }
    double2 sft = make_double2(0.0, 0.0);
    for (int d = 0; d < nd && d < GRAM_MAX_DENSE; ++d) cfma(sft, fd[d], gram[GRAM_PAIRS + d]);
    f2 += 2.0 * cmul(cconj(g), sft).x;
    const double cert = sqrt(tr) / sqrt(tv);
    a.sigma[m] = cert;
    a.accept[m] = (cert <= a.tol_verify * fmax(1.0, sqrt(fmax(f2, 0.0)) / sqrt((double)n))) ? 1 : 0;
  }
}

}  // namespace

size_t gram_partial_count() { return 256; }
size_t gram_entries() { return GRAM_PAIRS + GRAM_MAX_DENSE; }
int gram_max_dense() { return GRAM_MAX_DENSE; }

cudaError_t launch_gram(const ProblemDev* prob, double2* partial, double2* gram, cudaStream_t s) {
  k_gram_partial<<<(unsigned)gram_partial_count(), RT, 0, s>>>(prob, partial);
  k_gram_final<<<1, 32, 0, s>>>(prob, partial, (int)gram_partial_count(), gram);
  return cudaGetLastError();
}

cudaError_t launch_apply_dense(const ProblemDev* prob, int n, int n_dense, const double2* vecs,
                               const int64_t* vec_off, int m, double2* W, cudaStream_t s) {
  if (m <= 0 || n_dense <= 0) return cudaSuccess;
  dim3 grid((n + GT_R - 1) / GT_R, (m + GT_C - 1) / GT_C, n_dense);
  k_apply_dense<<<grid, RT, 0, s>>>(prob, vecs, vec_off, m, W);
  return cudaGetLastError();
}

cudaError_t launch_certify_products(const ValueArgs& a, const double2* W, const int64_t* w_col, const int32_t* w_m,
                                    const double2* gram, cudaStream_t s) {
  if (a.m <= 0) return cudaSuccess;
  k_certify_products<<<a.m, RT, 0, s>>>(a, W, w_col, w_m, gram);
  return cudaGetLastError();
}

cudaError_t launch_certify(const ValueArgs& a, cudaStream_t s) {
  if (a.m <= 0) return cudaSuccess;
  if (a.bie) k_certify<true><<<a.m, RT, 0, s>>>(a);
  else k_certify<false><<<a.m, RT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce_moments(const LevelArgs& a, cudaStream_t s) {
  if (a.R <= 0) return cudaSuccess;
  dim3 grid((a.max_nl + RT - 1) / RT, a.R);
  k_reduce_moments<<<grid, RT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_indicator(const LevelArgs& a, cudaStream_t s) {
  if (a.R <= 0) return cudaSuccess;
  k_indicator<<<a.R, RT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_border_rhs(const ValueArgs& a, const int64_t* off, double2* out, RegionDev* regions,
                              cudaStream_t s) {
  if (a.m <= 0) return cudaSuccess;
  k_border_rhs<<<a.m, RT, 0, s>>>(a, off, out, regions);
  return cudaGetLastError();
}

cudaError_t launch_gather_vecs(const double2* src, double2* dst, const VecItem* items, int count, int max_n,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  dim3 grid((max_n + 127) / 128, count);
  k_gather_vecs<<<grid, 128, 0, s>>>(src, dst, items);
  return cudaGetLastError();
}
