// Host build of the device library's boundary-integral arithmetic (bie.cuh), for
// the CPU tests that check it against SciPy's Bessel functions and the oracle's
// Nystrom matrix. Test infrastructure: not part of the library.
#include <stdint.h>
#include <stdlib.h>

#include "../paper_2312_13117_gb300/csrc/bie.cuh"

extern "C" void bie_host_j1_h1(int32_t m, const double* w, double* J, double* H) {
  for (int32_t k = 0; k < m; ++k) {
    double2 j, h;
    bie::j1_h1(make_double2(w[2 * k], w[2 * k + 1]), &j, &h);
    J[2 * k] = j.x;
    J[2 * k + 1] = j.y;
    H[2 * k] = h.x;
    H[2 * k + 1] = h.y;
  }
}

// K_n(kappa) column-major (2 n n doubles); returns 0, or -1 when the curve is rejected.
extern "C" int32_t bie_host_matrix(int32_t n, const double* samples, double kre, double kim, double* K) {
  double* G = (double*)malloc(sizeof(double) * (6 * (size_t)n + 1));
  if (!bie::build_geometry(samples, n, G)) {
    free(G);
    return -1;
  }
  for (int32_t j = 0; j < n; ++j)
    for (int32_t i = 0; i < n; ++i) {
      const double2 v = bie::dlp_entry(G, n, i, j, make_double2(kre, kim));
      K[2 * ((size_t)j * n + i)] = v.x;
      K[2 * ((size_t)j * n + i) + 1] = v.y;
    }
  free(G);
  return 0;
}

// 1 when the geometry builder finds the curve shift-invariant (circulant matrix), 0 when
// not, -1 when the curve is rejected.
extern "C" int32_t bie_host_circulant(int32_t n, const double* samples) {
  double* G = (double*)malloc(sizeof(double) * (6 * (size_t)n + 1));
  int32_t r = -1;
  if (bie::build_geometry(samples, n, G)) r = G[6 * (size_t)n] != 0.0 ? 1 : 0;
  free(G);
  return r;
}
