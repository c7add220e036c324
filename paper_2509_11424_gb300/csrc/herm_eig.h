// Host eigen-decomposition of a small Hermitian matrix by the cyclic Jacobi
// method (Jacobi 1846; the complex form: each rotation first turns a_pq real
// with a phase on column q, then applies the real plane rotation that zeroes
// it, with the tangent t = sgn(z) / (|z| + sqrt(z^2 + 1)), z = (a_qq - a_pp) /
// (2 |a_pq|) of Rutishauser's Handbook procedure).  Used for the m x m Gram
// matrices of the test-vector refinement (m <= 128); O(m^3) per sweep.
#pragma once

#include <cmath>
#include <complex>
#include <vector>

namespace mg {

// A: m x m Hermitian, row-major, overwritten.  On return w[j] and column j of
// Z (row-major m x m) are the eigenpairs, unsorted.  Returns the sweeps used,
// or -1 when the off-diagonal part did not fall below 1e-15 ||A||_F within
// max_sweeps.
inline int herm_eig_jacobi(std::vector<std::complex<double>> &A, int m, std::vector<double> &w,
                           std::vector<std::complex<double>> &Z, int max_sweeps = 60) {
  using cd = std::complex<double>;
  Z.assign((size_t)m * m, cd(0.0, 0.0));
  for (int i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
  double fro = 0.0;
  for (const cd &a : A) fro += std::norm(a);
  fro = std::sqrt(fro);
  int sweep = 0;
  bool done = fro == 0.0;
  for (; !done && sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q)
        if (p != q) off += std::norm(A[(size_t)p * m + q]);
    if (std::sqrt(off) <= 1e-15 * fro) {
      done = true;
      break;
    }
    for (int p = 0; p + 1 < m; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const cd apq = A[(size_t)p * m + q];
        const double b = std::abs(apq);
        if (b == 0.0) continue;
        const cd e = apq / b;  // a_pq = b e, |e| = 1
        const double z = (A[(size_t)q * m + q].real() - A[(size_t)p * m + p].real()) / (2.0 * b);
        const double t = (z >= 0.0 ? 1.0 : -1.0) / (std::fabs(z) + std::sqrt(z * z + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        // J on columns p, q: J_pp = c, J_pq = s, J_qp = -s conj(e), J_qq = c conj(e)
        const cd jqp = -s * std::conj(e), jqq = c * std::conj(e);
        for (int i = 0; i < m; ++i) {  // A <- A J and Z <- Z J
          cd &aip = A[(size_t)i * m + p], &aiq = A[(size_t)i * m + q];
          const cd x = aip, y = aiq;
          aip = x * c + y * jqp;
          aiq = x * s + y * jqq;
          cd &zip = Z[(size_t)i * m + p], &ziq = Z[(size_t)i * m + q];
          const cd u = zip, v = ziq;
          zip = u * c + v * jqp;
          ziq = u * s + v * jqq;
        }
        for (int j = 0; j < m; ++j) {  // A <- J^H A
          cd &apj = A[(size_t)p * m + j], &aqj = A[(size_t)q * m + j];
          const cd x = apj, y = aqj;
          apj = c * x + std::conj(jqp) * y;
          aqj = s * x + std::conj(jqq) * y;
        }
        A[(size_t)p * m + q] = A[(size_t)q * m + p] = 0.0;
        A[(size_t)p * m + p] = A[(size_t)p * m + p].real();
        A[(size_t)q * m + q] = A[(size_t)q * m + q].real();
      }
    }
  }
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = A[(size_t)i * m + i].real();
  return done ? sweep : -1;
}

}  // namespace mg
