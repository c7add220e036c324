// Reads "m" then m*m rows "re im" (row-major) of a Hermitian matrix on stdin;
// prints the sweep count, then m eigenvalues, then Z row-major as "re im".
#include <cstdio>
#include <vector>

#include "herm_eig.h"

int main() {
  int m = 0;
  if (std::scanf("%d", &m) != 1 || m < 1) return 2;
  std::vector<std::complex<double>> A((size_t)m * m), Z;
  for (auto &a : A) {
    double re, im;
    if (std::scanf("%lf %lf", &re, &im) != 2) return 2;
    a = {re, im};
  }
  std::vector<double> w;
  const int sweeps = mg::herm_eig_jacobi(A, m, w, Z);
  std::printf("%d\n", sweeps);
  for (double x : w) std::printf("%.17g\n", x);
  for (auto &z : Z) std::printf("%.17g %.17g\n", z.real(), z.imag());
  return 0;
}
