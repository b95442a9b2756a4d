// Host FP64 dense linear algebra used by rb_build (see linalg.cpp).
#pragma once
#include <complex>

namespace rb {
bool cholesky(int n, const std::complex<double>* A, std::complex<double>* L);
void lower_inverse(int n, const std::complex<double>* L, std::complex<double>* Li);
void herm_eig(int n, std::complex<double>* A, double* w, std::complex<double>* V);
}  // namespace rb
