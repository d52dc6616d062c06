// linalg.h -- host FP64 linear algebra used when a system is created.
#pragma once

#include <vector>

namespace cho {
namespace linalg {

// M = L L^T (row-major lower L).  False if M is not positive definite.
bool cholesky(int s, const double* M, std::vector<double>& L);

// B = M^{-1} K given the Cholesky factor L of M.
void dense_B(int s, const std::vector<double>& L, const double* K, double* B);

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal d (s)
// and off-diagonal e (s - 1), by Sturm-sequence bisection.
double tridiag_max_eig(int s, const double* d, const double* e);

// Largest natural frequency of a fixed-free chain (masses m, springs C).
double omega_max_chain(int s, const double* m, const double* C);

// Largest natural frequency of M x'' + K x = 0 given the Cholesky factor of M.
double omega_max_dense(int s, const std::vector<double>& L, const double* K);

}  // namespace linalg
}  // namespace cho
