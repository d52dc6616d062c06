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

// The k-step jump of classical RK4 on x'' = -B x.  One step maps (x, v) by
//   P = [[C, H], [G, C]],  C = I - W/2 + W^2/24,  H = h (I - W/6),  G = -h B (I - W/6),
// W = h^2 B (P(hA) of the first-order form, A = [[0, I], [-B, 0]]).  All blocks are
// polynomials in B, so P^k keeps the form [[C_k, H_k], [G_k, C_k]].  Returns
// Cm1 = C_k - I, H_k and G_k (row-major s x s, FP64).
void rk4_jump_blocks(int s, const double* B, double h, int k, std::vector<double>& Cm1, std::vector<double>& H,
                     std::vector<double>& G);

}  // namespace linalg
}  // namespace cho
