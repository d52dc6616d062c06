// linalg.cpp -- host FP64 linear algebra for system set-up (step a0).
//
// B = M^{-1} K for dense systems by a Cholesky solve, and the largest natural
// frequency omega_max (sqrt of the largest eigenvalue of the pencil (K, M)),
// which bounds the RK4 step: RK4 is stable on the imaginary axis for
// |omega h| <= 2 sqrt 2.  The eigenvalue is found by Sturm-sequence bisection
// on a symmetric tridiagonal matrix: directly for spring chains (whose
// M^{-1/2} K M^{-1/2} is tridiagonal) and after Householder reduction of
// L^{-1} K L^{-T} for dense systems.
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace cho {
namespace linalg {

bool cholesky(int s, const double* M, std::vector<double>& L)
{
    L.assign((size_t)s * s, 0.0);
    for (int j = 0; j < s; ++j) {
        double d = M[(size_t)j * s + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * s + k] * L[(size_t)j * s + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * s + j] = ljj;
        for (int i = j + 1; i < s; ++i) {
            double t = M[(size_t)i * s + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * s + k] * L[(size_t)j * s + k];
            L[(size_t)i * s + j] = t / ljj;
        }
    }
    return true;
}

// Y = L^{-1} A for an s x s row-major A (forward substitution per column).
static void lower_solve(int s, const std::vector<double>& L, const double* A, std::vector<double>& Y)
{
    Y.assign(A, A + (size_t)s * s);
    for (int i = 0; i < s; ++i) {
        double* yi = &Y[(size_t)i * s];
        for (int k = 0; k < i; ++k) {
            const double lik = L[(size_t)i * s + k];
            if (lik == 0.0) continue;
            const double* yk = &Y[(size_t)k * s];
            for (int c = 0; c < s; ++c) yi[c] -= lik * yk[c];
        }
        const double inv = 1.0 / L[(size_t)i * s + i];
        for (int c = 0; c < s; ++c) yi[c] *= inv;
    }
}

// X = L^{-T} Y (back substitution per column).
static void upper_solve_T(int s, const std::vector<double>& L, const std::vector<double>& Y, double* X)
{
    std::memcpy(X, Y.data(), sizeof(double) * (size_t)s * s);
    for (int i = s - 1; i >= 0; --i) {
        double* xi = X + (size_t)i * s;
        for (int k = i + 1; k < s; ++k) {
            const double lki = L[(size_t)k * s + i];
            if (lki == 0.0) continue;
            const double* xk = X + (size_t)k * s;
            for (int c = 0; c < s; ++c) xi[c] -= lki * xk[c];
        }
        const double inv = 1.0 / L[(size_t)i * s + i];
        for (int c = 0; c < s; ++c) xi[c] *= inv;
    }
}

void dense_B(int s, const std::vector<double>& L, const double* K, double* B)
{
    std::vector<double> Y;
    lower_solve(s, L, K, Y);
    upper_solve_T(s, L, Y, B);
}

// Number of eigenvalues of tridiag(d, e) below x (Sturm count of the LDL^T pivots).
static int sturm_count(int s, const double* d, const double* e, double x)
{
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < s; ++i) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

double tridiag_max_eig(int s, const double* d, const double* e)
{
    if (s == 1) return d[0];
    double lo = d[0], hi = d[0];
    for (int i = 0; i < s; ++i) {
        double r = 0.0;
        if (i > 0) r += std::fabs(e[i - 1]);
        if (i + 1 < s) r += std::fabs(e[i]);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    hi += 1e-300 + std::fabs(hi) * 1e-15;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(s, d, e, mid) == s) hi = mid; else lo = mid;
        if (hi - lo <= 1e-15 * std::max(std::fabs(lo), std::fabs(hi))) break;
    }
    return 0.5 * (lo + hi);
}

double omega_max_chain(int s, const double* m, const double* C)
{
    if (s == 1) return std::sqrt(C[0] / m[0]);
    std::vector<double> d(s), e(s - 1);
    for (int i = 0; i < s; ++i) d[i] = (C[i] + (i + 1 < s ? C[i + 1] : 0.0)) / m[i];
    if (s == 2) {
        // B = M^{-1} K is 2 x 2 with a non-negative off-diagonal product: closed form
        const double b11 = d[0], b22 = d[1];
        const double b12 = -C[1] / m[0], b21 = -C[1] / m[1];
        const double half = 0.5 * (b11 - b22);
        return std::sqrt(0.5 * (b11 + b22) + std::sqrt(half * half + b12 * b21));
    }
    for (int i = 0; i + 1 < s; ++i) e[i] = -C[i + 1] / std::sqrt(m[i] * m[i + 1]);
    return std::sqrt(std::max(0.0, tridiag_max_eig(s, d.data(), e.data())));
}

// Householder reduction of a symmetric matrix (destroyed) to tridiagonal (d, e).
static void householder_tridiag(int s, std::vector<double>& A, std::vector<double>& d, std::vector<double>& e)
{
    d.assign(s, 0.0);
    e.assign(s > 1 ? s - 1 : 1, 0.0);
    std::vector<double> v(s), p(s);
    for (int k = 0; k + 2 < s; ++k) {
        const int m = s - k - 1;                  // length of the column below the diagonal
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += A[(size_t)(k + 1 + i) * s + k] * A[(size_t)(k + 1 + i) * s + k];
        nrm = std::sqrt(nrm);
        const double x0 = A[(size_t)(k + 1) * s + k];
        const double alpha = x0 >= 0 ? -nrm : nrm;
        e[k] = alpha;
        if (nrm == 0.0) continue;
        for (int i = 0; i < m; ++i) v[i] = A[(size_t)(k + 1 + i) * s + k];
        v[0] -= alpha;
        double vn = 0.0;
        for (int i = 0; i < m; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = 0; i < m; ++i) v[i] /= vn;
        // p = A22 v, w = p - (v^T p) v, A22 -= 2 (v w^T + w v^T)
        double vp = 0.0;
        for (int i = 0; i < m; ++i) {
            double t = 0.0;
            const double* row = &A[(size_t)(k + 1 + i) * s + (k + 1)];
            for (int j = 0; j < m; ++j) t += row[j] * v[j];
            p[i] = t;
            vp += v[i] * t;
        }
        for (int i = 0; i < m; ++i) p[i] -= vp * v[i];
        for (int i = 0; i < m; ++i) {
            double* row = &A[(size_t)(k + 1 + i) * s + (k + 1)];
            for (int j = 0; j < m; ++j) row[j] -= 2.0 * (v[i] * p[j] + p[i] * v[j]);
        }
    }
    for (int i = 0; i < s; ++i) d[i] = A[(size_t)i * s + i];
    if (s >= 2) e[s - 2] = A[(size_t)(s - 1) * s + (s - 2)];
}

double omega_max_dense(int s, const std::vector<double>& L, const double* K)
{
    // C = L^{-1} K L^{-T} = L^{-1} (L^{-1} K)^T for symmetric K
    std::vector<double> Y, Yt((size_t)s * s), C;
    lower_solve(s, L, K, Y);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) Yt[(size_t)j * s + i] = Y[(size_t)i * s + j];
    lower_solve(s, L, Yt.data(), C);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < i; ++j) {
            const double a = 0.5 * (C[(size_t)i * s + j] + C[(size_t)j * s + i]);
            C[(size_t)i * s + j] = C[(size_t)j * s + i] = a;
        }
    if (s == 1) return std::sqrt(std::max(0.0, C[0]));
    std::vector<double> d, e;
    householder_tridiag(s, C, d, e);
    return std::sqrt(std::max(0.0, tridiag_max_eig(s, d.data(), e.data())));
}


// C = A B (row-major s x s), i-k-j order.
static void matmul(int s, const std::vector<double>& A, const std::vector<double>& B, std::vector<double>& C)
{
    C.assign((size_t)s * s, 0.0);
    for (int i = 0; i < s; ++i)
        for (int l = 0; l < s; ++l) {
            const double a = A[(size_t)i * s + l];
            if (a == 0.0) continue;
            const double* b = &B[(size_t)l * s];
            double* c = &C[(size_t)i * s];
            for (int j = 0; j < s; ++j) c[j] += a * b[j];
        }
}

namespace {
// A matrix of the form [[C, H], [G, C]] with commuting blocks.
struct Jump {
    std::vector<double> C, H, G;
};

// X Y for two such matrices: [[Cx Cy + Hx Gy, Cx Hy + Hx Cy], [Gx Cy + Cx Gy, ...]]
Jump jump_mul(int s, const Jump& X, const Jump& Y)
{
    Jump Z;
    std::vector<double> t;
    const size_t n = (size_t)s * s;
    matmul(s, X.C, Y.C, Z.C);
    matmul(s, X.H, Y.G, t);
    for (size_t i = 0; i < n; ++i) Z.C[i] += t[i];
    matmul(s, X.C, Y.H, Z.H);
    matmul(s, X.H, Y.C, t);
    for (size_t i = 0; i < n; ++i) Z.H[i] += t[i];
    matmul(s, X.G, Y.C, Z.G);
    matmul(s, X.C, Y.G, t);
    for (size_t i = 0; i < n; ++i) Z.G[i] += t[i];
    return Z;
}
}  // namespace

void rk4_jump_blocks(int s, const double* B, double h, int k, std::vector<double>& Cm1, std::vector<double>& H,
                     std::vector<double>& G)
{
    const size_t n = (size_t)s * s;
    std::vector<double> Bm(B, B + n), W(n), W2;
    for (size_t i = 0; i < n; ++i) W[i] = h * h * Bm[i];
    matmul(s, W, W, W2);
    Jump P;
    P.C.resize(n);
    P.H.resize(n);
    std::vector<double> S(n);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) {
            const size_t ij = (size_t)i * s + j;
            const double I = i == j ? 1.0 : 0.0;
            P.C[ij] = I - W[ij] / 2.0 + W2[ij] / 24.0;
            S[ij] = I - W[ij] / 6.0;
            P.H[ij] = h * S[ij];
        }
    matmul(s, Bm, S, P.G);
    for (size_t i = 0; i < n; ++i) P.G[i] *= -h;
    Jump R;
    bool have = false;
    Jump base = P;
    for (int kk = k; kk > 0; kk >>= 1) {
        if (kk & 1) {
            R = have ? jump_mul(s, R, base) : base;
            have = true;
        }
        if (kk > 1) base = jump_mul(s, base, base);
    }
    Cm1 = R.C;
    for (int i = 0; i < s; ++i) Cm1[(size_t)i * s + i] -= 1.0;
    H = R.H;
    G = R.G;
}

}  // namespace linalg
}  // namespace cho
