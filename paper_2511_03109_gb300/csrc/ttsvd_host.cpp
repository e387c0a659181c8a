// Host FP64 pieces of the near-field TT-SVD for d_theta > 1 (§4.3; TT-SVD of Oseledets 2011,
// Alg. 1): a one-sided Jacobi SVD for the small matrices of the cuts after the first, and the
// compression of the first cut's remainder.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "handle.h"

namespace ph {

// Thin SVD of the m x n column-major matrix A: A = U diag(s) Vt with s descending, U m x k,
// Vt k x n, k = min(m, n).  One-sided Jacobi (Hestenes) on the columns of A (or of A^T when
// m < n), rotations until every pair of columns is orthogonal to 1e-15 relative.
void svd_small(int m, int n, const std::vector<double>& A, std::vector<double>& U, std::vector<double>& s,
               std::vector<double>& Vt) {
    const bool tr = m < n;
    const int M = tr ? n : m, N = tr ? m : n;  // work on M x N, M >= N
    std::vector<double> W((size_t)M * N), V((size_t)N * N, 0.0);
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < M; ++i) W[i + (size_t)M * j] = tr ? A[j + (size_t)m * i] : A[i + (size_t)m * j];
    for (int j = 0; j < N; ++j) V[j + (size_t)N * j] = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < N - 1; ++p)
            for (int q = p + 1; q < N; ++q) {
                double a = 0, b = 0, c = 0;
                for (int i = 0; i < M; ++i) {
                    const double x = W[i + (size_t)M * p], y = W[i + (size_t)M * q];
                    a += x * x;
                    b += y * y;
                    c += x * y;
                }
                if (std::fabs(c) <= 1e-15 * std::sqrt(a * b) || c == 0.0) continue;
                rotated = true;
                const double zeta = (b - a) / (2.0 * c);
                const double t = std::copysign(1.0, zeta) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < M; ++i) {
                    const double x = W[i + (size_t)M * p], y = W[i + (size_t)M * q];
                    W[i + (size_t)M * p] = cs * x - sn * y;
                    W[i + (size_t)M * q] = sn * x + cs * y;
                }
                for (int i = 0; i < N; ++i) {
                    const double x = V[i + (size_t)N * p], y = V[i + (size_t)N * q];
                    V[i + (size_t)N * p] = cs * x - sn * y;
                    V[i + (size_t)N * q] = sn * x + cs * y;
                }
            }
        if (!rotated) break;
    }
    std::vector<double> nrm(N);
    for (int j = 0; j < N; ++j) {
        double t = 0;
        for (int i = 0; i < M; ++i) t += W[i + (size_t)M * j] * W[i + (size_t)M * j];
        nrm[j] = std::sqrt(t);
    }
    std::vector<int> ord(N);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
    // W = U_w S, A_w = W V^T: for A (m >= n) U = U_w, Vt = V^T; for A^T the roles swap
    std::vector<double> Uw((size_t)M * N), Vw((size_t)N * N);
    s.assign(N, 0.0);
    for (int k = 0; k < N; ++k) {
        const int j = ord[k];
        s[k] = nrm[j];
        const double inv = nrm[j] > 0 ? 1.0 / nrm[j] : 0.0;
        for (int i = 0; i < M; ++i) Uw[i + (size_t)M * k] = W[i + (size_t)M * j] * inv;
        for (int i = 0; i < N; ++i) Vw[i + (size_t)N * k] = V[i + (size_t)N * j];
    }
    if (!tr) {
        U = Uw;  // m x N
        Vt.assign((size_t)N * n, 0.0);
        for (int k = 0; k < N; ++k)
            for (int i = 0; i < n; ++i) Vt[k + (size_t)N * i] = Vw[i + (size_t)N * k];
    } else {
        // A^T = Uw S Vw^T  =>  A = Vw S Uw^T: U = Vw (m x N), Vt = Uw^T (N x n)
        U = Vw;
        Vt.assign((size_t)N * n, 0.0);
        for (int k = 0; k < N; ++k)
            for (int i = 0; i < n; ++i) Vt[k + (size_t)N * i] = Uw[i + (size_t)M * k];
    }
}

// The first cut of a near block's TT-SVD left A_b ~ U_r diag(s_r) V_r^T.  The remainder
// C = diag(s_r) V_r^T (r x P, the theta-grid index t = k_1 + p_1 (k_2 + ...) little-endian) is
// compressed by the remaining cuts of TT-SVD with the same delta^2 (the oracle's loop: cut k
// factors the (r_{k-1} p_k) x (p_{k+1} ... p_dtheta) unfolding of the running remainder and keeps
// S V^T), then contracted back: returns W = diag(1 / s_r) C~ (r x P, column-major), so that
// G_{b,1} = A_b V_r = U_r diag(s_r) gives D_b(theta) = G_{b,1} W (v_1 (x) ... (x) v_dtheta), the
// multilinear form of the stored cores (§4.3).
std::vector<double> near_theta_matrix(const double* s, const double* Vr, int P, int r, const int* pt, int dt,
                                      double delta2) {
    std::vector<double> W((size_t)r * P);
    for (int c = 0; c < r; ++c)
        for (int t = 0; t < P; ++t) W[c + (size_t)r * t] = Vr[t + (size_t)P * c];  // V_r^T
    if (dt == 1) return W;
    // running remainder R (rows = r_prev * p_k, cols = rest), Fortran order
    std::vector<double> R((size_t)r * P);
    for (int c = 0; c < r; ++c)
        for (int t = 0; t < P; ++t) R[c + (size_t)r * t] = s[c] * W[c + (size_t)r * t];
    std::vector<std::vector<double>> cores;  // cores[k]: (rprev, p_k, rnext)
    std::vector<int> ranks{r};
    int rprev = r;
    long long rest = P;
    for (int k = 0; k + 1 < dt; ++k) {
        const int rows = rprev * pt[k];
        rest /= pt[k];
        std::vector<double> U, sv, Vt;
        svd_small(rows, (int)rest, R, U, sv, Vt);
        const int kmax = (int)sv.size();
        int rn = choose_rank_sv(sv.data(), kmax, delta2, 0);
        cores.emplace_back(U.begin(), U.begin() + (size_t)rows * rn);
        std::vector<double> Rn((size_t)rn * rest);
        for (int a = 0; a < rn; ++a)
            for (long long j = 0; j < rest; ++j) Rn[a + (size_t)rn * j] = sv[a] * Vt[a + (size_t)kmax * j];
        R.swap(Rn);
        rprev = rn;
        ranks.push_back(rn);
    }
    // contract back: C~ = cores[0] ... cores[dt-2] * R (last core), as an r x P matrix
    std::vector<double> T = R;  // rprev x p_last
    long long cols = pt[dt - 1];
    for (int k = dt - 2; k >= 0; --k) {
        const int rp = ranks[k], pk = pt[k], rn = ranks[k + 1];
        const std::vector<double>& G = cores[k];  // (rp * pk) x rn
        std::vector<double> Tn((size_t)rp * pk * cols, 0.0);
        for (long long j = 0; j < cols; ++j)
            for (int a = 0; a < rn; ++a) {
                const double x = T[a + (size_t)rn * j];
                if (x == 0.0) continue;
                for (int i = 0; i < rp * pk; ++i) Tn[i + (size_t)rp * pk * j] += G[i + (size_t)rp * pk * a] * x;
            }
        T.swap(Tn);
        cols *= pk;
    }
    // T is r x (p_1 ... p_dt) with the row index first, then k_1 fastest: W = diag(1/s) T
    for (int c = 0; c < r; ++c) {
        const double inv = s[c] > 0 ? 1.0 / s[c] : 0.0;
        for (int t = 0; t < P; ++t) W[c + (size_t)r * t] = T[c + (size_t)r * t] * inv;
    }
    return W;
}

}  // namespace ph
