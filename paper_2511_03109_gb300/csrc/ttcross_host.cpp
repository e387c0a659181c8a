// TT-cross with greedy pivots and TT-rounding on the host (FP64): the compressor §2.1 uses for
// the far-field tensors M_k, an alternative to the TT-SVD of the offline build (option
// compressor = 1).  The tensor is never formed: entries are evaluated where the cross asks for
// them (kernel values on the Chebyshev grids), which is what makes it cheaper than TT-SVD for
// large p_s and theta grids.
//
// Greedy cross (Savostyanov 2014, Alg. 2, as §2.1 describes its variant): nested left index sets
// I_k (prefixes over modes 0..k-1) and right sets J_k (suffixes over modes k..q-1), starting from
// one index; each sweep visits the bonds and adds to each one pivot found by partially pivoted
// (rook) search on the residual of the bond's two-mode unfolding; a sweep whose pivot residuals
// are all below eps times the largest entry seen is checked on random entries, and a missed entry
// joins the bonds' sets through its prefixes and suffixes wherever the sets stay nested.  The interpolant
//   T~ = C_1 P_1^{-1} C_2 P_2^{-1} ... C_q,  C_k(i)[a, b] = T(I_k[a], i, J_{k+1}[b]),  P_k = T(I_{k+1}, J_{k+1})
// (C_k P_k^{-1} formed as Q Q[piv]^{-1} from an orthonormal basis Q of C_k's columns, which stays
// accurate when the pivots span many orders of magnitude) is recompressed by TT-rounding
// (Oseledets 2011, Alg. 2) with the truncation rule of TT-SVD.
#include <algorithm>
#include <cmath>
#include <functional>
#include <random>
#include <unordered_map>
#include <vector>

#include "handle.h"

namespace ph {

namespace {

using Tuple = std::vector<int>;

struct Entries {
    const std::vector<int>& dims;
    const std::function<double(const int*)>& f;
    std::unordered_map<unsigned long long, double> cache;
    Entries(const std::vector<int>& d, const std::function<double(const int*)>& fn) : dims(d), f(fn) {}
    double operator()(const int* idx) {
        unsigned long long key = 0;
        for (size_t k = dims.size(); k-- > 0;) key = key * (unsigned long long)dims[k] + (unsigned long long)idx[k];
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
        const double v = f(idx);
        cache.emplace(key, v);
        return v;
    }
};

// Pseudo-inverse of an m x n column-major matrix (singular values below 1e-13 s_1 dropped).
std::vector<double> pinv(int m, int n, const std::vector<double>& A) {
    std::vector<double> U, s, Vt;
    svd_small(m, n, A, U, s, Vt);
    const int k = (int)s.size();
    std::vector<double> X((size_t)n * m, 0.0);  // n x m
    const double cut = (k > 0 ? s[0] : 0.0) * 1e-13;
    for (int c = 0; c < k; ++c) {
        if (!(s[c] > cut)) continue;
        const double inv = 1.0 / s[c];
        for (int j = 0; j < m; ++j) {
            const double u = U[j + (size_t)m * c] * inv;
            if (u == 0.0) continue;
            for (int i = 0; i < n; ++i) X[i + (size_t)n * j] += Vt[c + (size_t)k * i] * u;
        }
    }
    return X;
}

// Inverse of a square r x r column-major matrix by Gauss-Jordan elimination with partial
// pivoting, without truncation: the greedy pivots make the elimination well ordered even when P
// spans many orders of magnitude, where a truncated pseudo-inverse would discard the small pivots
// the cross needs.  A pivot matrix made singular by an enrichment falls back to the pseudo-inverse.
std::vector<double> pivot_inverse(int r, const std::vector<double>& P) {
    std::vector<double> A(P), X((size_t)r * r, 0.0);
    double amax = 0.0;
    for (double v : P) amax = std::max(amax, std::fabs(v));
    for (int i = 0; i < r; ++i) X[i + (size_t)r * i] = 1.0;
    for (int c = 0; c < r; ++c) {
        int piv = c;
        for (int i = c + 1; i < r; ++i)
            if (std::fabs(A[i + (size_t)r * c]) > std::fabs(A[piv + (size_t)r * c])) piv = i;
        if (!(std::fabs(A[piv + (size_t)r * c]) > 1e-300 + 1e-15 * amax)) return pinv(r, r, P);
        if (piv != c)
            for (int k = 0; k < r; ++k) {
                std::swap(A[piv + (size_t)r * k], A[c + (size_t)r * k]);
                std::swap(X[piv + (size_t)r * k], X[c + (size_t)r * k]);
            }
        const double inv = 1.0 / A[c + (size_t)r * c];
        for (int k = 0; k < r; ++k) {
            A[c + (size_t)r * k] *= inv;
            X[c + (size_t)r * k] *= inv;
        }
        for (int i = 0; i < r; ++i) {
            if (i == c) continue;
            const double fct = A[i + (size_t)r * c];
            if (fct == 0.0) continue;
            for (int k = 0; k < r; ++k) {
                A[i + (size_t)r * k] -= fct * A[c + (size_t)r * k];
                X[i + (size_t)r * k] -= fct * X[c + (size_t)r * k];
            }
        }
    }
    return X;
}

// Orthonormal basis Q (m x n, column-major) of the columns of C by Gram-Schmidt with one
// reorthogonalisation pass (the columns of a cross fiber block are linearly independent).
std::vector<double> orth_columns(int m, int n, const std::vector<double>& C) {
    std::vector<double> Q(C);
    for (int j = 0; j < n; ++j) {
        double* qj = &Q[(size_t)m * j];
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < j; ++i) {
                const double* qi = &Q[(size_t)m * i];
                double d = 0.0;
                for (int t = 0; t < m; ++t) d += qi[t] * qj[t];
                for (int t = 0; t < m; ++t) qj[t] -= d * qi[t];
            }
        double nrm = 0.0;
        for (int t = 0; t < m; ++t) nrm += qj[t] * qj[t];
        nrm = std::sqrt(nrm);
        const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
        for (int t = 0; t < m; ++t) qj[t] *= inv;
    }
    return Q;
}

struct Cross {
    const std::vector<int>& dims;
    Entries& T;
    int q;
    std::vector<std::vector<Tuple>> I, J;  // I[k]: prefixes of length k; J[k]: suffixes of length q - k
    Cross(const std::vector<int>& d, Entries& e) : dims(d), T(e), q((int)d.size()) {}

    double at(const Tuple& a, const std::vector<int>& mid, const Tuple& b) {
        Tuple x(a);
        x.insert(x.end(), mid.begin(), mid.end());
        x.insert(x.end(), b.begin(), b.end());
        return T(x.data());
    }
    // C_k = T(I[k][a], i, J[k+1][b]), rows (a, i) with a fastest, column-major
    std::vector<double> fiber(int k) {
        const int r0 = (int)I[k].size(), n = dims[k], r1 = (int)J[k + 1].size();
        std::vector<double> C((size_t)r0 * n * r1);
        for (int b = 0; b < r1; ++b)
            for (int i = 0; i < n; ++i)
                for (int a = 0; a < r0; ++a) C[a + (size_t)r0 * (i + (size_t)n * b)] = at(I[k][a], {i}, J[k + 1][b]);
        return C;
    }
    // G_k = C_k P_k^{-1} for a bond k < q - 1, formed stably as Q Q[piv]^{-1}, Q an orthonormal basis
    // of C_k's columns and piv the rows of C_k that are the pivots I[k+1] (the sets are nested).
    std::vector<double> interp(int k) {
        const int r0 = (int)I[k].size(), n = dims[k], r1 = (int)I[k + 1].size();
        const int m = r0 * n;
        const std::vector<double> Q = orth_columns(m, r1, fiber(k));
        std::vector<double> Qp((size_t)r1 * r1);
        for (int e = 0; e < r1; ++e) {
            const Tuple& pre = I[k + 1][e];
            const Tuple head(pre.begin(), pre.end() - 1);
            const int a = (int)(std::find(I[k].begin(), I[k].end(), head) - I[k].begin());
            const int row = a + r0 * pre.back();
            for (int c = 0; c < r1; ++c) Qp[e + (size_t)r1 * c] = Q[row + (size_t)m * c];
        }
        const std::vector<double> Qi = pivot_inverse(r1, Qp);  // r1 x r1
        std::vector<double> G((size_t)m * r1, 0.0);
        for (int e = 0; e < r1; ++e)
            for (int c = 0; c < r1; ++c) {
                const double v = Qi[c + (size_t)r1 * e];
                if (v == 0.0) continue;
                for (int row = 0; row < m; ++row) G[row + (size_t)m * e] += Q[row + (size_t)m * c] * v;
            }
        return G;
    }
    // residual of bond k's super core on column (j, b): rows (a, i) with a fastest; Gk = interp(k)
    std::vector<double> residual_col(int k, int j, int b, const std::vector<double>& Gk) {
        const int ra = (int)I[k].size(), n = dims[k], r = (int)I[k + 1].size();
        const int m = ra * n;
        std::vector<double> right(r), out((size_t)m);
        for (int e = 0; e < r; ++e) right[e] = at(I[k + 1][e], {j}, J[k + 2][b]);
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < ra; ++a) {
                const int row = a + ra * i;
                double apx = 0.0;
                for (int e = 0; e < r; ++e) apx += Gk[row + (size_t)m * e] * right[e];
                out[row] = at(I[k][a], {i, j}, J[k + 2][b]) - apx;
            }
        return out;
    }
    // residual on row (a, i): columns (j, b) with j fastest
    std::vector<double> residual_row(int k, int a, int i, const std::vector<double>& Gk) {
        const int ra = (int)I[k].size(), n1 = dims[k + 1], rb = (int)J[k + 2].size(), r = (int)I[k + 1].size();
        const int m = ra * dims[k], row = a + ra * i;
        std::vector<double> out((size_t)n1 * rb);
        for (int b = 0; b < rb; ++b)
            for (int j = 0; j < n1; ++j) {
                double apx = 0.0;
                for (int e = 0; e < r; ++e) apx += Gk[row + (size_t)m * e] * at(I[k + 1][e], {j}, J[k + 2][b]);
                out[j + (size_t)n1 * b] = at(I[k][a], {i, j}, J[k + 2][b]) - apx;
            }
        return out;
    }
    // the TT cores: G_k (k < q - 1) and C_q (Fortran (r_k, n_k, r_{k+1}))
    std::vector<std::vector<double>> cores() {
        std::vector<std::vector<double>> G(q);
        for (int k = 0; k < q; ++k) G[k] = (k < q - 1) ? interp(k) : fiber(k);
        return G;
    }
};

double tt_entry(const std::vector<std::vector<double>>& G, const std::vector<int>& dims, const int* x) {
    std::vector<double> v(1, 1.0);
    for (size_t k = 0; k < G.size(); ++k) {
        const int r0 = (int)v.size(), n = dims[k];
        const int r1 = (int)(G[k].size() / ((size_t)r0 * n));
        std::vector<double> w(r1, 0.0);
        for (int b = 0; b < r1; ++b)
            for (int a = 0; a < r0; ++a) w[b] += v[a] * G[k][a + (size_t)r0 * (x[k] + (size_t)n * b)];
        v.swap(w);
    }
    return v[0];
}

}  // namespace

// kappa(x, y; theta) of the ph_kernel enumeration on the host (the formulas of the kernel table in
// ph.h), for the entries the cross asks for.
double kappa_host(int kernel, const double* x, const double* y, const double* th, int d) {
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) r2 += (x[k] - y[k]) * (x[k] - y[k]);
    const double l = th[0];
    switch (kernel) {
        case PH_KERNEL_GAUSS: return std::exp(-r2 / (2.0 * l * l));
        case PH_KERNEL_MATERN32: {
            const double s = std::sqrt(3.0 * r2) / l;
            return (1.0 + s) * std::exp(-s);
        }
        case PH_KERNEL_MATERN52: {
            const double s = std::sqrt(5.0 * r2) / l;
            return (1.0 + s + s * s / 3.0) * std::exp(-s);
        }
        case PH_KERNEL_ANISO_GAUSS: {
            double q = 0.0;
            for (int k = 0; k < d; ++k) q += (x[k] - y[k]) * (x[k] - y[k]) / (2.0 * th[k] * th[k]);
            return std::exp(-q);
        }
        case PH_KERNEL_SE: return std::exp(-r2 / (l * l));
        case PH_KERNEL_EXPONENTIAL: return std::exp(-std::sqrt(r2) / l);
        case PH_KERNEL_MULTIQUADRIC: return std::sqrt(1.0 + r2 / (l * l));
        case PH_KERNEL_POLY: return 1.0 + l * r2 + l * l * r2 * r2;
        case PH_KERNEL_POLY2: return 1.0 + th[0] * r2 + th[1] * th[1] * r2 * r2;
        case PH_KERNEL_POLYXY: {
            double dot = 0.0;
            for (int k = 0; k < d; ++k) dot += x[k] * y[k];
            return (1.0 + dot) * (1.0 + dot) * (1.0 + l);
        }
    }
    return 0.0;
}

// TT-rounding of cores (Fortran (r_k, n_k, r_{k+1})): right-to-left orthogonalisation, then
// left-to-right truncated SVDs with delta^2 = eps^2 ||T||^2 / (q - 1) and the rank rule of TT-SVD.
void tt_round(std::vector<std::vector<double>>& G, const std::vector<int>& dims, double eps, int cap,
              std::vector<int>& ranks) {
    const int q = (int)G.size();
    std::vector<int> r(q + 1, 1);
    for (int k = 0; k < q; ++k) r[k + 1] = (int)(G[k].size() / ((size_t)r[k] * dims[k]));
    for (int k = q - 1; k > 0; --k) {
        // unfolding (r_k x n_k r_{k+1})^T = U S V^T: core k <- U^T, core k-1 absorbs V S
        const int r0 = r[k], n = dims[k], r1 = r[k + 1];
        const int m = n * r1;
        std::vector<double> At((size_t)m * r0);
        for (int a = 0; a < r0; ++a)
            for (int col = 0; col < m; ++col) At[col + (size_t)m * a] = G[k][a + (size_t)r0 * col];
        std::vector<double> U, s, Vt;
        svd_small(m, r0, At, U, s, Vt);
        const int kk = (int)s.size();
        std::vector<double> Gk((size_t)kk * m);
        for (int c = 0; c < kk; ++c)
            for (int col = 0; col < m; ++col) Gk[c + (size_t)kk * col] = U[col + (size_t)m * c];
        // core k-1 (r_{k-1}, n_{k-1}, r0) times (V S) (r0 x kk)
        const int p0 = r[k - 1], np = dims[k - 1];
        const size_t rows = (size_t)p0 * np;
        std::vector<double> Gp(rows * kk, 0.0);
        for (int c = 0; c < kk; ++c)
            for (int a = 0; a < r0; ++a) {
                const double vs = Vt[c + (size_t)kk * a] * s[c];
                if (vs == 0.0) continue;
                for (size_t row = 0; row < rows; ++row) Gp[row + rows * c] += G[k - 1][row + rows * a] * vs;
            }
        G[k].swap(Gk);
        G[k - 1].swap(Gp);
        r[k] = kk;
    }
    double nrm2 = 0.0;
    for (double x : G[0]) nrm2 += x * x;
    const double delta2 = eps * eps * nrm2 / std::max(1, q - 1);
    for (int k = 0; k + 1 < q; ++k) {
        const int r0 = r[k], n = dims[k], r1 = r[k + 1];
        const int m = r0 * n;
        std::vector<double> U, s, Vt;
        svd_small(m, r1, G[k], U, s, Vt);
        const int kk = (int)s.size();
        const int rk = choose_rank_sv(s.data(), kk, delta2, cap);
        G[k].assign(U.begin(), U.begin() + (size_t)m * rk);
        // next core <- (S V^T)_{rk x r1} times core k+1 (r1, n_{k+1}, r_{k+2})
        const int n1 = dims[k + 1], r2 = r[k + 2];
        std::vector<double> Gn((size_t)rk * n1 * r2, 0.0);
        for (int b = 0; b < n1 * r2; ++b)
            for (int c = 0; c < r1; ++c) {
                const double g = G[k + 1][c + (size_t)r1 * b];
                if (g == 0.0) continue;
                for (int a = 0; a < rk; ++a) Gn[a + (size_t)rk * b] += s[a] * Vt[a + (size_t)kk * c] * g;
            }
        G[k + 1].swap(Gn);
        r[k + 1] = rk;
    }
    ranks = r;
}

// Greedy TT-cross of the tensor with entries f, then TT-rounding; returns the number of distinct
// entries evaluated.
long long tt_cross_round(const std::vector<int>& dims, const std::function<double(const int*)>& f, double eps, int cap,
                         unsigned long long seed, std::vector<std::vector<double>>& cores, std::vector<int>& ranks) {
    const int q = (int)dims.size();
    Entries T(dims, f);
    std::mt19937_64 gen(seed);
    auto rnd = [&](int n) { return (int)(gen() % (unsigned long long)n); };
    // the single starting index: the largest of 64 random entries
    Tuple start(q);
    double vmax = 0.0;
    for (int t = 0; t < 64; ++t) {
        Tuple x(q);
        for (int k = 0; k < q; ++k) x[k] = rnd(dims[k]);
        const double v = std::fabs(T(x.data()));
        if (t == 0 || v > vmax) {
            vmax = v;
            start = x;
        }
    }
    Cross X(dims, T);
    X.I.resize(q + 1);
    X.J.resize(q + 1);
    for (int k = 0; k <= q; ++k) {
        X.I[k].push_back(Tuple(start.begin(), start.begin() + k));
        X.J[k].push_back(Tuple(start.begin() + k, start.end()));
    }
    const int cap_r = cap > 0 ? cap : 1 << 20;
    for (int sweep = 0; sweep < 400; ++sweep) {
        double worst = 0.0;
        for (int k = 0; k + 1 < q; ++k) {
            const int rows_max = (int)X.I[k].size() * dims[k], cols_max = dims[k + 1] * (int)X.J[k + 2].size();
            if ((int)X.I[k + 1].size() >= std::min(std::min(rows_max, cols_max), cap_r)) continue;
            const std::vector<double> Gk = X.interp(k);
            int j = rnd(dims[k + 1]), b = rnd((int)X.J[k + 2].size());
            double best = 0.0;
            int ba = -1, bi = -1, bj = -1, bb = -1;
            for (int step = 0; step < 3; ++step) {
                const std::vector<double> e = X.residual_col(k, j, b, Gk);
                int ir = 0;
                for (size_t t = 1; t < e.size(); ++t)
                    if (std::fabs(e[t]) > std::fabs(e[ir])) ir = (int)t;
                const int a = ir % (int)X.I[k].size(), i = ir / (int)X.I[k].size();
                const std::vector<double> er = X.residual_row(k, a, i, Gk);
                int jc = 0;
                for (size_t t = 1; t < er.size(); ++t)
                    if (std::fabs(er[t]) > std::fabs(er[jc])) jc = (int)t;
                j = jc % dims[k + 1];
                b = jc / dims[k + 1];
                vmax = std::max(vmax, std::fabs(X.at(X.I[k][a], {i, j}, X.J[k + 2][b])));
                if (std::fabs(er[jc]) > best) {
                    best = std::fabs(er[jc]);
                    ba = a; bi = i; bj = j; bb = b;
                }
            }
            worst = std::max(worst, best);
            if (ba < 0 || best <= 0.1 * eps * vmax) continue;  // no pivots below the target accuracy
            Tuple ni(X.I[k][ba]);
            ni.push_back(bi);
            Tuple nj(1, bj);
            nj.insert(nj.end(), X.J[k + 2][bb].begin(), X.J[k + 2][bb].end());
            if (std::find(X.I[k + 1].begin(), X.I[k + 1].end(), ni) != X.I[k + 1].end() ||
                std::find(X.J[k + 1].begin(), X.J[k + 1].end(), nj) != X.J[k + 1].end())
                continue;
            X.I[k + 1].push_back(ni);
            X.J[k + 1].push_back(nj);
        }
        if (worst > eps * vmax) continue;
        // random check of the interpolant; a missed entry joins every bond's sets
        const std::vector<std::vector<double>> G = X.cores();
        double emax = -1.0;
        Tuple wx(q);
        for (int t = 0; t < 64; ++t) {
            Tuple x(q);
            for (int k = 0; k < q; ++k) x[k] = rnd(dims[k]);
            const double ex = T(x.data());
            vmax = std::max(vmax, std::fabs(ex));
            const double e = std::fabs(tt_entry(G, dims, x.data()) - ex);
            if (e > emax) {
                emax = e;
                wx = x;
            }
        }
        if (emax <= eps * vmax) break;
        // bonds that take the pair (prefix, suffix) of the missed entry: both new, room left, and
        // the sets stay nested (the pair's shorter prefix / suffix present or added with it)
        auto has = [](const std::vector<Tuple>& set, const Tuple& t) {
            return std::find(set.begin(), set.end(), t) != set.end();
        };
        std::vector<char> take(q, 0);
        for (int k = 0; k + 1 < q; ++k) {
            const int rows_max = (int)X.I[k].size() * dims[k], cols_max = dims[k + 1] * (int)X.J[k + 2].size();
            take[k] = (int)X.I[k + 1].size() < std::min(std::min(rows_max, cols_max), cap_r) &&
                      !has(X.I[k + 1], Tuple(wx.begin(), wx.begin() + k + 1)) &&
                      !has(X.J[k + 1], Tuple(wx.begin() + k + 1, wx.end()));
        }
        for (bool changed = true; changed;) {
            changed = false;
            for (int k = 0; k + 1 < q; ++k) {
                if (!take[k]) continue;
                const bool left_ok = (k == 0) || take[k - 1] || has(X.I[k], Tuple(wx.begin(), wx.begin() + k));
                const bool right_ok = (k + 2 >= q) || take[k + 1] || has(X.J[k + 2], Tuple(wx.begin() + k + 2, wx.end()));
                if (!left_ok || !right_ok) {
                    take[k] = 0;
                    changed = true;
                }
            }
        }
        bool grown = false;
        for (int k = 0; k + 1 < q; ++k)
            if (take[k]) {
                X.I[k + 1].push_back(Tuple(wx.begin(), wx.begin() + k + 1));
                X.J[k + 1].push_back(Tuple(wx.begin() + k + 1, wx.end()));
                grown = true;
            }
        if (!grown) break;
    }
    cores = X.cores();
    tt_round(cores, dims, eps, cap, ranks);
    return (long long)T.cache.size();
}

}  // namespace ph

namespace ph {

// The far-field tensor M_k of one translation class by TT-cross (the offline build's route for
// compressor = 1): modes (i_1..i_d, k_1..k_dtheta, j_1..j_d), entries kappa(x_i, y_j; theta_k)
// with x on the Chebyshev grid of the target box [s_lo, s_hi], y on the source box's, theta on the
// far-field theta nodes (theta_nodes: dtheta rows of kMaxPTheta).
long long far_cross(int kernel, int d, int dt, int ps, const int* pt, const double* s_lo, const double* s_hi,
                    const double* t_lo, const double* t_hi, const double* theta_nodes, double eps, int cap,
                    unsigned long long seed, std::vector<std::vector<double>>& cores, std::vector<int>& ranks) {
    std::vector<int> dims;
    for (int k = 0; k < d; ++k) dims.push_back(ps);
    for (int k = 0; k < dt; ++k) dims.push_back(pt[k]);
    for (int k = 0; k < d; ++k) dims.push_back(ps);
    std::vector<double> xs((size_t)kMaxDim * kMaxPs), yt((size_t)kMaxDim * kMaxPs);
    for (int k = 0; k < d; ++k) {
        cheb_nodes(s_lo[k], s_hi[k], ps, &xs[(size_t)k * kMaxPs]);
        cheb_nodes(t_lo[k], t_hi[k], ps, &yt[(size_t)k * kMaxPs]);
    }
    std::function<double(const int*)> f = [&](const int* x) {
        double a[kMaxDim], b[kMaxDim], th[kMaxDim];
        for (int k = 0; k < d; ++k) {
            a[k] = xs[(size_t)k * kMaxPs + x[k]];
            b[k] = yt[(size_t)k * kMaxPs + x[d + dt + k]];
        }
        for (int k = 0; k < dt; ++k) th[k] = theta_nodes[(size_t)k * kMaxPTheta + x[d + k]];
        return kappa_host(kernel, a, b, th, d);
    };
    return tt_cross_round(dims, f, eps, cap, seed, cores, ranks);
}

}  // namespace ph

// Test hook (no GPU): TT-cross + TT-rounding of a dense host tensor (Fortran order, dims[0]
// fastest); writes the ranks (q + 1 values) and the reconstructed tensor, and the number of
// distinct entries the cross evaluated.  Declared in include/ph.h.
extern "C" ph_status ph_tt_cross_check(int q, const int* dims, const double* tensor, double eps, int cap,
                                       int* ranks, double* approx, long* evals) {
    if (q < 2 || q > 16 || !dims || !tensor || !ranks || !approx || !evals || !(eps > 0))
        return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_tt_cross_check: invalid argument");
    return ph::guarded(nullptr, [&]() -> ph_status {
        std::vector<int> d(dims, dims + q);
        for (int k = 0; k < q; ++k)
            if (d[k] < 1) throw ph::Error(PH_ERR_INVALID_ARG, "ph_tt_cross_check: bad dimension");
        std::function<double(const int*)> f = [&](const int* x) {
            long long off = 0, stride = 1;
            for (int k = 0; k < q; ++k) {
                off += (long long)x[k] * stride;
                stride *= d[k];
            }
            return tensor[off];
        };
        std::vector<std::vector<double>> G;
        std::vector<int> r;
        *evals = (long)ph::tt_cross_round(d, f, eps, cap, 12345ull, G, r);
        for (int k = 0; k <= q; ++k) ranks[k] = r[k];
        long long total = 1;
        for (int k = 0; k < q; ++k) total *= d[k];
        std::vector<int> x(q, 0);
        for (long long t = 0; t < total; ++t) {
            long long rest = t;
            for (int k = 0; k < q; ++k) {
                x[k] = (int)(rest % d[k]);
                rest /= d[k];
            }
            approx[t] = ph::tt_entry(G, d, x.data());
        }
        return PH_OK;
    });
}

// Test hook (no GPU): the offline build's TT-cross of one far-field tensor (far_cross) for the
// boxes [s_lo, s_hi] (target) and [t_lo, t_hi] (source) of [0,1]^d and the parameter box
// [theta_lo, theta_hi] with degree[k] + 1 Chebyshev nodes per dimension; writes the ranks
// (2d + dtheta + 1 values) and the reconstructed tensor (Fortran order, modes i, theta, j).
// Declared in include/ph.h.
extern "C" ph_status ph_far_cross_check(int kernel, int d, int dtheta, int p_s, const int* degree,
                                        const double* s_lo, const double* s_hi, const double* t_lo,
                                        const double* t_hi, const double* theta_lo, const double* theta_hi,
                                        double eps, int cap, int* ranks, double* approx) {
    if (kernel < 0 || kernel > PH_KERNEL_POLY2 || d < 1 || d > 3 || dtheta < 1 || dtheta > 3 || p_s < 1 ||
        p_s > ph::kMaxPs || !degree || !s_lo || !s_hi || !t_lo || !t_hi || !theta_lo || !theta_hi || !ranks ||
        !approx || !(eps > 0))
        return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_far_cross_check: invalid argument");
    return ph::guarded(nullptr, [&]() -> ph_status {
        int pt[ph::kMaxDim] = {1, 1, 1};
        std::vector<double> nodes((size_t)ph::kMaxDim * ph::kMaxPTheta, 0.0);
        for (int k = 0; k < dtheta; ++k) {
            if (degree[k] < 0 || degree[k] + 1 > ph::kMaxPTheta)
                throw ph::Error(PH_ERR_INVALID_ARG, "ph_far_cross_check: bad degree");
            pt[k] = degree[k] + 1;
            ph::cheb_nodes(theta_lo[k], theta_hi[k], pt[k], &nodes[(size_t)k * ph::kMaxPTheta]);
        }
        std::vector<std::vector<double>> G;
        std::vector<int> r;
        ph::far_cross(kernel, d, dtheta, p_s, pt, s_lo, s_hi, t_lo, t_hi, nodes.data(), eps, cap, 7ull, G, r);
        const int q = 2 * d + dtheta;
        for (int k = 0; k <= q; ++k) ranks[k] = r[k];
        std::vector<int> dims;
        for (int k = 0; k < d; ++k) dims.push_back(p_s);
        for (int k = 0; k < dtheta; ++k) dims.push_back(pt[k]);
        for (int k = 0; k < d; ++k) dims.push_back(p_s);
        long long total = 1;
        for (int v : dims) total *= v;
        std::vector<int> x(q, 0);
        for (long long t = 0; t < total; ++t) {
            long long rest = t;
            for (int k = 0; k < q; ++k) {
                x[k] = (int)(rest % dims[k]);
                rest /= dims[k];
            }
            approx[t] = ph::tt_entry(G, dims, x.data());
        }
        return PH_OK;
    });
}
