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
// joins every bond's sets through its prefixes and suffixes.  The interpolant
//   T~ = C_1 P_1^+ C_2 P_2^+ ... C_q,  C_k(i)[a, b] = T(I_k[a], i, J_{k+1}[b]),  P_k = T(I_{k+1}, J_{k+1})
// is recompressed by TT-rounding (Oseledets 2011, Alg. 2) with the truncation rule of TT-SVD.
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
    // P_k = T(I[k+1], J[k+1]) (column-major) and its pseudo-inverse
    std::vector<double> pivots_pinv(int k) {
        const int r = (int)I[k + 1].size();
        std::vector<double> P((size_t)r * r);
        for (int b = 0; b < r; ++b)
            for (int a = 0; a < r; ++a) P[a + (size_t)r * b] = at(I[k + 1][a], {}, J[k + 1][b]);
        return pinv(r, r, P);
    }
    // residual of bond k's super core on column (j, b): rows (a, i) with a fastest
    std::vector<double> residual_col(int k, int j, int b, const std::vector<double>& Pi) {
        const int ra = (int)I[k].size(), n = dims[k], r = (int)I[k + 1].size();
        std::vector<double> right(r), w(r, 0.0), out((size_t)ra * n);
        for (int c = 0; c < r; ++c) right[c] = at(I[k + 1][c], {j}, J[k + 2][b]);
        for (int c = 0; c < r; ++c)
            for (int e = 0; e < r; ++e) w[c] += Pi[c + (size_t)r * e] * right[e];
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < ra; ++a) {
                double apx = 0.0;
                for (int c = 0; c < r; ++c) apx += at(I[k][a], {i}, J[k + 1][c]) * w[c];
                out[a + (size_t)ra * i] = at(I[k][a], {i, j}, J[k + 2][b]) - apx;
            }
        return out;
    }
    // residual on row (a, i): columns (j, b) with j fastest
    std::vector<double> residual_row(int k, int a, int i, const std::vector<double>& Pi) {
        const int n1 = dims[k + 1], rb = (int)J[k + 2].size(), r = (int)I[k + 1].size();
        std::vector<double> left(r), w(r, 0.0), out((size_t)n1 * rb);
        for (int c = 0; c < r; ++c) left[c] = at(I[k][a], {i}, J[k + 1][c]);
        for (int e = 0; e < r; ++e)
            for (int c = 0; c < r; ++c) w[e] += left[c] * Pi[c + (size_t)r * e];  // (P^+)[c][e]
        for (int b = 0; b < rb; ++b)
            for (int j = 0; j < n1; ++j) {
                double apx = 0.0;
                for (int e = 0; e < r; ++e) apx += w[e] * at(I[k + 1][e], {j}, J[k + 2][b]);
                out[j + (size_t)n1 * b] = at(I[k][a], {i, j}, J[k + 2][b]) - apx;
            }
        return out;
    }
    // cores C_k P_k^+ (Fortran (r_k, n_k, r_{k+1}))
    std::vector<std::vector<double>> cores() {
        std::vector<std::vector<double>> G(q);
        for (int k = 0; k < q; ++k) {
            const int r0 = (int)I[k].size(), n = dims[k], r1 = (int)J[k + 1].size();
            std::vector<double> C((size_t)r0 * n * r1);
            for (int b = 0; b < r1; ++b)
                for (int i = 0; i < n; ++i)
                    for (int a = 0; a < r0; ++a) C[a + (size_t)r0 * (i + (size_t)n * b)] = at(I[k][a], {i}, J[k + 1][b]);
            if (k < q - 1) {
                const std::vector<double> Pi = pivots_pinv(k);  // r1 x r1
                std::vector<double> Gk(C.size(), 0.0);
                const size_t rows = (size_t)r0 * n;
                for (int b = 0; b < r1; ++b)
                    for (int c = 0; c < r1; ++c) {
                        const double p = Pi[c + (size_t)r1 * b];
                        if (p == 0.0) continue;
                        for (size_t row = 0; row < rows; ++row) Gk[row + rows * b] += C[row + rows * c] * p;
                    }
                G[k].swap(Gk);
            } else {
                G[k].swap(C);
            }
        }
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
            const std::vector<double> Pi = X.pivots_pinv(k);
            int j = rnd(dims[k + 1]), b = rnd((int)X.J[k + 2].size());
            double best = 0.0;
            int ba = -1, bi = -1, bj = -1, bb = -1;
            for (int step = 0; step < 3; ++step) {
                const std::vector<double> e = X.residual_col(k, j, b, Pi);
                int ir = 0;
                for (size_t t = 1; t < e.size(); ++t)
                    if (std::fabs(e[t]) > std::fabs(e[ir])) ir = (int)t;
                const int a = ir % (int)X.I[k].size(), i = ir / (int)X.I[k].size();
                const std::vector<double> er = X.residual_row(k, a, i, Pi);
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
            if (ba < 0 || best <= 1e-14 * vmax) continue;
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
        bool grown = false;
        for (int k = 0; k + 1 < q; ++k) {
            const int rows_max = (int)X.I[k].size() * dims[k], cols_max = dims[k + 1] * (int)X.J[k + 2].size();
            if ((int)X.I[k + 1].size() >= std::min(std::min(rows_max + 1, cols_max + 1), cap_r)) continue;
            Tuple ni(wx.begin(), wx.begin() + k + 1), nj(wx.begin() + k + 1, wx.end());
            if (std::find(X.I[k + 1].begin(), X.I[k + 1].end(), ni) != X.I[k + 1].end() ||
                std::find(X.J[k + 1].begin(), X.J[k + 1].end(), nj) != X.J[k + 1].end())
                continue;
            X.I[k + 1].push_back(ni);
            X.J[k + 1].push_back(nj);
            grown = true;
        }
        if (!grown) break;
    }
    cores = X.cores();
    tt_round(cores, dims, eps, cap, ranks);
    return (long long)T.cache.size();
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
