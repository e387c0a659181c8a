// Host planning: cluster tree (§3.2), admissibility (§3.4, App. A.2), block
// cluster tree (Alg. ConstructBlockClusterTree) and translation classes of far
// blocks (§5.2).  Pure C++, no CUDA.
#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>
#include <tuple>

#include "ph_internal.h"

namespace ph {

namespace {

// Equality counts as admissible; the slack keeps exact ties (eta = sqrt(d) at
// a one-box gap) independent of rounding.
constexpr double kAdmSlack = 1e-12;
constexpr int kAdaptiveMaxDepth = 20;

double diam(const Node& a, int d) {
    double s = 0;
    for (int k = 0; k < d; ++k) s += (a.hi[k] - a.lo[k]) * (a.hi[k] - a.lo[k]);
    return std::sqrt(s);
}

double dist(const Node& a, const Node& b, int d) {
    double s = 0;
    for (int k = 0; k < d; ++k) {
        double g1 = std::max(0.0, a.lo[k] - b.hi[k]);
        double g2 = std::max(0.0, b.lo[k] - a.hi[k]);
        s += g1 * g1 + g2 * g2;
    }
    return std::sqrt(s);
}

bool admissible(const Node& a, const Node& b, int d, double eta) {
    return std::max(diam(a, d), diam(b, d)) <= eta * dist(a, b, d) * (1.0 + kAdmSlack);
}

struct Builder {
    const double* P;
    int d;
    int l_max;
    Plan& plan;
    std::vector<int> order;  // cluster order being assembled
    int leaf_size = 0;       // > 0: adaptive tree (split while more points than this, level < 20)

    // Splits node `id` holding the original indices `idx` (ascending).
    void split(int id, std::vector<int>& idx) {
        Node& nd = plan.nodes[id];
        nd.begin = (int)order.size();
        const bool leaf = leaf_size > 0 ? ((int)idx.size() <= leaf_size || nd.level >= kAdaptiveMaxDepth)
                                        : nd.level >= l_max;
        if (leaf) {
            order.insert(order.end(), idx.begin(), idx.end());
            nd.end = (int)order.size();
            nd.leaf = (int)plan.leaves.size();
            plan.leaves.push_back(id);
            plan.depth = std::max(plan.depth, nd.level);
            return;
        }
        double mid[kMaxDim];
        for (int k = 0; k < d; ++k) mid[k] = 0.5 * (nd.lo[k] + nd.hi[k]);
        // children in little-endian order of their halves (dimension 1 fastest)
        std::vector<std::vector<int>> parts(1 << d);
        for (int i : idx) {
            int code = 0;
            for (int k = 0; k < d; ++k)
                if (P[(long)i * d + k] > mid[k]) code |= 1 << k;  // (mid, b] is the high half
            parts[code].push_back(i);
        }
        const int level = nd.level;
        double lo[kMaxDim], hi[kMaxDim];
        for (int k = 0; k < d; ++k) { lo[k] = nd.lo[k]; hi[k] = nd.hi[k]; }
        for (int code = 0; code < (1 << d); ++code) {
            if (parts[code].empty()) continue;  // empty children carry no rows or columns
            Node ch;
            ch.level = level + 1;
            ch.parent = id;
            ch.halves = code;
            for (int k = 0; k < d; ++k) {
                if (code & (1 << k)) { ch.lo[k] = mid[k]; ch.hi[k] = hi[k]; }
                else { ch.lo[k] = lo[k]; ch.hi[k] = mid[k]; }
            }
            int cid = (int)plan.nodes.size();
            plan.nodes.push_back(ch);
            plan.nodes[id].children.push_back(cid);
            split(cid, parts[code]);
        }
        plan.nodes[id].end = (int)order.size();
    }
};

void block_recurse(Plan& plan, int s, int t, double eta, std::vector<std::pair<int, int>>& near,
                   std::vector<std::pair<int, int>>& far) {
    const Node& a = plan.nodes[s];
    const Node& b = plan.nodes[t];
    bool adm = admissible(a, b, plan.d, eta);
    if (!adm && !a.children.empty() && !b.children.empty()) {
        for (int sc : a.children)
            for (int tc : b.children) block_recurse(plan, sc, tc, eta, near, far);
    } else if (adm) {
        far.emplace_back(s, t);
    } else {
        near.emplace_back(s, t);
    }
}

}  // namespace

bool kernel_translation_invariant(ph_kernel k) { return k != PH_KERNEL_POLYXY; }

void build_plan(const double* points, long n, int d, int l_max, double eta, bool dedup, Plan& plan, int leaf_size) {
    if (d < 1 || d > kMaxDim) throw std::invalid_argument("d must be 1..3");
    if (n < 1) throw std::invalid_argument("n must be positive");
    for (long i = 0; i < n * d; ++i) {
        double x = points[i];
        if (!(x >= 0.0 && x <= 1.0)) throw std::invalid_argument("points must lie in [0,1]^d");
    }
    plan = Plan();
    plan.d = d;
    plan.n = n;
    Node root;
    for (int k = 0; k < d; ++k) { root.lo[k] = 0.0; root.hi[k] = 1.0; }
    plan.nodes.push_back(root);
    std::vector<int> idx(n);
    for (long i = 0; i < n; ++i) idx[i] = (int)i;
    Builder b{points, d, l_max, plan, {}, leaf_size};
    b.order.reserve(n);
    b.split(0, idx);
    plan.perm = std::move(b.order);

    std::vector<std::pair<int, int>> near, far;
    block_recurse(plan, 0, 0, eta, near, far);

    // near blocks grouped by target leaf (targets in cluster order, sources by node id)
    std::stable_sort(near.begin(), near.end(), [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        int lx = plan.nodes[x.first].leaf, ly = plan.nodes[y.first].leaf;
        return lx != ly ? lx < ly : x.second < y.second;
    });
    plan.near_by_leaf.assign(plan.leaves.size() + 1, 0);
    for (auto& p : near) {
        // an adaptive tree also has near blocks between a leaf and an inner cluster: they are
        // planned (counted) but not grouped by leaf; the offline build refuses such plans
        const bool leaves = plan.nodes[p.first].leaf >= 0 && plan.nodes[p.second].leaf >= 0;
        if (!leaves) {
            if (leaf_size <= 0) throw std::logic_error("near block between non-leaf clusters");
            plan.inner_near_s.push_back(p.first);
            plan.inner_near_t.push_back(p.second);
            continue;
        }
        plan.near_s.push_back(p.first);
        plan.near_t.push_back(p.second);
        plan.near_by_leaf[plan.nodes[p.first].leaf + 1]++;
    }
    for (size_t l = 0; l < plan.leaves.size(); ++l) plan.near_by_leaf[l + 1] += plan.near_by_leaf[l];

    // far blocks grouped by target node
    std::stable_sort(far.begin(), far.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        return x.first != y.first ? x.first < y.first : x.second < y.second;
    });
    std::map<std::vector<long>, int> classes;
    for (size_t i = 0; i < far.size(); ++i) {
        int s = far[i].first, t = far[i].second;
        if (plan.far_targets.empty() || plan.far_targets.back() != s) {
            plan.far_targets.push_back(s);
            plan.far_by_target.push_back((int)i);
        }
        plan.far_s.push_back(s);
        plan.far_t.push_back(t);
        int key;
        if (dedup) {
            // class = (both levels, offset of B_t from B_s in units of the finer box side): with
            // a translation-invariant kernel M_b depends only on it (§5.2); in a uniform tree both
            // levels are equal and this is (level, offset in box sides)
            const Node& a = plan.nodes[s];
            const Node& c = plan.nodes[t];
            const double unit = std::min(a.hi[0] - a.lo[0], c.hi[0] - c.lo[0]);
            std::vector<long> k{a.level, c.level};
            for (int q = 0; q < d; ++q) k.push_back(std::lround((c.lo[q] - a.lo[q]) / unit));
            auto it = classes.find(k);
            if (it == classes.end()) {
                key = (int)plan.key_rep.size();
                classes.emplace(k, key);
                plan.key_rep.push_back((int)i);
            } else {
                key = it->second;
            }
        } else {
            key = (int)plan.key_rep.size();
            plan.key_rep.push_back((int)i);
        }
        plan.far_key.push_back(key);
    }
    plan.far_by_target.push_back((int)far.size());
}

void cheb_nodes(double a, double b, int p, double* out) {
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= p; ++k)
        out[k - 1] = 0.5 * (a + b) - 0.5 * (b - a) * std::cos((2.0 * k - 1.0) * pi / (2.0 * p));
}

void bary_weights(const double* nodes, int p, double* w) {
    double mx = 0;
    for (int k = 0; k < p; ++k) {
        double prod = 1.0;
        for (int j = 0; j < p; ++j)
            if (j != k) prod *= (nodes[k] - nodes[j]);
        w[k] = 1.0 / prod;
        mx = std::max(mx, std::fabs(w[k]));
    }
    for (int k = 0; k < p; ++k) w[k] /= mx;
}

void lagrange_bary(const double* nodes, const double* w, int p, double x, double* out) {
    for (int k = 0; k < p; ++k)
        if (x == nodes[k]) {
            for (int j = 0; j < p; ++j) out[j] = (j == k) ? 1.0 : 0.0;
            return;
        }
    double den = 0;
    for (int k = 0; k < p; ++k) {
        out[k] = w[k] / (x - nodes[k]);
        den += out[k];
    }
    for (int k = 0; k < p; ++k) out[k] /= den;
}

}  // namespace ph
