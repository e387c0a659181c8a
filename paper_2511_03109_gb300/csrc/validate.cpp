// Consistency checks of a handle's host state: every index the online kernels follow and
// every offset they add to an arena pointer is checked against the table or arena it points
// into.  ph_load runs them on a file before anything reaches the device (a file whose
// lengths are consistent but whose contents are corrupt, or come from another build, is
// refused with PH_ERR_IO instead of letting a kernel read out of bounds); ph_offline_build
// runs them on what it built.
#include <algorithm>
#include <string>
#include <vector>

#include "handle.h"

namespace ph {

namespace {

[[noreturn]] void bad(const std::string& what) { throw Error(PH_ERR_IO, "inconsistent handle data: " + what); }

void need(bool ok, const char* what) {
    if (!ok) bad(what);
}

template <typename V>
void need_size(const std::vector<V>& v, size_t n, const char* what) {
    if (v.size() != n) bad(std::string(what) + " has " + std::to_string(v.size()) + " entries, expected " +
                           std::to_string(n));
}

// [off, off + len) inside [0, cap)
bool in_range(long long off, long long len, long long cap) { return off >= 0 && len >= 0 && off <= cap && len <= cap - off; }

// CSR offsets: size count + 1, starting at 0, non-decreasing, ending at total.
void need_csr(const std::vector<int>& off, size_t count, long long total, const char* what) {
    need_size(off, count + 1, what);
    need(off[0] == 0 && (long long)off[count] == total, what);
    for (size_t i = 0; i < count; ++i) need(off[i] <= off[i + 1], what);
}

}  // namespace

void validate_handle(const ph_handle& h, const std::vector<size_t>& arena_bytes) {
    const ph_build_opts& o = h.opts;
    const Plan& p = h.plan;
    // options and the quantities derived from them
    need(o.d >= 1 && o.d <= kMaxDim && o.dtheta >= 1 && o.dtheta <= kMaxDim, "dimensions");
    need(o.p_s >= 1 && o.p_s <= kMaxPs, "p_s");
    need(o.fmt == PH_FMT_H || o.fmt == PH_FMT_H2, "format");
    need(o.prec == PH_FP32 || o.prec == PH_FP64, "precision");
    need(o.coupling == 0 || o.coupling == 1, "coupling mode");
    need(o.compressor == 0 || o.compressor == 1, "compressor");
    need((int)h.kernel >= 0 && (int)h.kernel <= PH_KERNEL_POLY2, "kernel");
    need(h.scalar == (o.prec == PH_FP32 ? 4u : 8u), "scalar size");
    int PD = 1, Pf = 1, P = 1;  // P: the near-field grid
    for (int k = 0; k < o.d; ++k) PD *= o.p_s;
    for (int k = 0; k < o.dtheta; ++k) {
        need(o.degree[k] >= 0 && o.degree[k] + 1 <= kMaxPTheta, "theta degree");
        need(o.near_degree[k] >= 0 && o.near_degree[k] + 1 <= kMaxPTheta, "near-field theta degree");
        Pf *= o.degree[k] + 1;
        P *= (o.near_degree[k] > 0 ? o.near_degree[k] : o.degree[k]) + 1;
    }
    need(h.PD == PD && h.Delta == 2 * o.d + o.dtheta && h.p_theta_total == Pf && h.p_theta_near_total == P,
         "derived sizes");
    need_size(h.theta_nodes, (size_t)2 * kMaxDim * kMaxPTheta, "theta nodes");
    need_size(h.theta_bw, (size_t)2 * kMaxDim * kMaxPTheta, "barycentric weights");
    need_size(h.E64, (size_t)2 * o.p_s * o.p_s, "transfer factors");

    // cluster tree
    need(p.d == o.d && p.n >= 1 && p.n <= (1L << 30), "point count");
    const long n = p.n;
    const int nn = (int)p.nodes.size();
    need(nn >= 1 && p.depth >= 0 && p.depth <= 64, "tree size");
    need_size(p.perm, (size_t)n, "permutation");
    {
        std::vector<char> seen((size_t)n, 0);
        for (int v : p.perm) {
            need(v >= 0 && v < n && !seen[(size_t)v], "permutation entries");
            seen[(size_t)v] = 1;
        }
    }
    const int nl = (int)p.leaves.size();
    need(nl >= 1, "leaf count");
    for (int i = 0; i < nn; ++i) {
        const Node& c = p.nodes[i];
        need(c.begin >= 0 && c.begin <= c.end && c.end <= n, "node range");
        need(c.level >= 0 && c.level <= p.depth, "node level");
        need(i == 0 ? c.parent == -1 : (c.parent >= 0 && c.parent < i), "node parent");
        need(c.halves >= 0 && c.halves < (1 << o.d), "node halves");
        need(c.leaf >= -1 && c.leaf < nl, "node leaf index");
        need((c.leaf >= 0) == c.children.empty(), "leaf / children");
        for (int ch : c.children) need(ch > i && ch < nn && p.nodes[ch].parent == i, "node children");
        if (i > 0) {
            const Node& par = p.nodes[c.parent];
            need(c.level == par.level + 1 && c.begin >= par.begin && c.end <= par.end, "child inside parent");
        }
    }
    need(p.nodes[0].begin == 0 && p.nodes[0].end == n, "root range");
    for (int l = 0; l < nl; ++l) {
        const int id = p.leaves[l];
        need(id >= 0 && id < nn && p.nodes[id].leaf == l, "leaf list");
        need(p.nodes[id].size() >= 1, "empty leaf");
        need(l == 0 ? p.nodes[id].begin == 0 : p.nodes[id].begin == p.nodes[p.leaves[l - 1]].end, "leaf order");
    }
    need(p.nodes[p.leaves[nl - 1]].end == n, "leaves cover the points");

    // near blocks: leaf x leaf, grouped by target leaf
    const size_t nb = p.near_s.size();
    need_size(p.near_t, nb, "near sources");
    need_csr(p.near_by_leaf, (size_t)nl, (long long)nb, "near blocks by leaf");
    for (int l = 0; l < nl; ++l)
        for (int b = p.near_by_leaf[l]; b < p.near_by_leaf[l + 1]; ++b) {
            need(p.near_s[b] == p.leaves[l], "near target");
            const int t = p.near_t[b];
            need(t >= 0 && t < nn && p.nodes[t].leaf >= 0, "near source");
        }
    need_size(h.nb_rank, nb, "near ranks");
    need_size(h.nb_off, nb, "near core offsets");
    need_size(h.nb_toff, nb, "near theta-core offsets");
    need_size(h.nb_woff, nb + 1, "near weight offsets");
    need(h.nb_woff[0] == 0, "near weight offsets");
    for (size_t b = 0; b < nb; ++b) {
        const int r = h.nb_rank[b];
        need(r >= 1 && r <= kMaxNearRank, "near rank");
        const long long ent = (long long)p.nodes[p.near_s[b]].size() * p.nodes[p.near_t[b]].size();
        need(in_range(h.nb_off[b], ent * r, h.near_elems), "near core offset");
        need(in_range(h.nb_toff[b], (long long)r * P, h.near_theta_elems), "near theta-core offset");
        need(h.nb_woff[b + 1] == h.nb_woff[b] + r, "near weight offsets");
    }
    need(h.nb_woff[nb] == h.w_elems, "near weight count");
    // mirror sharing: a mirrored block reads the cores of its stored partner (t, s)
    need(o.near_unshared == 0 || o.near_unshared == 1, "near sharing option");
    need_size(h.nb_src, nb, "near core owners");
    for (size_t b = 0; b < nb; ++b) {
        const int src = h.nb_src[b];
        need(src >= 0 && (size_t)src < nb, "near core owner");
        if ((size_t)src == b) continue;
        need(o.near_unshared == 0 && h.nb_src[src] == src && p.near_s[src] == p.near_t[b] &&
                 p.near_t[src] == p.near_s[b],
             "mirrored near block");
        need(h.nb_rank[b] == h.nb_rank[src] && h.nb_off[b] == h.nb_off[src] && h.nb_toff[b] == h.nb_toff[src],
             "mirrored near block offsets");
    }

    // far blocks, translation classes and their cores
    const size_t nf = p.far_s.size();
    const size_t nk = p.key_rep.size();
    need_size(p.far_t, nf, "far sources");
    need_size(p.far_key, nf, "far keys");
    for (size_t b = 0; b < nf; ++b) {
        need(p.far_s[b] >= 0 && p.far_s[b] < nn && p.far_t[b] >= 0 && p.far_t[b] < nn, "far block nodes");
        need(p.far_key[b] >= 0 && (size_t)p.far_key[b] < nk, "far block key");
        need(p.nodes[p.far_s[b]].level == p.nodes[p.far_t[b]].level, "far block levels");
    }
    for (int r : p.key_rep) need(r >= 0 && (size_t)r < nf, "key representative");
    const size_t nt = p.far_targets.size();
    need_csr(p.far_by_target, nt, (long long)nf, "far blocks by target");
    for (size_t t = 0; t < nt; ++t) {
        need(p.far_targets[t] >= 0 && p.far_targets[t] < nn && (t == 0 || p.far_targets[t] > p.far_targets[t - 1]),
             "far targets");
        for (int b = p.far_by_target[t]; b < p.far_by_target[t + 1]; ++b)
            need(p.far_s[b] == p.far_targets[t], "far block target");
    }
    const int D = h.Delta;
    need_size(h.key_ranks, nk * (D + 1), "key ranks");
    need_size(h.key_off, nk * D, "key core offsets");
    need_size(h.key_hoff, nk, "key core-matrix offsets");
    const bool explicit_lr = o.fmt == PH_FMT_H2 && o.coupling == 0 && nk > 0;
    need_size(h.key_lroff, nk, "explicit factor offsets");
    need_size(h.key_tcoff, nk, "tensor-core offsets");
    const bool tc = h.tc_elems > 0;
    if (tc) need(explicit_lr && o.prec == PH_FP32 && PD % 32 == 0, "tensor-core layout");
    for (size_t k = 0; k < nk; ++k) {
        const int* rk = &h.key_ranks[k * (D + 1)];
        need(rk[0] == 1 && rk[D] == 1, "key end ranks");
        for (int i = 1; i < D; ++i) need(rk[i] >= 1 && rk[i] <= 4096, "key rank");
        for (int c = 0; c < D; ++c) {
            const bool theta = c >= o.d && c < o.d + o.dtheta;
            const int dim = theta ? o.degree[c - o.d] + 1 : o.p_s;
            need(in_range(h.key_off[k * D + c], (long long)rk[c] * dim * rk[c + 1],
                          theta ? h.far_theta_elems : h.far_elems),
                 "key core offset");
        }
        const int rd = rk[o.d], rp = rk[o.d + o.dtheta];
        need(in_range(h.key_hoff[k], (long long)rd * rp, h.H_elems), "key core-matrix offset");
        if (explicit_lr) {
            need(rd <= 64 && rp <= 64, "explicit coupling ranks");
            const long long rp4 = (rp + 3) & ~3;
            need(in_range(h.key_lroff[k], (long long)rd * PD + (long long)PD * rp4, h.lr_elems), "explicit factor offset");
        }
        if (tc) {
            const long long r16 = (rp + 15) & ~15;
            need(in_range(h.key_tcoff[k], 2 * 32 * r16 * (PD / 32), h.tc_elems), "tensor-core offset");
        }
    }
    need_size(h.fb_soff, nf, "S_b offsets");
    need_size(h.fb_toff, nf, "T_b offsets");
    if (o.fmt == PH_FMT_H) {
        for (size_t b = 0; b < nf; ++b) {
            const int* rk = &h.key_ranks[(size_t)p.far_key[b] * (D + 1)];
            need(in_range(h.fb_soff[b], (long long)p.nodes[p.far_s[b]].size() * rk[o.d], h.st_elems), "S_b offset");
            need(in_range(h.fb_toff[b], (long long)p.nodes[p.far_t[b]].size() * rk[o.d + o.dtheta], h.st_elems),
                 "T_b offset");
        }
    }

    // device arenas: the bytes stored must be exactly what the element counts say
    const size_t sc = h.scalar;
    const size_t want[] = {(size_t)h.near_elems * sc,       (size_t)h.near_theta_elems * 8,
                           (size_t)h.far_elems * sc,        (size_t)h.far_theta_elems * 8,
                           (size_t)h.st_elems * sc,         (size_t)n * o.d * o.p_s * sc,
                           (size_t)2 * o.p_s * o.p_s * sc,  (size_t)h.lr_elems * sc,
                           (size_t)h.tc_elems * 4};
    need(h.near_elems >= 0 && h.near_theta_elems >= 0 && h.far_elems >= 0 && h.far_theta_elems >= 0 &&
             h.st_elems >= 0 && h.lr_elems >= 0 && h.tc_elems >= 0 && h.H_elems >= 0 && h.w_elems >= 0,
         "arena sizes");
    need_size(arena_bytes, sizeof(want) / sizeof(want[0]), "arena list");
    for (size_t i = 0; i < arena_bytes.size(); ++i)
        if (arena_bytes[i] != want[i])
            bad("arena " + std::to_string(i) + " holds " + std::to_string(arena_bytes[i]) + " bytes, expected " +
                std::to_string(want[i]));
}

}  // namespace ph
