// The transposed far field for the adjoint X = K_hat(theta)^T Y.
//
// Far block b = (s, t) of class k contributes C_k(theta)^T yhat_s to xhat_t in the adjoint, with
// C_k^T = R_k H_k^T L_k^T (§4.2: C_b = L_b H_b R_b^T).  Seen from the adjoint, b is a block with
// target t and source s whose class has L' = R_k, R' = L_k and H' = H_k^T.  This file builds that
// transposed block list (grouped by the new targets, and by class for phase 1 of the explicit
// coupling), the exchanged factors in the layouts the coupling kernels read, and a device view
// that carries them, so that the forward sweep and coupling kernels compute the adjoint's far
// field unchanged.  Nothing here evaluates the method: it only rearranges stored data.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "handle.h"

namespace ph {

namespace {

template <typename V>
V* upload(ph_handle* h, const std::vector<V>& a) {
    V* p = (V*)dev_alloc(h, std::max<size_t>(1, a.size()) * sizeof(V));
    if (!a.empty()) PH_CUDA(cudaMemcpy(p, a.data(), a.size() * sizeof(V), cudaMemcpyHostToDevice));
    return p;
}

template <typename T>
void fill_transposed(ph_handle* h, DevView<T>& vt, const DevView<T>& v, const int* I, const long long* L,
                     const std::vector<long>& io, const std::vector<long>& lo, int n_targets, int max_target,
                     int n_citems) {
    vt = v;  // near field, tree, bases and workspace as the forward view
    vt.key_ranks = I + io[0];
    vt.fb_t = I + io[1];
    vt.fb_key = I + io[2];
    vt.far_targets = I + io[3];
    vt.far_by_target = I + io[4];
    vt.kb_off = I + io[5];
    vt.kb_list = I + io[6];
    vt.citem_key = I + io[7];
    vt.citem_first = I + io[8];
    vt.citem_count = I + io[9];
    vt.n_citems = n_citems;
    vt.n_tcitems = 0;  // the tensor-core layout of phase 1 exists for R_k only
    vt.key_lroff = L + lo[0];
    vt.fb_soff = L + lo[1];
    vt.fb_toff = L + lo[2];
    vt.far_lr = (const T*)h->d_lrT;
    vt.H = (T*)h->d_HT;
    vt.HT = nullptr;
    vt.zstride = h->zstride_adj;
    vt.n_far_targets = n_targets;
    vt.far_max_target = max_target;
}

}  // namespace

void build_adjoint(ph_handle* h, cudaStream_t stream) {
    if (h->adj_ready) return;
    const Plan& plan = h->plan;
    const int d = plan.d, dt = h->opts.dtheta, D = h->Delta, PD = h->PD;
    const bool h2 = h->opts.fmt == PH_FMT_H2;
    if (h2 && h->opts.coupling != 0)
        throw Error(PH_ERR_UNSUPPORTED, "the adjoint of the H^2 format needs the explicit coupling (coupling = 0)");
    const int nf = (int)plan.far_s.size(), nk = (int)plan.key_rep.size();
    // transposed blocks grouped by their target (the original source), then by source
    std::vector<int> ord(nf);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        return plan.far_t[x] != plan.far_t[y] ? plan.far_t[x] < plan.far_t[y] : plan.far_s[x] < plan.far_s[y];
    });
    std::vector<int> fb_t(nf), fb_key(nf), targets, by_target;
    std::vector<long long> soff(nf, 0), toff(nf, 0);
    int max_target = 1;
    for (int i = 0; i < nf; ++i) {
        const int b = ord[i];
        fb_t[i] = plan.far_s[b];
        fb_key[i] = plan.far_key[b];
        if (targets.empty() || targets.back() != plan.far_t[b]) {
            targets.push_back(plan.far_t[b]);
            by_target.push_back(i);
            max_target = std::max(max_target, plan.nodes[plan.far_t[b]].size());
        }
        if (!h->fb_soff.empty()) {
            soff[i] = h->fb_toff[b];  // S' = T_b
            toff[i] = h->fb_soff[b];  // T' = S_b
        }
    }
    by_target.push_back(nf);
    // exchanged ranks: r'_d = r_{d+d_theta}, r'_{d+d_theta} = r_d
    std::vector<int> ranks = h->key_ranks;
    for (int k = 0; k < nk; ++k) std::swap(ranks[(size_t)k * (D + 1) + d], ranks[(size_t)k * (D + 1) + d + dt]);
    // phase-1 items of the transposed blocks: up to 16 blocks of one class (as the forward items)
    std::vector<int> kb_off(nk + 1, 0), kb_list(nf, 0), ck, cf, cc;
    for (int i = 0; i < nf; ++i) kb_off[fb_key[i] + 1]++;
    for (int k = 0; k < nk; ++k) kb_off[k + 1] += kb_off[k];
    {
        std::vector<int> fill(kb_off.begin(), kb_off.end() - 1);
        for (int i = 0; i < nf; ++i) kb_list[fill[fb_key[i]]++] = i;
    }
    h->zstride_adj = 1;
    for (int k = 0; k < nk; ++k) {
        const int rdp = ranks[(size_t)k * (D + 1) + d], rpp = ranks[(size_t)k * (D + 1) + d + dt];
        h->zstride_adj = std::max(h->zstride_adj, rdp);
        const int rp4 = (rpp + 3) & ~3;
        const int nb = std::max(1, std::min(16, 512 / std::max(4, rp4)));
        for (int i = kb_off[k]; i < kb_off[k + 1]; i += nb) {
            ck.push_back(k);
            cf.push_back(i);
            cc.push_back(std::min(nb, kb_off[k + 1] - i));
        }
    }
    if (h->zstride_adj > h->zstride) h->mcap = 0;  // the z buffer is reallocated for the wider rows
    // exchanged explicit factors (H^2): per class L'^T = R_k^T (r' x PD, row-major) then R' = L_k
    // (PD x r_d padded to 4, row-major), from the forward arena [L_k^T (r_d x PD) | R_k (PD x r'_4)]
    std::vector<long long> lroff(nk, 0);
    const size_t sc = h->scalar;
    if (h2 && nk > 0) {
        std::vector<unsigned char> fwd((size_t)h->lr_elems * sc);
        PH_CUDA(cudaMemcpy(fwd.data(), h->d_lr, fwd.size(), cudaMemcpyDeviceToHost));
        auto at = [&](size_t i) -> double {
            return sc == 4 ? (double)reinterpret_cast<const float*>(fwd.data())[i]
                           : reinterpret_cast<const double*>(fwd.data())[i];
        };
        std::vector<double> arena;
        for (int k = 0; k < nk; ++k) {
            const int rd = h->key_ranks[(size_t)k * (D + 1) + d], rp = h->key_ranks[(size_t)k * (D + 1) + d + dt];
            const int rp4 = (rp + 3) & ~3, rd4 = (rd + 3) & ~3;
            const size_t base = (size_t)h->key_lroff[k];
            lroff[k] = (long long)arena.size();
            for (int s = 0; s < rp; ++s)
                for (int J = 0; J < PD; ++J) arena.push_back(at(base + (size_t)rd * PD + (size_t)J * rp4 + s));
            for (int J = 0; J < PD; ++J)
                for (int q = 0; q < rd4; ++q) arena.push_back(q < rd ? at(base + (size_t)q * PD + J) : 0.0);
        }
        if (sc == 4) {
            std::vector<float> f(arena.begin(), arena.end());
            h->d_lrT = upload(h, f);
        } else {
            h->d_lrT = upload(h, arena);
        }
    }
    h->d_HT = dev_alloc(h, std::max<long long>(1, h->H_elems) * sc);
    // pack the index arrays
    std::vector<int> ints;
    std::vector<long> io;
    auto put = [&](const std::vector<int>& a) {
        io.push_back((long)ints.size());
        ints.insert(ints.end(), a.begin(), a.end());
        ints.push_back(0);
    };
    put(ranks);      // 0
    put(fb_t);       // 1
    put(fb_key);     // 2
    put(targets);    // 3
    put(by_target);  // 4
    put(kb_off);     // 5
    put(kb_list);    // 6
    put(ck);         // 7
    put(cf);         // 8
    put(cc);         // 9
    std::vector<long long> lls;
    std::vector<long> lo;
    auto putl = [&](const std::vector<long long>& a) {
        lo.push_back((long)lls.size());
        lls.insert(lls.end(), a.begin(), a.end());
        lls.push_back(0);
    };
    putl(lroff);  // 0
    putl(soff);   // 1
    putl(toff);   // 2
    h->d_adj_int = upload(h, ints);
    h->d_adj_ll = upload(h, lls);
    // the forward views now carry H^T for the instantiate kernel; the transposed views mirror them
    h->vf.HT = (float*)h->d_HT;
    h->vd.HT = (double*)h->d_HT;
    fill_transposed(h, h->vfT, h->vf, h->d_adj_int, h->d_adj_ll, io, lo, (int)targets.size(), max_target,
                    (int)ck.size());
    fill_transposed(h, h->vdT, h->vd, h->d_adj_int, h->d_adj_ll, io, lo, (int)targets.size(), max_target,
                    (int)ck.size());
    h->adj_io = io;
    h->adj_lo = lo;
    h->adj_n_targets = (int)targets.size();
    h->adj_max_target = max_target;
    h->adj_n_citems = (int)ck.size();
    h->adj_ready = true;
    if (h->instantiated) transpose_H(h, stream);
}

void refresh_transposed(ph_handle* h) {
    if (!h->adj_ready) return;
    h->vf.HT = (float*)h->d_HT;
    h->vd.HT = (double*)h->d_HT;
    fill_transposed(h, h->vfT, h->vf, h->d_adj_int, h->d_adj_ll, h->adj_io, h->adj_lo, h->adj_n_targets,
                    h->adj_max_target, h->adj_n_citems);
    fill_transposed(h, h->vdT, h->vd, h->d_adj_int, h->d_adj_ll, h->adj_io, h->adj_lo, h->adj_n_targets,
                    h->adj_max_target, h->adj_n_citems);
}

}  // namespace ph
