// The C ABI of libph (include/ph.h): argument checks, error capture, device
// views, workspace, save / load.  No computation of the method happens here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <fstream>
#include <new>
#include <stdexcept>
#include <string>
#include <unordered_map>

#include "common.cuh"
#include "handle.h"

namespace {

thread_local std::string g_last_error;

using ph::fail;
using ph::guarded;

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace ph {

ph_status fail(ph_handle* h, ph_status s, const std::string& msg) {
    g_last_error = msg;
    if (h) h->last_error = msg;
    return s;
}

void post_timeout_flag(ph_handle* h, cudaStream_t stream) {
    if (h->host_flags && h->d_flags)
        PH_CUDA(cudaMemcpyAsync(h->host_flags, h->d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, stream));
}

ph_status take_timeout(ph_handle* h) {
    if (!h->host_flags) return PH_OK;
    const int seen = *(volatile int*)h->host_flags;
    if (seen > h->seen_timeouts) {
        h->seen_timeouts = seen;
        return fail(h, PH_ERR_TIMEOUT, "a bounded device-side wait of an earlier call ran out (its result is invalid)");
    }
    return PH_OK;
}

void dev_free(ph_handle* h, void* p) {
    if (!p) return;
    for (auto it = h->buffers.begin(); it != h->buffers.end(); ++it)
        if (it->ptr == p) {
            cudaFree(p);
            h->buffers.erase(it);
            return;
        }
}

template <typename T>
static void fill_view(ph_handle* h, DevView<T>& v, const std::vector<long>& io, const std::vector<long>& lo) {
    const Plan& plan = h->plan;
    const int* I = h->d_int;
    const long long* L = h->d_ll;
    v = DevView<T>{};
    v.n = (int)plan.n;
    v.d = plan.d;
    v.p_s = h->opts.p_s;
    v.PD = h->PD;
    v.n_leaves = (int)plan.leaves.size();
    v.n_nodes = (int)plan.nodes.size();
    v.perm = I + io[0];
    v.node_begin = I + io[1];
    v.node_end = I + io[2];
    v.node_halves = I + io[3];
    v.node_children = I + io[4];
    v.node_child_off = I + io[5];
    v.leaf_node = I + io[6];
    v.node_leaf = I + io[7];
    v.node_level = I + io[8];
    v.near_by_leaf = I + io[9];
    v.nb_t = I + io[10];
    v.nb_s = I + io[33];
    v.near_share = h->near_share;
    v.n_mslots = h->n_mslots;
    v.nb_mslot = I + io[34];
    v.mirror_by_leaf = I + io[35];
    v.mslot_block = I + io[36];
    v.nb_rank = I + io[11];
    v.nb_woff = I + io[12];
    v.key_ranks = I + io[13];
    v.fb_t = I + io[14];
    v.fb_key = I + io[15];
    v.far_targets = I + io[16];
    v.far_by_target = I + io[17];
    v.level_slot = I + io[18];
    v.n_items = (int)h->item_first.size();
    v.item_first = I + io[20];
    v.item_count = I + io[21];
    v.item_leaf = I + io[22];
    v.items_by_leaf = I + io[23];
    v.node_parent = I + io[24];
    v.far_lr = (const T*)h->d_lr;
    v.key_lroff = L + lo[6];
    v.kb_off = I + io[25];
    v.kb_list = I + io[26];
    v.n_citems = (int)h->citem_key.size();
    v.citem_key = I + io[27];
    v.citem_first = I + io[28];
    v.citem_count = I + io[29];
    v.far_tc = (const float*)h->d_tc;
    v.key_tcoff = L + lo[7];
    v.n_tcitems = (int)h->tcitem_key.size();
    v.tcitem_key = I + io[30];
    v.tcitem_first = I + io[31];
    v.tcitem_count = I + io[32];
    v.zstride = h->zstride;
    v.zbuf = (T*)h->d_zbuf;
    v.part_stride = h->max_leaf;
    v.partials = (T*)h->d_partials;
    v.nb_off = L + lo[0];
    v.nb_toff = L + lo[1];
    v.key_off = L + lo[2];
    v.key_hoff = L + lo[3];
    v.fb_soff = L + lo[4];
    v.fb_toff = L + lo[5];
    v.dtheta = h->opts.dtheta;
    for (int k = 0; k < 3; ++k) v.p_theta[k] = (k < h->opts.dtheta) ? h->opts.degree[k] + 1 : 1;
    // d_dbl: nodes (far grid, near grid), then barycentric weights (far grid, near grid)
    v.theta_nodes = h->d_dbl;
    v.theta_nodes_near = h->d_dbl + kMaxDim * kMaxPTheta;
    v.theta_bw = h->d_dbl + 2 * kMaxDim * kMaxPTheta;
    v.theta_bw_near = h->d_dbl + 3 * kMaxDim * kMaxPTheta;
    for (int k = 0; k < 3; ++k)
        v.p_theta_near[k] = (k < h->opts.dtheta)
                                ? (h->opts.near_degree[k] > 0 ? h->opts.near_degree[k] : h->opts.degree[k]) + 1
                                : 1;
    v.v64 = h->d_v64;
    v.n_near = (int)plan.near_s.size();
    v.near_cores = (const T*)h->d_near;
    v.near_theta = h->d_near_theta;
    v.w = (T*)h->d_w;
    v.n_keys = (int)plan.key_rep.size();
    v.Delta = h->Delta;
    v.far_cores = (const T*)h->d_far;
    v.far_theta = h->d_far_theta;
    v.H = (T*)h->d_H;
    v.HT = (T*)h->d_HT;
    v.n_far = (int)plan.far_s.size();
    v.n_far_targets = (int)plan.far_targets.size();
    v.far_max_target = 1;
    for (int t : plan.far_targets) v.far_max_target = std::max(v.far_max_target, plan.nodes[t].size());
    v.st = (const T*)h->d_st;
    v.n_far_levels = h->n_far_levels;
    v.U = (const T*)h->d_U;
    v.E = (const T*)h->d_E;
    v.mcap = h->mcap;
    v.Xc = (T*)h->d_Xc;
    v.yfar = (T*)h->d_yfar;
    v.xhat = (T*)h->d_xhat;
    v.yhat = (T*)h->d_yhat;
    v.flags = h->d_flags;
}

void near_mirror_map(ph_handle* h) {
    const Plan& plan = h->plan;
    const int nn = (int)plan.near_s.size();
    h->near_share = h->opts.near_unshared ? 0 : 1;
    h->nb_src.resize(nn);
    for (int b = 0; b < nn; ++b) h->nb_src[b] = b;
    if (!h->near_share) return;
    const long long nodes = (long long)plan.nodes.size();
    std::unordered_map<long long, int> at;
    at.reserve((size_t)nn * 2);
    for (int b = 0; b < nn; ++b) at[(long long)plan.near_s[b] * nodes + plan.near_t[b]] = b;
    for (int b = 0; b < nn; ++b) {
        if (plan.near_s[b] <= plan.near_t[b]) continue;
        auto it = at.find((long long)plan.near_t[b] * nodes + plan.near_s[b]);
        if (it == at.end()) throw Error(PH_ERR_IO, "inconsistent handle data: near block without its mirror");
        h->nb_src[b] = it->second;
    }
}

// Packs the plan's index arrays into two device allocations and fills the views.
void refresh_views(ph_handle* h) {
    const Plan& plan = h->plan;
    h->near_rank_max = 0;
    for (int r : h->nb_rank) h->near_rank_max = std::max(h->near_rank_max, r);
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess && nsm > 0)
        h->num_sms = nsm;
    else
        cudaGetLastError();
    std::vector<int> ints;
    std::vector<long> io;
    auto put = [&](const std::vector<int>& a) {
        io.push_back((long)ints.size());
        ints.insert(ints.end(), a.begin(), a.end());
        ints.push_back(0);  // keep every segment non-empty
    };
    const int nn = (int)plan.nodes.size();
    std::vector<int> nb(nn), ne(nn), nh(nn), ch, choff(nn + 1, 0), nl(nn), lev(nn);
    for (int i = 0; i < nn; ++i) {
        nb[i] = plan.nodes[i].begin;
        ne[i] = plan.nodes[i].end;
        nh[i] = plan.nodes[i].halves;
        nl[i] = plan.nodes[i].leaf;
        lev[i] = plan.nodes[i].level;
        for (int c : plan.nodes[i].children) ch.push_back(c);
        choff[i + 1] = (int)ch.size();
    }
    // levels that own far targets get a slot in y_far (H format)
    h->level_slot.assign(plan.depth + 1, -1);
    h->n_far_levels = 0;
    h->min_far_level = plan.depth;
    for (int s : plan.far_targets) {
        int l = plan.nodes[s].level;
        h->min_far_level = std::min(h->min_far_level, l);
        if (h->level_slot[l] < 0) h->level_slot[l] = 1;
    }
    for (int l = 0; l <= plan.depth; ++l)
        if (h->level_slot[l] > 0) h->level_slot[l] = h->n_far_levels++;
    // inner nodes per level, for the sweeps
    h->level_nodes.assign(plan.depth + 1, {});
    for (int i = 0; i < nn; ++i)
        if (!plan.nodes[i].children.empty()) h->level_nodes[plan.nodes[i].level].push_back(i);
    h->level_has_inner_child.assign(plan.depth + 1, 0);
    for (int i = 0; i < nn; ++i)
        for (int c : plan.nodes[i].children)
            if (!plan.nodes[c].children.empty()) h->level_has_inner_child[plan.nodes[i].level] = 1;
    std::vector<int> lvl_flat;
    h->level_nodes_off.assign(plan.depth + 2, 0);
    for (int l = 0; l <= plan.depth; ++l) {
        lvl_flat.insert(lvl_flat.end(), h->level_nodes[l].begin(), h->level_nodes[l].end());
        h->level_nodes_off[l + 1] = (int)lvl_flat.size();
    }
    // near work items: up to kNearItemBlocks consecutive stored near blocks of one target leaf
    // (two with mirror sharing, whose kernel also stages x_s and a slice of D_b).  With sharing a
    // leaf's stored blocks (s, t >= s) end its run: the plan orders a leaf's blocks by source id.
    const int kNearItemBlocks = h->near_share ? 2 : 4;
    const int nnear = (int)plan.near_s.size();
    if ((int)h->nb_src.size() != nnear) near_mirror_map(h);
    h->item_first.clear();
    h->item_count.clear();
    h->item_leaf.clear();
    h->items_by_leaf.assign(plan.leaves.size() + 1, 0);
    h->max_leaf = 1;
    for (size_t l = 0; l < plan.leaves.size(); ++l) {
        h->max_leaf = std::max(h->max_leaf, plan.nodes[plan.leaves[l]].size());
        std::vector<int> run;
        for (int b = plan.near_by_leaf[l]; b < plan.near_by_leaf[l + 1]; ++b)
            if (h->nb_src[b] == b) run.push_back(b);
        for (size_t q = 0; q < run.size();) {
            // items cover consecutive block indices
            size_t e = q + 1;
            while (e < run.size() && (int)(e - q) < kNearItemBlocks && run[e] == run[e - 1] + 1) ++e;
            h->item_first.push_back(run[q]);
            h->item_count.push_back((int)(e - q));
            h->item_leaf.push_back((int)l);
            q = e;
        }
        h->items_by_leaf[l + 1] = (int)h->item_first.size();
    }
    // mirror slots: one per stored block (s, t), s != t, grouped by the leaf t that receives them
    h->nb_mslot.assign(nnear, -1);
    h->mirror_by_leaf.assign(plan.leaves.size() + 1, 0);
    h->mslot_block.clear();
    h->n_mslots = 0;
    if (h->near_share) {
        std::vector<std::vector<int>> by_t(plan.leaves.size());
        for (int b = 0; b < nnear; ++b)
            if (h->nb_src[b] == b && plan.near_s[b] != plan.near_t[b])
                by_t[plan.nodes[plan.near_t[b]].leaf].push_back(b);
        for (size_t l = 0; l < plan.leaves.size(); ++l) {
            for (int b : by_t[l]) {
                h->nb_mslot[b] = h->n_mslots++;
                h->mslot_block.push_back(b);
            }
            h->mirror_by_leaf[l + 1] = h->n_mslots;
        }
    }
    // longest intermediate of the coupling chain kept in shared memory (all steps but the
    // first input and the last output): right-core outputs a r_out, H output, left-core outputs
    h->coupling_zmax = 1;
    if (!plan.key_rep.empty()) {
        const int d = plan.d, p = h->opts.p_s, D = h->Delta;
        for (size_t k = 0; k < plan.key_rep.size(); ++k) {
            const int* rk = &h->key_ranks[k * (D + 1)];
            int a = h->PD / p;
            for (int i = 0; i < d; ++i) {
                h->coupling_zmax = std::max(h->coupling_zmax, a * rk[D - 1 - i]);
                a /= p;
            }
            h->coupling_zmax = std::max(h->coupling_zmax, rk[d]);
            int bsz = 1;
            for (int i = 0; i + 1 < d; ++i) {
                const int core = d - 1 - i;
                h->coupling_zmax = std::max(h->coupling_zmax, rk[core] * p * bsz);
                bsz *= p;
            }
        }
        h->coupling_zmax = (h->coupling_zmax + 3) & ~3;
    }
    std::vector<int> fbt = plan.far_by_target;
    if (fbt.empty()) fbt.push_back(0);
    put(plan.perm);                 // 0
    put(nb);                        // 1
    put(ne);                        // 2
    put(nh);                        // 3
    put(ch);                        // 4
    put(choff);                     // 5
    put(plan.leaves);               // 6
    put(nl);                        // 7
    put(lev);                       // 8
    put(plan.near_by_leaf);         // 9
    put(plan.near_t);               // 10
    put(h->nb_rank);                // 11
    put(h->nb_woff);                // 12
    put(h->key_ranks);              // 13
    put(plan.far_t);                // 14
    put(plan.far_key);              // 15
    put(plan.far_targets);          // 16
    put(fbt);                       // 17
    put(h->level_slot);             // 18
    put(lvl_flat);                  // 19
    put(h->item_first);             // 20
    put(h->item_count);             // 21
    put(h->item_leaf);              // 22
    put(h->items_by_leaf);          // 23
    std::vector<int> par(nn);
    for (int i = 0; i < nn; ++i) par[i] = plan.nodes[i].parent;
    put(par);                       // 24
    // far blocks grouped by translation class, and the key-grouped items of the explicit coupling
    // (up to kCouplingItemBlocks blocks of one key per item)
    constexpr int kCouplingItemBlocks = 16;
    const int nkeys = (int)plan.key_rep.size();
    h->kb_off.assign(nkeys + 1, 0);
    for (int k : plan.far_key) h->kb_off[k + 1]++;
    for (int k = 0; k < nkeys; ++k) h->kb_off[k + 1] += h->kb_off[k];
    h->kb_list.assign(plan.far_key.size(), 0);
    {
        std::vector<int> fill(h->kb_off.begin(), h->kb_off.end() - (nkeys > 0 ? 1 : 0));
        if (nkeys == 0) fill.clear();
        for (size_t b = 0; b < plan.far_key.size(); ++b) h->kb_list[fill[plan.far_key[b]]++] = (int)b;
    }
    h->citem_key.clear();
    h->citem_first.clear();
    h->citem_count.clear();
    h->zstride = 1;
    h->rank_max_lr = 1;
    for (int k = 0; k < nkeys; ++k) {
        h->zstride = std::max(h->zstride, h->key_ranks[(size_t)k * (h->Delta + 1) + plan.d]);
        h->rank_max_lr = std::max(h->rank_max_lr, std::max(h->key_ranks[(size_t)k * (h->Delta + 1) + plan.d],
                                                           h->key_ranks[(size_t)k * (h->Delta + 1) + plan.d + h->opts.dtheta]));
        // blocks per item: about 8192 outputs of P = R_k^T X per CTA at 16 right-hand sides
        // (256 threads with tiles of 4 x 8)
        const int rp4 = (h->key_ranks[(size_t)k * (h->Delta + 1) + plan.d + h->opts.dtheta] + 3) & ~3;
        const int nb = std::max(1, std::min(kCouplingItemBlocks, 512 / std::max(4, rp4)));
        for (int i = h->kb_off[k]; i < h->kb_off[k + 1]; i += nb) {
            h->citem_key.push_back(k);
            h->citem_first.push_back(i);
            h->citem_count.push_back(std::min(nb, h->kb_off[k + 1] - i));
        }
    }
    put(h->kb_off);                 // 25
    put(h->kb_list);                // 26
    put(h->citem_key);              // 27
    put(h->citem_first);            // 28
    put(h->citem_count);            // 29
    // tensor-core items: 8 blocks of one class (M = 128 columns at 16 right-hand sides)
    h->tcitem_key.clear();
    h->tcitem_first.clear();
    h->tcitem_count.clear();
    for (int k = 0; k < nkeys; ++k)
        for (int i = h->kb_off[k]; i < h->kb_off[k + 1]; i += 8) {
            h->tcitem_key.push_back(k);
            h->tcitem_first.push_back(i);
            h->tcitem_count.push_back(std::min(8, h->kb_off[k + 1] - i));
        }
    put(h->tcitem_key);             // 30
    put(h->tcitem_first);           // 31
    put(h->tcitem_count);           // 32
    put(plan.near_s);               // 33
    put(h->nb_mslot);               // 34
    put(h->mirror_by_leaf);         // 35
    put(h->mslot_block);            // 36
    std::vector<long long> lls;
    std::vector<long> lo;
    auto putl = [&](const std::vector<long long>& a) {
        lo.push_back((long)lls.size());
        lls.insert(lls.end(), a.begin(), a.end());
        lls.push_back(0);
    };
    putl(h->nb_off);
    putl(h->nb_toff);
    putl(h->key_off);
    putl(h->key_hoff);
    putl(h->fb_soff);
    putl(h->fb_toff);
    putl(h->key_lroff);
    putl(h->key_tcoff);
    dev_free(h, h->d_int);
    dev_free(h, h->d_ll);
    dev_free(h, h->d_dbl);
    h->d_int = (int*)dev_alloc(h, ints.size() * sizeof(int));
    PH_CUDA(cudaMemcpy(h->d_int, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->d_ll = (long long*)dev_alloc(h, lls.size() * sizeof(long long));
    PH_CUDA(cudaMemcpy(h->d_ll, lls.data(), lls.size() * sizeof(long long), cudaMemcpyHostToDevice));
    std::vector<double> dbl(h->theta_nodes);
    dbl.insert(dbl.end(), h->theta_bw.begin(), h->theta_bw.end());
    h->d_dbl = (double*)dev_alloc(h, dbl.size() * sizeof(double));
    PH_CUDA(cudaMemcpy(h->d_dbl, dbl.data(), dbl.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (!h->d_v64) h->d_v64 = (double*)dev_alloc(h, kMaxDim * kMaxPTheta * sizeof(double));
    if (!h->d_flags) {
        h->d_flags = (int*)dev_alloc(h, 4 * sizeof(int));
        PH_CUDA(cudaMemset(h->d_flags, 0, 4 * sizeof(int)));
    }
    if (!h->host_flags) {
        PH_CUDA(cudaHostAlloc((void**)&h->host_flags, sizeof(int), cudaHostAllocDefault));
        *h->host_flags = 0;
        h->seen_timeouts = 0;
    }
    h->d_level_nodes = h->d_int + io[19];
    fill_view<float>(h, h->vf, io, lo);
    fill_view<double>(h, h->vd, io, lo);
    h->view_io = io;
    h->view_lo = lo;
    refresh_transposed(h);
}

// Sizes the per-call workspace for m right-hand sides (padded to the chunk width).
void ensure_workspace(ph_handle* h, int m) {
    const int mc = (m <= 1) ? 1 : (m <= 2) ? 2 : (m <= 4) ? 4 : (m <= 8) ? 8 : 16;
    const int S = (int)ceil_div(m, mc) * mc;
    if (S <= h->mcap) return;
    const Plan& plan = h->plan;
    const size_t sc = h->scalar;
    for (void* p : {h->d_Xc, h->d_yfar, h->d_xhat, h->d_yhat, h->d_partials, h->d_zbuf}) dev_free(h, p);
    // nothing may point at the freed buffers should an allocation below fail
    h->d_Xc = h->d_yfar = h->d_xhat = h->d_yhat = h->d_partials = h->d_zbuf = nullptr;
    h->mcap = 0;
    fill_view<float>(h, h->vf, h->view_io, h->view_lo);
    fill_view<double>(h, h->vd, h->view_io, h->view_lo);
    h->d_Xc = dev_alloc(h, (size_t)plan.n * S * sc);
    h->d_partials = dev_alloc(h, std::max<size_t>(1, h->item_first.size() + h->n_mslots) * h->max_leaf * S * sc);
    h->d_yfar = nullptr;
    h->d_xhat = h->d_yhat = nullptr;
    if (h->opts.fmt == PH_FMT_H && h->n_far_levels > 0)
        h->d_yfar = dev_alloc(h, (size_t)h->n_far_levels * plan.n * S * sc);
    if (h->opts.fmt == PH_FMT_H2 && !plan.far_targets.empty()) {
        h->d_xhat = dev_alloc(h, (size_t)plan.nodes.size() * h->PD * S * sc);
        h->d_yhat = dev_alloc(h, (size_t)plan.nodes.size() * h->PD * S * sc);
        if (h->opts.coupling == 0)
            h->d_zbuf = dev_alloc(h, plan.far_s.size() * (size_t)std::max(h->zstride, h->zstride_adj) * S * sc);
    }
    h->mcap = S;
    fill_view<float>(h, h->vf, h->view_io, h->view_lo);
    fill_view<double>(h, h->vd, h->view_io, h->view_lo);
    refresh_transposed(h);
}

}  // namespace ph

extern "C" {

const char* ph_version(void) { return "libph 0.1 (sm_103a)"; }

ph_status ph_selftest_wait_bound(int device, double* waited) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, PH_ERR_INVALID_ARG, "ph_selftest_wait_bound: no CUDA device " + std::to_string(device));
    }
    try {
        return ph::wait_bound_selftest(device, waited);
    } catch (const ph::Error& e) {
        return fail(nullptr, e.status, e.what());
    }
}

const char* ph_last_error(const ph_handle* h) {
    if (h) return h->last_error.c_str();
    return g_last_error.c_str();
}

static ph_status plan_counts(const double* points, long n, int d, int l_max, double eta, int leaf_size, long* counts,
                             int* perm) {
    return guarded(nullptr, [&]() -> ph_status {
        ph::Plan plan;
        ph::build_plan(points, n, d, l_max, eta, true, plan, leaf_size);
        long sum_near = 0;
        for (size_t b = 0; b < plan.near_s.size(); ++b)
            sum_near += (long)plan.nodes[plan.near_s[b]].size() * plan.nodes[plan.near_t[b]].size();
        for (size_t b = 0; b < plan.inner_near_s.size(); ++b)
            sum_near += (long)plan.nodes[plan.inner_near_s[b]].size() * plan.nodes[plan.inner_near_t[b]].size();
        int maxper = 0;
        for (size_t l = 0; l + 1 < plan.near_by_leaf.size(); ++l)
            maxper = std::max(maxper, plan.near_by_leaf[l + 1] - plan.near_by_leaf[l]);
        counts[0] = (long)plan.nodes.size();
        counts[1] = (long)plan.leaves.size();
        counts[2] = (long)(plan.near_s.size() + plan.inner_near_s.size());
        counts[3] = (long)plan.far_s.size();
        counts[4] = (long)plan.key_rep.size();
        counts[5] = sum_near;
        counts[6] = maxper;
        counts[7] = plan.depth;
        if (perm)
            for (long i = 0; i < n; ++i) perm[i] = plan.perm[i];
        return PH_OK;
    });
}

ph_status ph_plan(const double* points, long n, int d, int l_max, double eta, long* counts, int* perm) {
    if (!points || !counts || n < 1 || d < 1 || d > 3 || l_max < 0 || l_max > 10 || !(eta > 0))
        return fail(nullptr, PH_ERR_INVALID_ARG, "ph_plan: invalid argument");
    return plan_counts(points, n, d, l_max, eta, 0, counts, perm);
}

ph_status ph_plan_adaptive(const double* points, long n, int d, int leaf_size, double eta, long* counts, int* perm) {
    if (!points || !counts || n < 1 || d < 1 || d > 3 || leaf_size < 1 || !(eta > 0))
        return fail(nullptr, PH_ERR_INVALID_ARG, "ph_plan_adaptive: invalid argument");
    return plan_counts(points, n, d, 0, eta, leaf_size, counts, perm);
}

ph_status ph_offline_build(const double* points, long n, ph_kernel kernel, const ph_build_opts* o,
                           ph_handle** out) {
    if (!out) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_offline_build: out is NULL");
    *out = nullptr;
    if (!points || !o || n < 1) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_offline_build: invalid argument");
    if (o->d < 1 || o->d > 3 || o->dtheta < 1 || o->dtheta > 3 || o->p_s < 1 || o->p_s > ph::kMaxPs ||
        o->l_max < 0 || o->l_max > 10 || !(o->eta > 0) || !(o->tol >= 0) || o->rank_cap < 0 ||
        (o->fmt != PH_FMT_H && o->fmt != PH_FMT_H2) || (o->prec != PH_FP32 && o->prec != PH_FP64) ||
        (int)kernel < 0 || (int)kernel > PH_KERNEL_POLY2)
        return fail(nullptr, PH_ERR_INVALID_ARG, "ph_offline_build: option out of range");
    if (kernel == PH_KERNEL_ANISO_GAUSS && o->dtheta != o->d)
        return fail(nullptr, PH_ERR_INVALID_ARG, "anisotropic Gaussian needs d_theta = d");
    if (kernel == PH_KERNEL_POLY2 && o->dtheta != 2)
        return fail(nullptr, PH_ERR_INVALID_ARG, "the two-parameter polynomial kernel needs d_theta = 2");
    if (kernel != PH_KERNEL_ANISO_GAUSS && kernel != PH_KERNEL_POLY2 && o->dtheta != 1)
        return fail(nullptr, PH_ERR_INVALID_ARG, "this kernel has one parameter (d_theta = 1)");
    for (int k = 0; k < o->dtheta; ++k)
        if (!(o->theta_lo[k] < o->theta_hi[k]) || o->degree[k] < 0 || o->degree[k] + 1 > ph::kMaxPTheta ||
            o->near_degree[k] < 0 || o->near_degree[k] + 1 > ph::kMaxPTheta)
            return fail(nullptr, PH_ERR_INVALID_ARG, "ph_offline_build: bad parameter box or degree");
    if (o->near_unshared != 0 && o->near_unshared != 1)
        return fail(nullptr, PH_ERR_INVALID_ARG, "ph_offline_build: near_unshared must be 0 or 1");
    if (o->compressor != 0 && o->compressor != 1)
        return fail(nullptr, PH_ERR_INVALID_ARG, "ph_offline_build: compressor must be 0 (TT-SVD) or 1 (TT-cross)");
    ph_handle* h = nullptr;
    try {
        h = new ph_handle();
    } catch (...) {
        return fail(nullptr, PH_ERR_OOM, "host allocation failed");
    }
    h->kernel = kernel;
    h->opts = *o;
    h->device = o->device;
    ph_status st = guarded(h, [&]() -> ph_status {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= o->device || o->device < 0) {
            cudaGetLastError();
            throw ph::Error(PH_ERR_CUDA, "no CUDA device " + std::to_string(o->device));
        }
        ph::offline_build(h, points, n);
        const size_t sc = h->scalar;
        ph::validate_handle(*h, {(size_t)h->near_elems * sc, (size_t)h->near_theta_elems * 8,
                                 (size_t)h->far_elems * sc, (size_t)h->far_theta_elems * 8, (size_t)h->st_elems * sc,
                                 (size_t)n * o->d * o->p_s * sc, (size_t)2 * o->p_s * o->p_s * sc,
                                 (size_t)h->lr_elems * sc, (size_t)h->tc_elems * 4});
        ph::refresh_views(h);
        PH_CUDA(cudaDeviceSynchronize());
        return PH_OK;
    });
    if (st != PH_OK) {
        g_last_error = h->last_error;
        ph::free_device(h);
        delete h;
        return st;
    }
    *out = h;
    return PH_OK;
}

static ph_status instantiate_common(ph_handle* h, const double* theta, int deriv, void* stream) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_instantiate: NULL handle");
    if (!theta) return fail(h, PH_ERR_INVALID_ARG, "ph_instantiate: NULL theta");
    if (deriv < -1 || deriv >= h->opts.dtheta)
        return fail(h, PH_ERR_INVALID_ARG, "ph_instantiate_derivative: dim outside [0, d_theta)");
    for (int k = 0; k < h->opts.dtheta; ++k) {
        if (!std::isfinite(theta[k])) return fail(h, PH_ERR_NONFINITE, "theta is not finite");
        if (theta[k] < h->opts.theta_lo[k] || theta[k] > h->opts.theta_hi[k])
            return fail(h, PH_ERR_THETA_OUT_OF_BOX, "theta outside the parameter box");
    }
    if (ph::take_timeout(h) != PH_OK) return PH_ERR_TIMEOUT;
    return guarded(h, [&]() -> ph_status {
        ph::NvtxRange range(deriv < 0 ? "ph_instantiate" : "ph_instantiate_derivative");
        PH_CUDA(cudaSetDevice(h->device));
        ph::online_instantiate(h, theta, as_stream(stream), deriv);
        h->instantiated = true;
        return PH_OK;
    });
}

ph_status ph_instantiate(ph_handle* h, const double* theta, void* stream) {
    return instantiate_common(h, theta, -1, stream);
}

ph_status ph_instantiate_derivative(ph_handle* h, const double* theta, int dim, void* stream) {
    if (dim < 0) return fail(h, PH_ERR_INVALID_ARG, "ph_instantiate_derivative: dim outside [0, d_theta)");
    return instantiate_common(h, theta, dim, stream);
}

static ph_status check_mv(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_matvec: NULL handle");
    if (!X || !Y || m < 1 || m > 1024 || ldx < h->plan.n || ldy < h->plan.n)
        return fail(h, PH_ERR_INVALID_ARG, "ph_matvec: invalid argument");
    if (!h->instantiated) return fail(h, PH_ERR_NOT_INSTANTIATED, "ph_matvec before ph_instantiate");
    return ph::take_timeout(h);
}

ph_status ph_matvec(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy, void* stream) {
    ph_status s = check_mv(h, X, ldx, m, Y, ldy);
    if (s != PH_OK) return s;
    return guarded(h, [&]() -> ph_status {
        ph::NvtxRange range("ph_matvec");
        PH_CUDA(cudaSetDevice(h->device));
        return ph::online_matvec(h, X, ldx, m, Y, ldy, as_stream(stream));
    });
}

ph_status ph_matvec_transpose(ph_handle* h, const void* Y, long ldy, int m, void* X, long ldx, void* stream) {
    ph_status s = check_mv(h, Y, ldy, m, X, ldx);
    if (s != PH_OK) return s;
    return guarded(h, [&]() -> ph_status {
        ph::NvtxRange range("ph_matvec_transpose");
        PH_CUDA(cudaSetDevice(h->device));
        return ph::online_matvec_transpose(h, Y, ldy, m, X, ldx, as_stream(stream));
    });
}

ph_status ph_matvec_batched(ph_handle* h, const double* thetas, int n_theta, const void* X, long ldx, int m, void* Y,
                            long ldy, long stride_y, int deriv, void* stream) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_matvec_batched: NULL handle");
    if (!thetas || n_theta < 1 || n_theta > 65535 * 32 || !X || !Y || m < 1 || m > 1024 || ldx < h->plan.n ||
        ldy < h->plan.n || stride_y < ldy * (long)m || deriv < -1 || deriv >= h->opts.dtheta)
        return fail(h, PH_ERR_INVALID_ARG, "ph_matvec_batched: invalid argument");
    if (h->opts.dtheta != 1) return fail(h, PH_ERR_UNSUPPORTED, "ph_matvec_batched: d_theta must be 1");
    if (ph::take_timeout(h) != PH_OK) return PH_ERR_TIMEOUT;
    for (int t = 0; t < n_theta; ++t) {
        if (!std::isfinite(thetas[t])) return fail(h, PH_ERR_NONFINITE, "theta is not finite");
        if (thetas[t] < h->opts.theta_lo[0] || thetas[t] > h->opts.theta_hi[0])
            return fail(h, PH_ERR_THETA_OUT_OF_BOX, "theta outside the parameter box");
    }
    return guarded(h, [&]() -> ph_status {
        ph::NvtxRange range("ph_matvec_batched");
        PH_CUDA(cudaSetDevice(h->device));
        ph_status st = ph::online_matvec_batched(h, thetas, n_theta, X, ldx, m, Y, ldy, stride_y, deriv,
                                                 as_stream(stream));
        h->instantiated = true;
        return st;
    });
}

ph_status ph_matvec_host(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy, void* stream) {
    ph_status s = check_mv(h, X, ldx, m, Y, ldy);
    if (s != PH_OK) return s;
    return guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        cudaStream_t st = as_stream(stream);
        const size_t sc = h->scalar, n = (size_t)h->plan.n;
        const size_t need = n * m * sc;
        if (h->host_stage_x.bytes < need) {
            ph::dev_free(h, h->host_stage_x.ptr);
            ph::dev_free(h, h->host_stage_y.ptr);
            h->host_stage_x = {ph::dev_alloc(h, need), need};
            h->host_stage_y = {ph::dev_alloc(h, need), need};
        }
        PH_CUDA(cudaMemcpy2DAsync(h->host_stage_x.ptr, n * sc, X, (size_t)ldx * sc, n * sc, m,
                                  cudaMemcpyHostToDevice, st));
        ph::online_matvec(h, h->host_stage_x.ptr, (long)n, m, h->host_stage_y.ptr, (long)n, st);
        PH_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * sc, h->host_stage_y.ptr, n * sc, n * sc, m,
                                  cudaMemcpyDeviceToHost, st));
        PH_CUDA(cudaStreamSynchronize(st));
        return PH_OK;
    });
}

ph_status ph_check(ph_handle* h, void* stream) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_check: NULL handle");
    ph_status st = guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        PH_CUDA(cudaStreamSynchronize(as_stream(stream)));
        if (h->side) PH_CUDA(cudaStreamSynchronize(h->side));
        return PH_OK;
    });
    if (st != PH_OK) return st;
    return ph::take_timeout(h);
}

ph_status ph_selftest_timeout(ph_handle* h, void* stream) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_selftest_timeout: NULL handle");
    return guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        return ph::handle_timeout_selftest(h, as_stream(stream));
    });
}

ph_status ph_inject_alloc_failure(long after) {
    ph::set_alloc_failure(after);
    return PH_OK;
}

ph_status ph_get_info(const ph_handle* h, ph_info* info) {
    if (!h || !info) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_get_info: NULL argument");
    const ph::Plan& plan = h->plan;
    ph_info r{};
    r.n = plan.n;
    r.d = plan.d;
    r.dtheta = h->opts.dtheta;
    r.p_s = h->opts.p_s;
    for (int k = 0; k < 3; ++k) r.p_theta[k] = (k < h->opts.dtheta) ? h->opts.degree[k] + 1 : 0;
    r.prec = h->opts.prec;
    r.fmt = h->opts.fmt;
    r.n_nodes = (int)plan.nodes.size();
    r.n_leaves = (int)plan.leaves.size();
    r.tree_depth = plan.depth;
    r.n_near = (long)plan.near_s.size();
    r.n_far = (long)plan.far_s.size();
    r.n_far_keys = (long)plan.key_rep.size();
    const int D = h->Delta, d = plan.d;
    for (size_t b = 0; b < plan.near_s.size(); ++b) {
        r.near_entries += (long)plan.nodes[plan.near_s[b]].size() * plan.nodes[plan.near_t[b]].size();
        r.near_rank_sum += h->nb_rank[b];
        r.near_rank_max = std::max(r.near_rank_max, h->nb_rank[b]);
    }
    double rank_sum = 0;
    for (size_t k = 0; k < plan.key_rep.size(); ++k)
        for (int i = 0; i <= D; ++i) r.far_rank_max = std::max(r.far_rank_max, h->key_ranks[k * (D + 1) + i]);
    for (size_t b = 0; b < plan.far_s.size(); ++b) {
        const int* rk = &h->key_ranks[(size_t)plan.far_key[b] * (D + 1)];
        rank_sum += std::max(rk[d], rk[d + h->opts.dtheta]);
    }
    r.far_rank_mean = plan.far_s.empty() ? 0.0 : rank_sum / plan.far_s.size();
    const size_t sc = h->scalar;
    r.near_bytes = (long)(h->near_elems * sc);
    r.near_theta_bytes = (long)(h->near_theta_elems * 8);
    r.far_bytes = (long)(h->far_elems * sc + h->far_theta_elems * 8 + h->st_elems * sc);
    r.basis_bytes = (long)((size_t)plan.n * d * h->opts.p_s * sc + 2 * h->opts.p_s * h->opts.p_s * sc);
    // one call moves every stored core the online stage reads once, plus H_k and w_b written and read
    double alg = (double)r.near_bytes + r.near_theta_bytes + (double)h->far_theta_elems * 8 +
                 2.0 * (double)(h->H_elems + h->w_elems) * sc;
    if (h->opts.fmt == PH_FMT_H2 && !plan.far_s.empty())
        alg += (double)h->far_elems * sc + (double)r.basis_bytes;
    if (h->opts.fmt == PH_FMT_H) alg += (double)h->st_elems * sc;
    r.alg_bytes_per_call = alg;
    r.tensor_core_phase1 = (h->tc_elems > 0 && h->use_tc && h->rank_max_lr <= 64) ? 1 : 0;  // for 8 < m <= 16
    r.kernel_variants = h->last_variants;
    r.far_core_elems = (long)h->H_elems;
    for (int k = 0; k < 3; ++k)
        r.p_theta_near[k] = (k < h->opts.dtheta)
                                ? (h->opts.near_degree[k] > 0 ? h->opts.near_degree[k] : h->opts.degree[k]) + 1
                                : 0;
    // flops per right-hand side
    double fl = 2.0 * (double)r.near_entries;  // D_b x
    for (size_t b = 0; b < plan.near_s.size(); ++b) {
        if (!h->nb_src.empty() && h->nb_src[b] != (int)b) continue;  // a shared pair forms d_ij once
        fl += 2.0 * h->nb_rank[b] * (double)plan.nodes[plan.near_s[b]].size() * plan.nodes[plan.near_t[b]].size() /
              16.0;  // forming d_ij, shared by 16 right-hand sides in a chunk
    }
    const int p = h->opts.p_s, PD = h->PD, dt = h->opts.dtheta;
    for (size_t b = 0; b < plan.far_s.size(); ++b) {
        const int* rk = &h->key_ranks[(size_t)plan.far_key[b] * (D + 1)];
        if (h->opts.fmt == PH_FMT_H) {
            fl += 2.0 * (plan.nodes[plan.far_s[b]].size() * (double)rk[d] +
                         plan.nodes[plan.far_t[b]].size() * (double)rk[d + dt] + (double)rk[d] * rk[d + dt]);
        } else if (h->opts.coupling == 0) {
            const double fa = 2.0 * PD * rk[d + dt] + 2.0 * rk[d] * rk[d + dt], fbb = 2.0 * PD * rk[d];
            r.coupling_a_flops_per_rhs += fa;
            r.coupling_b_flops_per_rhs += fbb;
            fl += fa + fbb;
        } else {
            double a = PD / p, chain = 0;
            for (int i = 0; i < d; ++i) {  // right cores
                int core = D - 1 - i;
                chain += 2.0 * a * rk[core] * p * rk[core + 1];
                a /= p;
            }
            chain += 2.0 * rk[d] * rk[d + dt];
            double bsz = 1;
            for (int i = 0; i < d; ++i) {  // left cores
                int core = d - 1 - i;
                chain += 2.0 * rk[core] * p * rk[core + 1] * bsz;
                bsz *= p;
            }
            fl += chain;
            r.coupling_a_flops_per_rhs += chain;
        }
    }
    if (h->opts.fmt == PH_FMT_H2 && !plan.far_s.empty()) {
        fl += 2.0 * 2.0 * (double)plan.n * PD;                                           // leaf up / down
        fl += 2.0 * 2.0 * (double)plan.nodes.size() * d * (double)PD * p;                  // transfers
    }
    r.flops_per_rhs = fl;
    r.offline_seconds = h->offline_seconds;
    *info = r;
    return PH_OK;
}

ph_status ph_set_overlap(ph_handle* h, int enable) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_set_overlap: NULL handle");
    h->overlap = enable != 0;
    return PH_OK;
}

ph_status ph_set_tensor_cores(ph_handle* h, int enable) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_set_tensor_cores: NULL handle");
    h->use_tc = enable != 0;
    return PH_OK;
}

ph_status ph_profile_enable(ph_handle* h, int enable) {
    if (!h) return fail(nullptr, PH_ERR_INVALID_ARG, "ph_profile_enable: NULL handle");
    h->prof = enable != 0;
    return PH_OK;
}

ph_status ph_profile_read(ph_handle* h, double* ms, long* launches) {
    if (!h || !ms || !launches) return fail(h, PH_ERR_INVALID_ARG, "ph_profile_read: NULL argument");
    return guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        for (int k = 0; k < PH_PROF_KINDS; ++k) {
            ms[k] = 0.0;
            launches[k] = 0;
        }
        for (auto& r : h->prof_recs) {
            PH_CUDA(cudaEventSynchronize(r.b));
            float t = 0.f;
            PH_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            if (r.kind >= 0 && r.kind < PH_PROF_KINDS) {
                ms[r.kind] += t;
                launches[r.kind] += 1;
            }
            h->prof_pool.push_back(r.a);
            h->prof_pool.push_back(r.b);
        }
        h->prof_recs.clear();
        return PH_OK;
    });
}

void ph_destroy(ph_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto& r : h->prof_recs) {
        h->prof_pool.push_back(r.a);
        h->prof_pool.push_back(r.b);
    }
    for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
    ph::free_device(h);
    delete h;
}

}  // extern "C"
