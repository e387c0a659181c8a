// ph_save / ph_load: the offline stage is the expensive part (minutes at large n),
// so a built handle can be written to a file and mapped back onto a device.
// Format: a magic word, the options, the plan, every host array and every
// stored device arena, all little-endian binary.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace {

const char kMagic[8] = {'P', 'H', 'L', 'I', 'B', '0', '0', '5'};  // 005: near sharing, near grid, compressor
constexpr int kArenas = 9;  // near, near theta, far, far theta, S/T, U, E, L/R, tensor-core R (this order)

struct Writer {
    FILE* f;
    void raw(const void* p, size_t n) {
        if (n && fwrite(p, 1, n, f) != n) throw ph::Error(PH_ERR_IO, "write failed");
    }
    template <typename T> void val(const T& v) { raw(&v, sizeof(T)); }
    template <typename T> void vec(const std::vector<T>& v) {
        unsigned long long n = v.size();
        val(n);
        raw(v.data(), n * sizeof(T));
    }
    void dev(const void* p, size_t bytes) {
        std::vector<unsigned char> tmp(bytes);
        if (bytes) PH_CUDA(cudaMemcpy(tmp.data(), p, bytes, cudaMemcpyDeviceToHost));
        vec(tmp);
    }
};

struct Reader {
    FILE* f;
    unsigned long long left = 0;  // bytes not yet read
    explicit Reader(FILE* file) : f(file) {
        if (fseek(f, 0, SEEK_END) == 0) {
            const long end = ftell(f);
            left = end > 0 ? (unsigned long long)end : 0ull;
        }
        fseek(f, 0, SEEK_SET);
    }
    void raw(void* p, size_t n) {
        if (n > left || (n && fread(p, 1, n, f) != n)) throw ph::Error(PH_ERR_IO, "truncated file");
        left -= n;
    }
    template <typename T> void val(T& v) { raw(&v, sizeof(T)); }
    template <typename T> void vec(std::vector<T>& v) {
        unsigned long long n = 0;
        val(n);
        // a length the rest of the file cannot hold is corrupt: refuse it before allocating
        if (n > left / sizeof(T)) throw ph::Error(PH_ERR_IO, "corrupt file");
        v.resize(n);
        raw(v.data(), n * sizeof(T));
    }
};

template <typename IO, typename P>
void plan_io(IO& io, P& plan) {
    io.val(plan.d);
    io.val(plan.n);
    io.val(plan.depth);
    io.vec(plan.perm);
    io.vec(plan.leaves);
    io.vec(plan.near_s);
    io.vec(plan.near_t);
    io.vec(plan.far_s);
    io.vec(plan.far_t);
    io.vec(plan.far_key);
    io.vec(plan.key_rep);
    io.vec(plan.near_by_leaf);
    io.vec(plan.far_targets);
    io.vec(plan.far_by_target);
}

template <typename IO, typename H>
void scalars_io(IO& io, H& h) {
    io.val(h.kernel);
    io.val(h.opts);
    io.val(h.PD);
    io.val(h.Delta);
    io.val(h.p_theta_total);
    io.val(h.p_theta_near_total);
    io.val(h.scalar);
    io.val(h.offline_seconds);
    io.vec(h.nb_rank);
    io.vec(h.nb_off);
    io.vec(h.nb_toff);
    io.vec(h.nb_woff);
    io.vec(h.key_ranks);
    io.vec(h.key_off);
    io.vec(h.key_hoff);
    io.vec(h.fb_soff);
    io.vec(h.fb_toff);
    io.vec(h.key_lroff);
    io.val(h.lr_elems);
    io.vec(h.key_tcoff);
    io.val(h.tc_elems);
    io.val(h.near_elems);
    io.val(h.near_theta_elems);
    io.val(h.far_elems);
    io.val(h.far_theta_elems);
    io.val(h.H_elems);
    io.val(h.st_elems);
    io.val(h.w_elems);
    io.vec(h.theta_nodes);
    io.vec(h.theta_bw);
    io.vec(h.E64);
}

}  // namespace

extern "C" ph_status ph_save(const ph_handle* hc, const char* path) {
    if (!hc || !path) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_save: NULL argument");
    ph_handle* h = const_cast<ph_handle*>(hc);
    FILE* f = fopen(path, "wb");
    if (!f) {
        h->last_error = std::string("cannot open ") + path;
        return PH_ERR_IO;
    }
    try {
        PH_CUDA(cudaSetDevice(h->device));
        PH_CUDA(cudaDeviceSynchronize());
        Writer w{f};
        w.raw(kMagic, 8);
        scalars_io(w, *h);
        plan_io(w, h->plan);
        unsigned long long nn = h->plan.nodes.size();
        w.val(nn);
        for (const auto& nd : h->plan.nodes) {
            w.val(nd.level); w.val(nd.parent); w.val(nd.halves); w.val(nd.begin); w.val(nd.end); w.val(nd.leaf);
            w.raw(nd.lo, sizeof(nd.lo)); w.raw(nd.hi, sizeof(nd.hi));
            w.vec(nd.children);
        }
        const size_t sc = h->scalar;
        w.dev(h->d_near, h->near_elems * sc);
        w.dev(h->d_near_theta, h->near_theta_elems * 8);
        w.dev(h->d_far, h->far_elems * sc);
        w.dev(h->d_far_theta, h->far_theta_elems * 8);
        w.dev(h->d_st, h->st_elems * sc);
        w.dev(h->d_U, (size_t)h->plan.n * h->plan.d * h->opts.p_s * sc);
        w.dev(h->d_E, (size_t)2 * h->opts.p_s * h->opts.p_s * sc);
        w.dev(h->d_lr, h->lr_elems * sc);
        w.dev(h->d_tc, h->tc_elems * 4);
    } catch (const ph::Error& e) {
        fclose(f);
        h->last_error = e.what();
        return e.status;
    }
    if (fclose(f) != 0) return PH_ERR_IO;
    return PH_OK;
}

extern "C" ph_status ph_load(const char* path, int device, ph_handle** out) {
    if (!path || !out) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_load: NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return ph::fail(nullptr, PH_ERR_IO, std::string("cannot open ") + path);
    ph_handle* h = nullptr;
    try {
        h = new ph_handle();
    } catch (...) {
        fclose(f);
        return ph::fail(nullptr, PH_ERR_OOM, "host allocation failed");
    }
    // everything is read and checked on the host before the device is touched
    ph_status st = ph::guarded(nullptr, [&]() -> ph_status {
        Reader r(f);
        char magic[8];
        r.raw(magic, 8);
        if (std::memcmp(magic, kMagic, 8) != 0) throw ph::Error(PH_ERR_IO, "not a libph file of this version");
        scalars_io(r, *h);
        h->device = device;
        h->opts.device = device;
        plan_io(r, h->plan);
        unsigned long long nn = 0;
        r.val(nn);
        // a node takes at least its fixed fields: refuse a count the file cannot hold
        if (nn > r.left / (6 * sizeof(int) + 6 * sizeof(double) + 8)) throw ph::Error(PH_ERR_IO, "corrupt file");
        h->plan.nodes.resize(nn);
        for (auto& nd : h->plan.nodes) {
            r.val(nd.level); r.val(nd.parent); r.val(nd.halves); r.val(nd.begin); r.val(nd.end); r.val(nd.leaf);
            r.raw(nd.lo, sizeof(nd.lo)); r.raw(nd.hi, sizeof(nd.hi));
            r.vec(nd.children);
        }
        std::vector<std::vector<unsigned char>> arenas(kArenas);
        std::vector<size_t> sizes(kArenas);
        for (int i = 0; i < kArenas; ++i) {
            r.vec(arenas[i]);
            sizes[i] = arenas[i].size();
        }
        if (r.left != 0) throw ph::Error(PH_ERR_IO, "trailing bytes after the last arena");
        ph::near_mirror_map(h);
        ph::validate_handle(*h, sizes);

        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
            cudaGetLastError();
            throw ph::Error(PH_ERR_CUDA, "no CUDA device " + std::to_string(device));
        }
        PH_CUDA(cudaSetDevice(device));
        // the far-field chain is the longer path of a matvec: its stream gets the highest priority so
        // its blocks are scheduled ahead of the near-field blocks that fill the remaining SM slots
        {
            int lo = 0, hi = 0;
            PH_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            PH_CUDA(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi));
        }
        PH_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        PH_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        void** dst[kArenas] = {&h->d_near, (void**)&h->d_near_theta, &h->d_far, (void**)&h->d_far_theta,
                               &h->d_st,   &h->d_U,                  &h->d_E,   &h->d_lr,
                               &h->d_tc};
        for (int i = 0; i < kArenas; ++i) {
            *dst[i] = ph::dev_alloc(h, arenas[i].size());
            if (!arenas[i].empty())
                PH_CUDA(cudaMemcpy(*dst[i], arenas[i].data(), arenas[i].size(), cudaMemcpyHostToDevice));
        }
        h->d_H = ph::dev_alloc(h, (h->H_elems > 0 ? h->H_elems : 1) * h->scalar);
        h->d_w = ph::dev_alloc(h, (h->w_elems > 0 ? h->w_elems : 1) * h->scalar);
        ph::refresh_views(h);
        return PH_OK;
    });
    fclose(f);
    if (st != PH_OK) {
        ph::free_device(h);
        delete h;
        return st;
    }
    *out = h;
    return PH_OK;
}
