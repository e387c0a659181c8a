// ph_matvec_noalloc: ph_matvec for callers that must not allocate device memory.
//
// The per-call workspace of ph_matvec (X in cluster order, the near-field partial sums, the
// up- and down-sweep coefficients or the H-format level buffers) normally lives in buffers
// the handle allocates on first use.  This entry point instead carves it out of one
// file-scope device array of kNoAllocScratchBytes, so the call itself performs no cudaMalloc,
// cudaFree or allocating library call.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "handle.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB on every device that loads libph
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `dev` (which must be current).  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per device.
void* scratch_address(int dev) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        PH_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" ph_status ph_matvec_noalloc(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy,
                                       void* stream) {
    if (!h) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_matvec_noalloc: NULL handle");
    if (!X || !Y || m < 1 || m > 1024 || ldx < h->plan.n || ldy < h->plan.n)
        return ph::fail(h, PH_ERR_INVALID_ARG, "ph_matvec_noalloc: invalid argument");
    if (!h->instantiated) return ph::fail(h, PH_ERR_NOT_INSTANTIATED, "ph_matvec_noalloc before ph_instantiate");
    if (h->device < 0 || h->device >= kMaxDevices)
        return ph::fail(h, PH_ERR_INVALID_ARG, "ph_matvec_noalloc: device ordinal out of range");
    if (ph::take_timeout(h) != PH_OK) return PH_ERR_TIMEOUT;
    return ph::guarded(h, [&]() -> ph_status {
        const int mc = (m <= 1) ? 1 : (m <= 2) ? 2 : (m <= 4) ? 4 : (m <= 8) ? 8 : 16;
        const size_t S = (size_t)ph::ceil_div(m, mc) * mc;
        const size_t sc = h->scalar, n = (size_t)h->plan.n;
        const size_t items = std::max<size_t>(1, h->item_first.size() + h->n_mslots);  // item and mirror slots
        const bool h2 = (h->opts.fmt == PH_FMT_H2) && !h->plan.far_targets.empty();
        const bool hfar = (h->opts.fmt == PH_FMT_H) && h->n_far_levels > 0;
        // layout of the scratch array: Xc | partials | xhat | yhat | zbuf (H^2)  or  Xc | partials | yfar (H)
        const size_t o_xc = 0;
        const size_t o_part = align256(o_xc + n * S * sc);
        const size_t o_xhat = align256(o_part + items * h->max_leaf * S * sc);
        const size_t node_bytes = h2 ? h->plan.nodes.size() * (size_t)h->PD * S * sc : 0;
        const size_t o_yhat = align256(o_xhat + node_bytes);
        const size_t o_yfar = align256(o_yhat + node_bytes);
        const size_t o_zbuf = align256(o_yfar + (hfar ? (size_t)h->n_far_levels * n * S * sc : 0));
        const bool zb = h2 && h->opts.coupling == 0;
        const size_t need = o_zbuf + (zb ? h->plan.far_s.size() * (size_t)h->zstride * S * sc : 0);
        if (need > kNoAllocScratchBytes)
            return ph::fail(h, PH_ERR_INVALID_ARG,
                            "ph_matvec_noalloc: this problem needs " + std::to_string(need) +
                                " bytes of scratch; the limit is " + std::to_string(kNoAllocScratchBytes) +
                                " bytes (use ph_matvec)");
        PH_CUDA(cudaSetDevice(h->device));
        unsigned char* base = static_cast<unsigned char*>(scratch_address(h->device));
        DevView<float> vf = h->vf;
        DevView<double> vd = h->vd;
        auto place = [&](auto& v) {
            using T = std::remove_pointer_t<decltype(v.Xc)>;
            v.Xc = reinterpret_cast<T*>(base + o_xc);
            v.partials = reinterpret_cast<T*>(base + o_part);
            v.xhat = h2 ? reinterpret_cast<T*>(base + o_xhat) : nullptr;
            v.yhat = h2 ? reinterpret_cast<T*>(base + o_yhat) : nullptr;
            v.yfar = hfar ? reinterpret_cast<T*>(base + o_yfar) : nullptr;
            v.zbuf = zb ? reinterpret_cast<T*>(base + o_zbuf) : nullptr;
            v.mcap = (int)S;
        };
        place(vf);
        place(vd);
        return ph::online_matvec_view(h, vf, vd, X, ldx, m, Y, ldy, reinterpret_cast<cudaStream_t>(stream));
    });
}
