// The handle behind the opaque ph_handle pointer, and the device views the
// online kernels receive.
#pragma once

#include <cuda_runtime.h>

#include <new>
#include <stdexcept>
#include <string>
#include <functional>
#include <vector>

#include "common.cuh"
#include "ph_internal.h"

// Device pointers of the online stage for compute type T (float or double).
// Passed by value to kernels.
template <typename T>
struct DevView {
    // geometry / tree
    int n, d, p_s, PD;          // PD = p_s^d
    int n_leaves, n_nodes;
    const int* perm;            // cluster position -> original index
    const int* node_begin;      // per node
    const int* node_end;
    const int* node_halves;
    const int* node_children;   // CSR over nodes
    const int* node_child_off;
    const int* leaf_node;       // leaf -> node id
    const int* node_leaf;       // node -> leaf index or -1
    const int* node_parent;     // parent node id, -1 at the root
    // theta
    int dtheta;
    int p_theta[3];
    const double* theta_nodes;  // dtheta x 32 (far-field grid)
    const double* theta_bw;     // barycentric weights, dtheta x 32
    const double* theta_nodes_near;  // the near-field grid's nodes and weights, dtheta x 32 each
    const double* theta_bw_near;
    int p_theta_near[3];
    double* v64;                // instantiated parametric vectors, dtheta x 32
    // near field
    int n_near;
    const int* near_by_leaf;    // CSR over leaves
    const int* nb_t;            // source node of each near block
    const int* nb_s;            // target leaf node of each near block
    const int* nb_rank;
    const long long* nb_off;    // element offset of G_{b,1} (r slabs of n_s x n_t) in near_cores
    const long long* nb_toff;   // offset of the theta cores in near_theta (FP64)
    const int* nb_woff;         // offset of w_b in w
    const T* near_cores;        // G_{b,1}, column-interleaved: (i, j, slab k) at [(j r + k) n_s + i]
    const double* near_theta;
    T* w;                       // instantiated near weights
    int n_items;                // near work items: runs of consecutive near blocks of one target leaf
    const int* item_first;
    const int* item_count;
    const int* item_leaf;
    const int* items_by_leaf;   // CSR over leaves
    int part_stride;            // rows per item in the partial buffer (max leaf size)
    T* partials;                // (n_items + n_mslots) x part_stride x mcap
    // mirror sharing: a stored block (s, t) with s != t also gives D_ts = D_st^T, whose product
    // D_st^T x_s lands in partial slot n_items + nb_mslot[b] (-1: no mirror); the mirror slots of
    // a leaf t are the contiguous range [mirror_by_leaf[t], mirror_by_leaf[t + 1])
    int near_share;
    int n_mslots;
    const int* nb_mslot;
    const int* mirror_by_leaf;
    const int* mslot_block;     // the stored block of each mirror slot
    // far field
    int n_keys, Delta;
    const int* key_ranks;       // (Delta + 1) per key
    const long long* key_off;   // Delta per key: element offset of each core (spatial cores in far_cores,
                                // theta cores in far_theta)
    const long long* key_hoff;  // offset of H_k in H
    const T* far_cores;
    const double* far_theta;
    T* H;
    T* HT;                      // H_k^T per class at the same offsets (written when the adjoint is set up)
    const T* far_lr;            // explicit L_k^T (r_d x PD) then R_k^T (r_{d+1} x PD) per key, row-major
    const long long* key_lroff; // offset of L_k^T in far_lr (R_k^T follows)
    const int* kb_off;          // CSR over keys: far blocks of each key
    const int* kb_list;
    int n_citems;               // key-grouped work items of the explicit coupling
    const int* citem_key;
    const int* citem_first;     // index into kb_list
    const int* citem_count;
    const float* far_tc;        // R_k^T for tcgen05: per key, per 32-chunk of J, TF32 high then low part
    const long long* key_tcoff;
    int n_tcitems;              // key-grouped items of 8 blocks (tensor-core phase 1)
    const int* tcitem_key;
    const int* tcitem_first;
    const int* tcitem_count;
    int zstride;                // rows per far block in zbuf (max r_d)
    T* zbuf;                    // n_far x zstride x mcap: z_b = H_k R_k^T xhat_t
    int n_far;
    const int* fb_t;            // source node per far block
    const int* fb_key;
    int n_far_targets;
    int far_max_target;         // largest target node (host use: shared memory of the H-format kernel)
    const int* far_targets;     // target node ids
    const int* far_by_target;   // CSR over far_targets
    // H format
    const long long* fb_soff;   // S_b offset in st
    const long long* fb_toff;   // T_b offset in st
    const T* st;
    const int* node_level;
    int n_far_levels;
    const int* level_slot;      // level -> slot in yfar, -1 if no far targets on that level
    // bases
    const T* U;                 // n x d x p_s (cluster order)
    const T* E;                 // 2 x p_s x p_s: E_lo then E_hi, [j * p_s + i] = ell_i^{parent}(eta_j^{child})
    // workspace
    int mcap;
    T* Xc;                      // n x mcap, cluster order, row-major
    T* yfar;                    // n_far_levels x n x mcap (H format)
    T* xhat;                    // n_nodes x PD x mcap
    T* yhat;
    int* flags;                 // [0]: non-finite input count, [1]: bounded device waits that ran out
};

struct DeviceBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

namespace ph {
struct Surrogate;  // surrogate.cu
}

struct ph_handle {
    // configuration
    ph_kernel kernel = PH_KERNEL_GAUSS;
    ph_build_opts opts{};
    int device = 0;
    int num_sms = 1;  // streaming multiprocessors of the device (persistent grids)
    int PD = 0, Delta = 0, p_theta_total = 1, p_theta_near_total = 1;
    size_t scalar = 8;  // sizeof compute type
    ph::Plan plan;
    double offline_seconds = 0;
    std::string last_error;
    // host copies of everything stored (for ph_save and ph_get_info)
    std::vector<int> nb_rank;
    std::vector<long long> nb_off, nb_toff;
    std::vector<int> nb_woff;
    std::vector<int> key_ranks;
    std::vector<long long> key_off, key_hoff;
    std::vector<long long> fb_soff, fb_toff;
    std::vector<long long> key_lroff, key_tcoff;
    long long tc_elems = 0;
    void* d_tc = nullptr;
    std::vector<int> tcitem_key, tcitem_first, tcitem_count;
    long long lr_elems = 0;
    void* d_lr = nullptr;
    std::vector<int> kb_off, kb_list, citem_key, citem_first, citem_count;
    int zstride = 1;
    int rank_max_lr = 1;                        // max over keys of r_d and r_{d+d_theta}
    void* d_zbuf = nullptr;
    long long near_elems = 0, near_theta_elems = 0, far_elems = 0, far_theta_elems = 0, H_elems = 0,
              st_elems = 0, w_elems = 0;
    std::vector<double> theta_nodes, theta_bw;  // 2 x 3 x 32: far-field grid, then near-field grid
    std::vector<double> E64;                    // 2 x p_s x p_s
    // device data
    std::vector<DeviceBuffer> buffers;          // every device allocation, freed in ph_destroy
    void* d_near = nullptr;
    double* d_near_theta = nullptr;
    void* d_far = nullptr;
    double* d_far_theta = nullptr;
    void* d_st = nullptr;
    void* d_U = nullptr;
    void* d_E = nullptr;
    void* d_w = nullptr;
    void* d_H = nullptr;
    double* d_v64 = nullptr;
    int* d_flags = nullptr;
    int* d_int = nullptr;                       // packed integer index arrays
    long long* d_ll = nullptr;                  // packed 64-bit offset arrays
    double* d_dbl = nullptr;                    // theta nodes / weights
    // workspace, sized for mcap right-hand sides
    int mcap = 0;
    void* d_Xc = nullptr;
    void* d_ynodes = nullptr;                   // K_hat(eta_q) X at the theta nodes (ph_matvec_batched)
    size_t ynodes_bytes = 0;
    double* d_thetas = nullptr;                 // the theta values of a batched call
    size_t thetas_cap = 0;
    void* d_yfar = nullptr;
    void* d_xhat = nullptr;
    void* d_yhat = nullptr;
    void* d_partials = nullptr;
    std::vector<int> item_first, item_count, item_leaf, items_by_leaf;
    int max_leaf = 1;
    // mirror sharing of near blocks (§4.3 with a symmetric kernel): nb_src[b] is the block whose
    // stored cores b uses (b itself, or the block (t, s) when b = (s, t) is the mirrored one)
    int near_share = 0;
    std::vector<int> nb_src, nb_mslot, mirror_by_leaf, mslot_block;
    int n_mslots = 0;
    int coupling_zmax = 1;                      // longest shared-memory intermediate of the TT chain
    DeviceBuffer ws;
    DeviceBuffer host_stage_x, host_stage_y;    // device staging for ph_matvec_host
    int n_far_levels = 0;
    std::vector<int> level_slot;
    std::vector<std::vector<int>> level_nodes;  // nodes per level (for the sweeps)
    int* d_level_nodes = nullptr;
    std::vector<int> level_nodes_off;
    int min_far_level = 0;
    std::vector<char> level_has_inner_child;    // level -> some node on it has a non-leaf child
    // streams
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_thetas = nullptr;            // after the last copy out of host_thetas_pinned
    int* host_flags = nullptr;                  // pinned copy of flags[1], written at the end of each matvec
    int seen_timeouts = 0;                      // flags[1] already reported as PH_ERR_TIMEOUT
    double* host_thetas_pinned = nullptr;       // pinned source of a batched call's theta copy
    size_t host_thetas_cap = 0;
    // adjoint K_hat^T (ph_matvec_transpose): far blocks with targets and sources swapped and the
    // classes' factors exchanged (L' = R_k, R' = L_k, H' = H_k^T), built on first use
    bool adj_ready = false;
    int* d_adj_int = nullptr;
    long long* d_adj_ll = nullptr;
    void* d_lrT = nullptr;
    void* d_HT = nullptr;
    int zstride_adj = 1;
    std::vector<long> adj_io, adj_lo;
    int adj_n_targets = 0, adj_max_target = 1, adj_n_citems = 0;
    DevView<float> vfT{};
    DevView<double> vdT{};
    bool instantiated = false;
    // learned surrogate of the far-field cores (surrogate.cu); null until ph_surrogate_train or
    // ph_far_project
    ph::Surrogate* sur = nullptr;
    bool overlap = true;                        // far path on the side stream (ph_set_overlap)
    bool use_bulk = true;                       // bulk-copy pipelined near field and phase 2 when they apply
    int last_variants = 0;                      // kernels the last ph_matvec chose (ph_info.kernel_variants)
    int near_rank_max = 0;                      // max near-block rank
    bool use_tc = false;                        // tensor-core phase 1 when available (ph_set_tensor_cores)
    // per-kernel timing (ph_profile_enable / ph_profile_read)
    bool prof = false;
    std::vector<cudaEvent_t> prof_pool;
    struct ProfRec { int kind; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_recs;
    // index views (into d_int / d_ll)
    std::vector<long> view_io, view_lo;
    DevView<float> vf{};
    DevView<double> vd{};
};

namespace ph {
// offline.cu
ph_status offline_build(ph_handle* h, const double* points, long n);
// online.cu
ph_status online_instantiate(ph_handle* h, const double* theta, cudaStream_t stream, int deriv = -1);
// the near-field part of the online stage only (w_b for every near block)
void online_instantiate_near(ph_handle* h, const double* theta, cudaStream_t stream);
// far-field cores from the surrogate network at theta into H (surrogate.cu); false if not in use
bool surrogate_instantiate_far(ph_handle* h, const double* theta, cudaStream_t stream);
void surrogate_free(ph_handle* h);
ph_status online_matvec_batched(ph_handle* h, const double* thetas, int n_theta, const void* X, long ldx, int m,
                                void* Y, long ldy, long stride_y, int deriv, cudaStream_t stream);
ph_status wait_bound_selftest(int device, double* waited);  // bounded mbarrier wait on a barrier nothing completes
ph_status handle_timeout_selftest(ph_handle* h, cudaStream_t stream);  // the same wait, counted in h's flags
ph_status online_matvec(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy,
                        cudaStream_t stream);
// X = K_hat(theta)^T Y (the adjoint): near blocks transposed, far field through the transposed view.
ph_status online_matvec_transpose(ph_handle* h, const void* Y, long ldy, int m, void* X, long ldx,
                                  cudaStream_t stream);
// Builds the transposed far view (adjoint.cpp) and H_k^T of the current instantiation.
void build_adjoint(ph_handle* h, cudaStream_t stream);
void refresh_transposed(ph_handle* h);  // the transposed views after the forward views changed
void transpose_H(ph_handle* h, cudaStream_t stream);  // online.cu: H_k^T of the current H
void ensure_workspace(ph_handle* h, int m);
// ph_matvec with the caller's device views (their workspace pointers replace the handle's).
ph_status online_matvec_view(ph_handle* h, DevView<float>& vf, DevView<double>& vd, const void* X, long ldx, int m,
                             void* Y, long ldy, cudaStream_t stream);
void refresh_views(ph_handle* h);
// h->near_share and h->nb_src from the options and the plan's near blocks (throws PH_ERR_IO when a
// block's mirror is missing)
void near_mirror_map(ph_handle* h);
void free_device(ph_handle* h);
void* dev_alloc(ph_handle* h, size_t bytes);  // throws ph::Error(PH_ERR_OOM) on failure
// Test hook behind ph_inject_alloc_failure: after `after` more successful dev_alloc calls in
// this process every further one fails with PH_ERR_OOM (after < 0 switches it off).
void set_alloc_failure(long after);
// Stream-ordered copy of the device wait-timeout counter into pinned host memory (no sync).
void post_timeout_flag(ph_handle* h, cudaStream_t stream);
// PH_ERR_TIMEOUT (once) when a bounded device wait of an earlier call ran out, else PH_OK.
ph_status take_timeout(ph_handle* h);
// TT-SVD truncation rank at one cut (offline.cu): smallest r >= 1 whose discarded tail is at
// most delta2, then the cap (0: none), then numerically tied singular values kept together.
int choose_rank_sv(const double* s, int n, double delta2, int cap);
// ttcross_host.cpp: greedy TT-cross of a tensor given entry-wise, then TT-rounding (cores Fortran
// (r_k, n_k, r_{k+1}), ranks r_0..r_q); returns the number of distinct entries evaluated
long long tt_cross_round(const std::vector<int>& dims, const std::function<double(const int*)>& f, double eps, int cap,
                         unsigned long long seed, std::vector<std::vector<double>>& cores, std::vector<int>& ranks);
double kappa_host(int kernel, const double* x, const double* y, const double* th, int d);
long long far_cross(int kernel, int d, int dt, int ps, const int* pt, const double* s_lo, const double* s_hi,
                    const double* t_lo, const double* t_hi, const double* theta_nodes, double eps, int cap,
                    unsigned long long seed, std::vector<std::vector<double>>& cores, std::vector<int>& ranks);
// Host FP64 thin SVD of a small m x n column-major matrix, s descending (ttsvd_host.cpp).
void svd_small(int m, int n, const std::vector<double>& A, std::vector<double>& U, std::vector<double>& s,
               std::vector<double>& Vt);
// The r x P matrix that turns the tensor product of the parametric vectors into the near weights
// w_b, from the first TT cut (s, V_r) and the remaining cuts (ttsvd_host.cpp).
std::vector<double> near_theta_matrix(const double* s, const double* Vr, int P, int r, const int* pt, int dt,
                                      double delta2);
// Checks every offset, index and size the kernels rely on (ph_load refuses a file that fails,
// ph_offline_build checks what it built); throws ph::Error(PH_ERR_IO) with the first violation.
void validate_handle(const ph_handle& h, const std::vector<size_t>& arena_bytes);
// Records msg as the last error (of h, and of the thread) and returns s.
ph_status fail(ph_handle* h, ph_status s, const std::string& msg);
// Runs f and maps any exception to a status recorded by fail().
template <typename F>
ph_status guarded(ph_handle* h, F&& f) {
    try {
        return f();
    } catch (const Error& e) {
        return fail(h, e.status, e.what());
    } catch (const std::bad_alloc&) {
        return fail(h, PH_ERR_OOM, "host allocation failed");
    } catch (const std::invalid_argument& e) {
        return fail(h, PH_ERR_INVALID_ARG, e.what());
    } catch (const std::exception& e) {
        return fail(h, PH_ERR_CUDA, e.what());
    } catch (...) {
        return fail(h, PH_ERR_CUDA, "unknown exception");
    }
}
void dev_free(ph_handle* h, void* p);
// NVTX range for tools (nsys, ncu --nvtx); a no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
// NVTX range named for the launch's kind, and an event pair around the launch when profiling
// is on.
struct ProfScope {
    ph_handle* h;
    int kind;
    cudaStream_t s;
    cudaEvent_t b = nullptr;
    ProfScope(ph_handle* h_, int kind_, cudaStream_t s_);
    ~ProfScope();
};
}  // namespace ph
