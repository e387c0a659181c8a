// Offline stage of the parametric H / H^2 matrix (Algs. "Offline Stage: Parametric
// H-matrix" and "... H^2-matrix", §4.4), in FP64 on the GPU.
//
//  * near field (§4.3): A_b[(i,j), k] = kappa(x_{s,i}, x_{t,j}; eta_k) is never stored.
//    One kernel reduces A_b to its triangular factor R_b by Householder QR over
//    row chunks generated on the fly (R <- qr([R; A_chunk])), cuSOLVER's batched
//    Jacobi SVD gives R_b = U S V^T for all blocks at once, and a second kernel
//    re-evaluates A_b and writes G_{b,1} = A_b V_r (r slabs of n_s x n_t, i
//    fastest) with G_{b,2} = V_r^T: the truncated SVD of TT-SVD's single cut for
//    d_theta = 1, in the gauge U_r S_r / V_r^T.
//  * far field (§4.2, App. A.4): M_b on the Chebyshev grids, compressed by
//    TT-SVD (Oseledets 2011, Alg. 1); each cut is a QR of the tall side of the
//    unfolding (cuSOLVER geqrf) followed by an SVD of its square factor
//    (cuSOLVER gesvd), so singular values carry absolute error eps ||A|| and the
//    truncation matches a dense SVD; one tensor per translation class
//    (level, offset) when the kernel is translation-invariant (§5.2).
//  * H format: S_b = U_s L_b and T_b = U_t R_b by the recurrences of Phase 3 of
//    the PTTK offline algorithm (App. A.4), on the host in FP64.
//  * H^2 format: leaf factor matrices U_{s,k} (§3.3) and the two transfer
//    factors of a midpoint split (§3.6.1).
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace ph {

namespace {

#define PH_BLAS(call)                                                                         \
    do {                                                                                      \
        cublasStatus_t st_ = (call);                                                          \
        if (st_ != CUBLAS_STATUS_SUCCESS)                                                     \
            throw Error(PH_ERR_CUDA, std::string("cuBLAS: ") + #call + " status " +          \
                                         std::to_string((int)st_));                           \
    } while (0)
#define PH_SOLVER(call)                                                                       \
    do {                                                                                      \
        cusolverStatus_t st_ = (call);                                                        \
        if (st_ != CUSOLVER_STATUS_SUCCESS)                                                   \
            throw Error(PH_ERR_CUDA, std::string("cuSOLVER: ") + #call + " status " +        \
                                         std::to_string((int)st_));                           \
    } while (0)

constexpr double kTieRel = 1e-9;

// kappa(x, y; theta) in FP64 for the kernels of include/ph.h.
__device__ __forceinline__ double kappa64(int kernel, const double* x, const double* y,
                                          const double* th, int d) {
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double df = x[k] - y[k];
        r2 += df * df;
    }
    const double l = th[0];
    switch (kernel) {
        case PH_KERNEL_GAUSS: return exp(-r2 / (2.0 * l * l));
        case PH_KERNEL_MATERN32: {
            double s = sqrt(3.0) * sqrt(r2) / l;
            return (1.0 + s) * exp(-s);
        }
        case PH_KERNEL_MATERN52: {
            double s = sqrt(5.0) * sqrt(r2) / l;
            return (1.0 + s + s * s / 3.0) * exp(-s);
        }
        case PH_KERNEL_ANISO_GAUSS: {
            double q = 0.0;
            for (int k = 0; k < d; ++k) {
                double df = x[k] - y[k];
                q += df * df / (2.0 * th[k] * th[k]);
            }
            return exp(-q);
        }
        case PH_KERNEL_SE: return exp(-r2 / (l * l));
        case PH_KERNEL_EXPONENTIAL: return exp(-sqrt(r2) / l);
        case PH_KERNEL_MULTIQUADRIC: return sqrt(1.0 + r2 / (l * l));
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

struct NearBuild {
    int kernel, d, P, dt;
    const double* pts;       // cluster order, n x d
    const int* s_begin;      // per near block
    const int* s_n;
    const int* t_begin;
    const int* t_n;
    const double* grid;      // P x dt theta grid points (k fastest over dimension 1)
};

constexpr int kChunk = 256;

// Fills A[row][k] for rows q0 .. q0 + chunk - 1 of block b into shared memory.
__device__ void eval_near_chunk(const NearBuild& a, int b, long long q0, long long nq, double* A, int chunk = kChunk) {
    const int ns = a.s_n[b];
    const int sb = a.s_begin[b], tb = a.t_begin[b];
    for (int row = threadIdx.x; row < chunk; row += blockDim.x) {
        long long q = q0 + row;
        if (q < nq) {
            int i = (int)(q % ns), j = (int)(q / ns);  // (i, j) little-endian, i fastest (§4.3)
            double x[kMaxDim], y[kMaxDim];
            for (int k = 0; k < a.d; ++k) {
                x[k] = a.pts[(long long)(sb + i) * a.d + k];
                y[k] = a.pts[(long long)(tb + j) * a.d + k];
            }
            for (int k = 0; k < a.P; ++k) A[row * a.P + k] = kappa64(a.kernel, x, y, a.grid + k * a.dt, a.d);
        } else {
            for (int k = 0; k < a.P; ++k) A[row * a.P + k] = 0.0;
        }
    }
}

// Triangular factor R_b (P x P, column-major, upper) of every near block A_b, one CTA per block:
// the rows of A_b are generated in chunks and folded in by Householder QR of the stacked
// matrix [R; A_chunk] (LAPACK dlarfg convention).  Only R is kept: the right singular
// vectors and singular values of A_b are those of R_b.
__global__ void near_tsqr_kernel(NearBuild a, double* Rout, int chunk) {
    extern __shared__ double sm[];
    const int P = a.P, LD = P + chunk;
    double* W = sm;                 // LD x P, column-major: rows 0..P-1 hold R, rows P.. the chunk
    double* A = sm + (size_t)LD * P; // chunk x P row-major scratch for the evaluation
    const int b = blockIdx.x;
    const long long nq = (long long)a.s_n[b] * a.t_n[b];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) W[(e % P) + LD * (e / P)] = 0.0;
    for (long long q0 = 0; q0 < nq; q0 += chunk) {
        __syncthreads();
        eval_near_chunk(a, b, q0, nq, A, chunk);
        __syncthreads();
        for (int e = threadIdx.x; e < chunk * P; e += blockDim.x) {
            const int row = e / P, k = e % P;
            W[P + row + LD * k] = A[e];
        }
        __syncthreads();
        for (int k = 0; k < P; ++k) {
            // every warp recomputes the reflector of column k (column k is read-only in this step)
            double x2 = 0.0;
            for (int row = lane; row < chunk; row += 32) {
                double x = W[P + row + LD * k];
                x2 += x * x;
            }
            for (int o = 16; o > 0; o >>= 1) x2 += __shfl_xor_sync(0xffffffffu, x2, o);
            const double alpha = W[k + LD * k];
            if (x2 > 0.0) {
                const double beta = -copysign(sqrt(alpha * alpha + x2), alpha);
                const double tau = (beta - alpha) / beta;
                const double scale = 1.0 / (alpha - beta);
                for (int j = k + 1 + warp; j < P; j += nwarps) {
                    double w = 0.0;
                    for (int row = lane; row < chunk; row += 32) w += W[P + row + LD * k] * scale * W[P + row + LD * j];
                    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                    w += W[k + LD * j];
                    const double tw = tau * w;
                    for (int row = lane; row < chunk; row += 32)
                        W[P + row + LD * j] -= tw * W[P + row + LD * k] * scale;
                    if (lane == 0) W[k + LD * j] -= tw;
                }
                __syncthreads();
                if (threadIdx.x == 0) W[k + LD * k] = beta;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int r = e % P, c = e / P;
        Rout[(long long)b * P * P + e] = (r <= c) ? W[r + LD * c] : 0.0;
    }
}

// G_{b,1} = A_b V_r in compute type T, stored column-interleaved: entry (i, j) of slab c at
// [(j r + c) n_s + i], so that one column j of all r slabs is one contiguous run.  V_r of block
// b (P x r_b, column-major) at vecs + voff[b]; rows of A_b generated `chunk` at a time.
template <typename T>
__global__ void near_project_kernel(NearBuild a, const double* vecs, const long long* voff, const int* rank,
                                    const long long* off, T* out, int chunk) {
    extern __shared__ double sA[];
    double* sV = sA + (size_t)chunk * a.P;  // P x r_b, column-major
    const int b = blockIdx.x;
    const int r = rank[b];
    const long long nq = (long long)a.s_n[b] * a.t_n[b];
    const double* V = vecs + voff[b];
    for (int e = threadIdx.x; e < a.P * r; e += blockDim.x) sV[e] = V[e];
    T* G = out + off[b];
    for (long long q0 = 0; q0 < nq; q0 += chunk) {
        __syncthreads();
        eval_near_chunk(a, b, q0, nq, sA, chunk);
        __syncthreads();
        const int ns = a.s_n[b];
        for (int e = threadIdx.x; e < chunk * r; e += blockDim.x) {
            int row = e % chunk, c = e / chunk;
            long long q = q0 + row;
            if (q < nq) {
                double s = 0.0;
                for (int k = 0; k < a.P; ++k) s += sA[row * a.P + k] * sV[c * a.P + k];
                const long long i = q % ns, j = q / ns;
                G[(j * r + c) * ns + i] = (T)s;  // column-interleaved: (j, slab c, i)
            }
        }
    }
}

// A_b of the near blocks b0 .. b0 + nb - 1, each as a maxrows x P column-major matrix (rows
// (i, j) little-endian, i fastest, §4.3; rows past n_s n_t are zero, so A_b^T A_b is unchanged).
__global__ void near_form_kernel(NearBuild a, int b0, int nb, long long maxrows, double* out) {
    const long long total = (long long)nb * maxrows;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int bi = (int)(e / maxrows);
        const long long q = e % maxrows;
        const int b = b0 + bi;
        const int ns = a.s_n[b];
        const long long nq = (long long)ns * a.t_n[b];
        double* col = out + (long long)bi * maxrows * a.P + q;
        if (q >= nq) {
            for (int k = 0; k < a.P; ++k) col[maxrows * k] = 0.0;
            continue;
        }
        const int i = (int)(q % ns), j = (int)(q / ns);
        double x[kMaxDim], y[kMaxDim];
        for (int k = 0; k < a.d; ++k) {
            x[k] = a.pts[(long long)(a.s_begin[b] + i) * a.d + k];
            y[k] = a.pts[(long long)(a.t_begin[b] + j) * a.d + k];
        }
        for (int k = 0; k < a.P; ++k) col[maxrows * k] = kappa64(a.kernel, x, y, a.grid + k * a.dt, a.d);
    }
}

// M_b on the Chebyshev grids, modes (i_1..i_d, k_1..k_dt, j_1..j_d), little-endian (App. A.4).
__global__ void far_tensor_kernel(int kernel, int d, int dt, int ps, const int* pt, long long PD,
                                  long long PT, const double* sx, const double* tx,
                                  const double* tn, double* M) {
    const long long total = PD * PT * PD;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long i = idx % PD, rest = idx / PD;
        long long kk = rest % PT, j = rest / PT;
        double x[kMaxDim], y[kMaxDim], th[kMaxDim];
        for (int q = 0; q < d; ++q) {
            x[q] = sx[q * ps + (int)(i % ps)];
            y[q] = tx[q * ps + (int)(j % ps)];
            i /= ps;
            j /= ps;
        }
        for (int q = 0; q < dt; ++q) {
            th[q] = tn[q * kMaxPTheta + (int)(kk % pt[q])];
            kk /= pt[q];
        }
        M[idx] = kappa64(kernel, x, y, th, d);
    }
}


// Copies the upper triangle of the first n rows of T (ld m) into R (n x n), zeros below.
__global__ void copy_upper_kernel(const double* T, long long m, int n, double* R) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int r = e % n, c = e / n;
        R[e] = (r <= c) ? T[r + m * c] : 0.0;
    }
}

// TT-SVD on the device.  Each cut factors the tall side of the unfolding by Householder QR
// and takes the SVD of the square factor, so the singular values and the kept subspace have
// the accuracy of a dense SVD (absolute error ~ eps ||A||).
struct TTEngine {
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t solver = nullptr;
    double *C = nullptr, *Cn = nullptr, *T = nullptr, *tau = nullptr, *R = nullptr, *VT = nullptr, *V = nullptr, *Uw = nullptr,
           *S = nullptr, *work = nullptr, *rwork = nullptr;
    int* info = nullptr;
    size_t capT = 0, capN = 0, capWork = 0;
    ph_handle* h = nullptr;
    ~TTEngine() {
        if (blas) cublasDestroy(blas);
        if (solver) cusolverDnDestroy(solver);
    }

    void reserve(size_t total, size_t maxn) {
        if (total > capT) {
            C = (double*)dev_alloc(h, total * sizeof(double));
            Cn = (double*)dev_alloc(h, total * sizeof(double));
            T = (double*)dev_alloc(h, total * sizeof(double));
            capT = total;
        }
        if (maxn > capN) {
            R = (double*)dev_alloc(h, maxn * maxn * sizeof(double));
            VT = (double*)dev_alloc(h, maxn * maxn * sizeof(double));
            V = (double*)dev_alloc(h, maxn * maxn * sizeof(double));
            Uw = (double*)dev_alloc(h, maxn * maxn * sizeof(double));
            S = (double*)dev_alloc(h, maxn * sizeof(double));
            tau = (double*)dev_alloc(h, maxn * sizeof(double));
            rwork = (double*)dev_alloc(h, maxn * sizeof(double));
            capN = maxn;
        }
        if (!info) info = (int*)dev_alloc(h, sizeof(int));
    }

    void need_work(int lwork) {
        if ((size_t)lwork > capWork) {
            work = (double*)dev_alloc(h, (size_t)lwork * sizeof(double));
            capWork = lwork;
        }
    }

    void check_info(const char* what) {
        int hinfo = 0;
        PH_CUDA(cudaMemcpy(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost));
        if (hinfo != 0) throw Error(PH_ERR_CUDA, std::string(what) + " failed, info = " + std::to_string(hinfo));
    }

    // T (m x n, m >= n, destroyed) = Q R;  R = U_R S V_R^T.  Leaves V_R (n x n) in V and returns S.
    void qr_svd(long long m, int n, std::vector<double>& s) {
        int lwork = 0;
        PH_SOLVER(cusolverDnDgeqrf_bufferSize(solver, (int)m, n, T, (int)m, &lwork));
        need_work(lwork);
        PH_SOLVER(cusolverDnDgeqrf(solver, (int)m, n, T, (int)m, tau, work, lwork, info));
        check_info("geqrf");
        copy_upper_kernel<<<(n * n + 255) / 256, 256>>>(T, m, n, R);
        PH_LAUNCH("copy_upper_kernel");
        PH_SOLVER(cusolverDnDgesvd_bufferSize(solver, n, n, &lwork));
        need_work(lwork);
        PH_SOLVER(cusolverDnDgesvd(solver, 'N', 'A', n, n, R, n, S, Uw, n, VT, n, work, lwork, rwork, info));
        check_info("gesvd");
        const double one = 1.0, zero = 0.0;
        PH_BLAS(cublasDgeam(blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, &one, VT, n, &zero, V, n, V, n));
        s.resize(n);
        PH_CUDA(cudaMemcpy(s.data(), S, n * sizeof(double), cudaMemcpyDeviceToHost));
    }

    // TT-SVD of the tensor already in C (Fortran order, dims).  Returns host cores
    // (core k is r_k x dims[k] x r_{k+1}, Fortran) and the ranks r_0..r_q.
    void run(const std::vector<int>& dims, double eps, int cap, std::vector<std::vector<double>>& cores,
             std::vector<int>& ranks) {
        const int q = (int)dims.size();
        long long size = 1;
        for (int v : dims) size *= v;
        double nrm = 0.0;
        PH_BLAS(cublasDnrm2(blas, (int)size, C, 1, &nrm));
        const double delta2 = eps * eps * nrm * nrm / std::max(1, q - 1);
        cores.assign(q, {});
        ranks.assign(q + 1, 1);
        int rp = 1;
        std::vector<double> s;
        const double one = 1.0, zero = 0.0;
        for (int k = 0; k < q - 1; ++k) {
            const long long rows = (long long)rp * dims[k];
            const long long cols = size / rows;
            int r;
            if (rows <= cols) {
                // C^T = Q R, so C = R^T Q^T and the left singular vectors of C are V_R
                PH_BLAS(cublasDgeam(blas, CUBLAS_OP_T, CUBLAS_OP_N, (int)cols, (int)rows, &one, C, (int)rows, &zero,
                                    T, (int)cols, T, (int)cols));
                qr_svd(cols, (int)rows, s);
                r = choose_rank_sv(s.data(), (int)rows, delta2, cap);
                cores[k].resize(rows * r);
                PH_CUDA(cudaMemcpy(cores[k].data(), V, rows * r * sizeof(double), cudaMemcpyDeviceToHost));
                PH_BLAS(cublasDgemm(blas, CUBLAS_OP_T, CUBLAS_OP_N, r, (int)cols, (int)rows, &one, V, (int)rows, C,
                                    (int)rows, &zero, Cn, r));
            } else {
                // C = Q R = (Q U_R) S V_R^T: core = C V_r S_r^{-1}, remainder S_r V_r^T
                PH_CUDA(cudaMemcpy(T, C, size * sizeof(double), cudaMemcpyDeviceToDevice));
                qr_svd(rows, (int)cols, s);
                r = choose_rank_sv(s.data(), (int)cols, delta2, cap);
                PH_BLAS(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)rows, r, (int)cols, &one, C, (int)rows, V,
                                    (int)cols, &zero, T, (int)rows));
                std::vector<double> Vh(cols * r);
                PH_CUDA(cudaMemcpy(Vh.data(), V, cols * r * sizeof(double), cudaMemcpyDeviceToHost));
                cores[k].resize(rows * r);
                PH_CUDA(cudaMemcpy(cores[k].data(), T, rows * r * sizeof(double), cudaMemcpyDeviceToHost));
                std::vector<double> next(r * cols);
                for (int c = 0; c < r; ++c) {
                    const double inv = s[c] > 0 ? 1.0 / s[c] : 0.0;
                    for (long long row = 0; row < rows; ++row) cores[k][c * rows + row] *= inv;
                    for (long long col = 0; col < cols; ++col) next[c + r * col] = s[c] * Vh[c * cols + col];
                }
                PH_CUDA(cudaMemcpy(Cn, next.data(), next.size() * sizeof(double), cudaMemcpyHostToDevice));
            }
            std::swap(C, Cn);
            size = (long long)r * cols;
            rp = r;
            ranks[k + 1] = r;
        }
        cores[q - 1].resize(size);
        PH_CUDA(cudaMemcpy(cores[q - 1].data(), C, size * sizeof(double), cudaMemcpyDeviceToHost));
    }
};

template <typename T>
T* upload_as(ph_handle* h, const std::vector<double>& v) {
    std::vector<T> tmp(v.begin(), v.end());
    T* p = (T*)dev_alloc(h, std::max<size_t>(1, tmp.size()) * sizeof(T));
    if (!tmp.empty()) PH_CUDA(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

template <typename V>
V* upload_vec(ph_handle* h, const std::vector<V>& v) {
    V* p = (V*)dev_alloc(h, std::max<size_t>(1, v.size()) * sizeof(V));
    if (!v.empty()) PH_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    return p;
}

}  // namespace

// Rank kept at a TT-SVD cut from the singular values s[0] >= s[1] >= ... >= s[n-1]:
// the smallest r >= 1 whose discarded tail sum_{i>r} s_i^2 <= delta2, extended over numerically
// tied singular values (s_r - s_{r+1} <= 1e-9 s_1), then the cap, backed off below a tied group
// the cap would split.
int choose_rank_sv(const double* s, int n, double delta2, int cap) {
    std::vector<double> tail(n + 1, 0.0);
    for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[i] * s[i];
    const int lim = (cap > 0) ? std::min(n, cap) : n;
    int r = n;
    for (int k = 1; k <= n; ++k)
        if (tail[k] <= delta2) {
            r = k;
            break;
        }
    r = std::max(1, r);
    // a cut between tied singular values keeps an arbitrary part of their subspace: keep the whole
    // group, and if the cap then cuts through a group, drop that group instead
    auto tied = [&](int k) { return n > 0 && s[0] > 0 && k < n && s[k - 1] - s[k] <= kTieRel * s[0]; };
    while (tied(r)) ++r;
    if (r > lim) {
        r = lim;
        while (r > 1 && tied(r)) --r;
    }
    return r;
}

namespace {
std::atomic<long> g_alloc_budget{-1};  // successful allocations left before injected failures (< 0: off)
}  // namespace

void set_alloc_failure(long after) { g_alloc_budget.store(after < 0 ? -1 : after); }

void* dev_alloc(ph_handle* h, size_t bytes) {
    void* p = nullptr;
    long budget = g_alloc_budget.load();
    while (budget >= 0) {
        if (budget == 0) throw Error(PH_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: injected failure");
        if (g_alloc_budget.compare_exchange_weak(budget, budget - 1)) break;
    }
    // 64 bytes of slack: bulk copies round the end of a range up to 16 bytes
    cudaError_t e = cudaMalloc(&p, bytes + 64);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(PH_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                    cudaGetErrorString(e));
    }
    h->buffers.push_back({p, bytes});
    return p;
}

void free_device(ph_handle* h) {
    surrogate_free(h);  // host state of the surrogate (its device buffers are in h->buffers)
    for (auto& b : h->buffers)
        if (b.ptr) cudaFree(b.ptr);
    h->buffers.clear();
    if (h->host_flags) cudaFreeHost(h->host_flags);
    if (h->host_thetas_pinned) cudaFreeHost(h->host_thetas_pinned);
    h->host_flags = nullptr;
    h->host_thetas_pinned = nullptr;
    h->host_thetas_cap = 0;
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_thetas) {
        cudaEventSynchronize(h->ev_thetas);
        cudaEventDestroy(h->ev_thetas);
    }
    h->ev_thetas = nullptr;
    h->side = nullptr;
    h->ev_fork = h->ev_join = nullptr;
}

ph_status offline_build(ph_handle* h, const double* points, long n) {
    auto t0 = std::chrono::steady_clock::now();
    const ph_build_opts& o = h->opts;
    const int d = o.d, dt = o.dtheta, ps = o.p_s;
    Plan& plan = h->plan;
    const bool dedup = o.dedup && kernel_translation_invariant(h->kernel);
    build_plan(points, n, d, o.l_max, o.eta, dedup, plan);

    PH_CUDA(cudaSetDevice(h->device));
    // the far-field chain is the longer path of a matvec: its stream gets the highest priority so
    // its blocks are scheduled ahead of the near-field blocks that fill the remaining SM slots
    {
        int lo = 0, hi = 0;
        PH_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        PH_CUDA(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi));
    }
    PH_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    PH_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));

    h->scalar = (o.prec == PH_FP32) ? 4 : 8;
    h->PD = 1;
    for (int k = 0; k < d; ++k) h->PD *= ps;
    h->Delta = 2 * d + dt;
    int pt[kMaxDim] = {1, 1, 1};
    h->p_theta_total = 1;
    for (int k = 0; k < dt; ++k) {
        pt[k] = o.degree[k] + 1;
        h->p_theta_total *= pt[k];
    }
    const int P = h->p_theta_total;  // theta-grid points (product over the parameter dimensions)
    if (P > kMaxThetaGrid) throw Error(PH_ERR_UNSUPPORTED, "at most 1024 theta-grid points");
    if (ps < 1 || ps > kMaxPs) throw Error(PH_ERR_INVALID_ARG, "p_s must be 1..16");

    // the near field's own theta grid (near_degree, 0 = degree)
    int ptn[kMaxDim] = {1, 1, 1};
    h->p_theta_near_total = 1;
    for (int k = 0; k < dt; ++k) {
        ptn[k] = (o.near_degree[k] > 0 ? o.near_degree[k] : o.degree[k]) + 1;
        h->p_theta_near_total *= ptn[k];
    }
    const int Pn = h->p_theta_near_total;
    if (Pn > kMaxThetaGrid) throw Error(PH_ERR_UNSUPPORTED, "at most 1024 near-field theta-grid points");

    // theta nodes and barycentric weights (3 x 32 per grid: the far-field grid, then the near-field grid)
    constexpr int kGrid = kMaxDim * kMaxPTheta;
    h->theta_nodes.assign(2 * kGrid, 0.0);
    h->theta_bw.assign(2 * kGrid, 0.0);
    for (int k = 0; k < dt; ++k) {
        cheb_nodes(o.theta_lo[k], o.theta_hi[k], pt[k], &h->theta_nodes[k * kMaxPTheta]);
        bary_weights(&h->theta_nodes[k * kMaxPTheta], pt[k], &h->theta_bw[k * kMaxPTheta]);
        cheb_nodes(o.theta_lo[k], o.theta_hi[k], ptn[k], &h->theta_nodes[kGrid + k * kMaxPTheta]);
        bary_weights(&h->theta_nodes[kGrid + k * kMaxPTheta], ptn[k], &h->theta_bw[kGrid + k * kMaxPTheta]);
    }
    auto grid_points = [&](const int* p, int count, const double* nodes) {
        std::vector<double> g((size_t)count * dt);  // grid points, k_1 fastest
        for (int idx = 0; idx < count; ++idx) {
            int rest = idx;
            for (int k = 0; k < dt; ++k) {
                g[(size_t)idx * dt + k] = nodes[k * kMaxPTheta + rest % p[k]];
                rest /= p[k];
            }
        }
        return g;
    };
    const std::vector<double> gridn = grid_points(ptn, Pn, &h->theta_nodes[kGrid]);

    // points in cluster order
    std::vector<double> pts(n * d);
    for (long i = 0; i < n; ++i)
        for (int k = 0; k < d; ++k) pts[i * d + k] = points[(long)plan.perm[i] * d + k];
    double* d_pts = upload_vec(h, pts);
    double* d_gridn = upload_vec(h, gridn);

    // ------------------------------------------------------------------ near field
    // Compressed blocks: all near blocks, or with mirror sharing those (s, t) with s <= t; a
    // mirrored block (t, s) takes the stored block's rank and offsets (its cores are read
    // transposed).  Below, nn counts the compressed blocks and q indexes them (block bl[q]).
    const int nnear = (int)plan.near_s.size();
    near_mirror_map(h);
    std::vector<int> bl;
    for (int b = 0; b < nnear; ++b)
        if (h->nb_src[b] == b) bl.push_back(b);
    const int nn = (int)bl.size();
    std::vector<int> sb(nn), sn(nn), tb(nn), tn(nn);
    for (int q = 0; q < nn; ++q) {
        const Node& s = plan.nodes[plan.near_s[bl[q]]];
        const Node& t = plan.nodes[plan.near_t[bl[q]]];
        sb[q] = s.begin; sn[q] = s.size(); tb[q] = t.begin; tn[q] = t.size();
    }
    NearBuild nbld{(int)h->kernel, d, Pn, dt, d_pts, upload_vec(h, sb), upload_vec(h, sn), upload_vec(h, tb),
                   upload_vec(h, tn), d_gridn};
    h->nb_rank.assign(nnear, 0);
    h->nb_off.assign(nnear, 0);
    h->nb_toff.assign(nnear, 0);
    h->nb_woff.assign(nnear + 1, 0);
    std::vector<double> near_theta;
    if (nn > 0) {
        const double ntol = (o.near_tol >= 0) ? o.near_tol : o.tol;
        // per block, from the first TT cut of A_b (rows x Pn): the rank r_{b,1}, the theta matrix W
        // (near_theta_matrix) and V_r (Pn x r, packed for the projection G_{b,1} = A_b V_r)
        std::vector<double> vr_pack;
        std::vector<long long> voff(nn, 0);
        long long off = 0, toff = 0;
        auto finish_block = [&](int q, const double* s, const double* V) {  // s descending, V Pn x Pn
            double fro2 = 0.0;
            for (int k = 0; k < Pn; ++k) fro2 += s[k] * s[k];
            const double delta2 = ntol * ntol * fro2 / dt;
            const int r = choose_rank_sv(s, Pn, delta2, kMaxNearRank);
            const int b = bl[q];
            h->nb_rank[b] = r;
            h->nb_off[b] = off;
            h->nb_toff[b] = toff;
            off += (long long)sn[q] * tn[q] * r;
            toff += (long long)r * Pn;
            const std::vector<double> W = near_theta_matrix(s, V, Pn, r, ptn, dt, delta2);
            near_theta.insert(near_theta.end(), W.begin(), W.end());
            voff[q] = (long long)vr_pack.size();
            vr_pack.insert(vr_pack.end(), V, V + (size_t)Pn * r);
        };
        if (Pn <= 32) {
            // R_b of every block by TSQR, then a batched Jacobi SVD of the Pn x Pn factors
            double* d_R = (double*)dev_alloc(h, (size_t)nn * Pn * Pn * sizeof(double));
            double* d_S = (double*)dev_alloc(h, (size_t)nn * Pn * sizeof(double));
            double* d_U = (double*)dev_alloc(h, (size_t)nn * Pn * Pn * sizeof(double));
            double* d_V = (double*)dev_alloc(h, (size_t)nn * Pn * Pn * sizeof(double));
            size_t smem = ((size_t)(Pn + kChunk) * Pn + (size_t)kChunk * Pn) * sizeof(double);
            PH_CUDA(cudaFuncSetAttribute(near_tsqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            near_tsqr_kernel<<<nn, 256, smem>>>(nbld, d_R, kChunk);
            PH_LAUNCH("near_tsqr_kernel");
            struct Solver {  // released on every exit path
                cusolverDnHandle_t sol = nullptr;
                gesvdjInfo_t params = nullptr;
                ~Solver() {
                    if (params) cusolverDnDestroyGesvdjInfo(params);
                    if (sol) cusolverDnDestroy(sol);
                }
            } svd;
            PH_SOLVER(cusolverDnCreate(&svd.sol));
            PH_SOLVER(cusolverDnCreateGesvdjInfo(&svd.params));
            cusolverDnHandle_t sol = svd.sol;
            gesvdjInfo_t params = svd.params;
            PH_SOLVER(cusolverDnXgesvdjSetTolerance(params, 1e-15));
            PH_SOLVER(cusolverDnXgesvdjSetMaxSweeps(params, 100));
            PH_SOLVER(cusolverDnXgesvdjSetSortEig(params, 1));
            int lwork = 0;
            PH_SOLVER(cusolverDnDgesvdjBatched_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, Pn, Pn, d_R, Pn, d_S, d_U, Pn,
                                                          d_V, Pn, &lwork, params, nn));
            double* d_work = (double*)dev_alloc(h, (size_t)std::max(lwork, 1) * sizeof(double));
            int* d_info = (int*)dev_alloc(h, (size_t)nn * sizeof(int));
            PH_SOLVER(cusolverDnDgesvdjBatched(sol, CUSOLVER_EIG_MODE_VECTOR, Pn, Pn, d_R, Pn, d_S, d_U, Pn, d_V, Pn,
                                               d_work, lwork, d_info, params, nn));
            std::vector<int> infos(nn);
            PH_CUDA(cudaMemcpy(infos.data(), d_info, nn * sizeof(int), cudaMemcpyDeviceToHost));
            for (int b = 0; b < nn; ++b)
                if (infos[b] != 0) throw Error(PH_ERR_CUDA, "batched Jacobi SVD did not converge");
            std::vector<double> sv((size_t)nn * Pn), vecs((size_t)nn * Pn * Pn);
            PH_CUDA(cudaMemcpy(sv.data(), d_S, sv.size() * sizeof(double), cudaMemcpyDeviceToHost));
            PH_CUDA(cudaMemcpy(vecs.data(), d_V, vecs.size() * sizeof(double), cudaMemcpyDeviceToHost));
            for (int b = 0; b < nn; ++b) finish_block(b, &sv[(size_t)b * Pn], &vecs[(size_t)b * Pn * Pn]);
            for (void* p : {(void*)d_R, (void*)d_S, (void*)d_U, (void*)d_V, (void*)d_work, (void*)d_info}) dev_free(h, p);
        } else if (Pn <= 128) {
            // 33..128 theta-grid points: R_b by TSQR (row chunks sized to shared memory), then a
            // one-sided Jacobi SVD of each Pn x Pn factor on the host (FP64, one thread per block at a
            // time), which keeps singular values near the truncation threshold and the kept
            // subspaces accurate to rounding (so the kept ranks are the oracle's)
            int chunk = 256;
            while (chunk > 16 && ((size_t)(Pn + chunk) * Pn + (size_t)chunk * Pn) * sizeof(double) > 200 * 1024) chunk /= 2;
            const size_t smem = ((size_t)(Pn + chunk) * Pn + (size_t)chunk * Pn) * sizeof(double);
            double* d_R = (double*)dev_alloc(h, (size_t)nn * Pn * Pn * sizeof(double));
            PH_CUDA(cudaFuncSetAttribute(near_tsqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            near_tsqr_kernel<<<nn, 256, smem>>>(nbld, d_R, chunk);
            PH_LAUNCH("near_tsqr_kernel");
            std::vector<double> Rall((size_t)nn * Pn * Pn);
            PH_CUDA(cudaMemcpy(Rall.data(), d_R, Rall.size() * sizeof(double), cudaMemcpyDeviceToHost));
            dev_free(h, d_R);
            std::vector<double> sv((size_t)nn * Pn), vecs((size_t)nn * Pn * Pn);
            const int nthr = std::max(1, std::min(64, (int)std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            std::atomic<int> next{0};
            for (int w = 0; w < nthr; ++w)
                pool.emplace_back([&]() {
                    std::vector<double> R((size_t)Pn * Pn), U, sg, Vt;
                    for (int b = next++; b < nn; b = next++) {
                        std::copy(Rall.begin() + (size_t)b * Pn * Pn, Rall.begin() + (size_t)(b + 1) * Pn * Pn, R.begin());
                        svd_small(Pn, Pn, R, U, sg, Vt);
                        for (int k = 0; k < Pn; ++k) {
                            sv[(size_t)b * Pn + k] = sg[k];
                            for (int t = 0; t < Pn; ++t) vecs[(size_t)b * Pn * Pn + t + (size_t)Pn * k] = Vt[k + (size_t)Pn * t];
                        }
                    }
                });
            for (auto& th : pool) th.join();
            for (int b = 0; b < nn; ++b) finish_block(b, &sv[(size_t)b * Pn], &vecs[(size_t)b * Pn * Pn]);
        } else {
            // more than 128 theta-grid points (the triangular factor no longer fits in shared
            // memory): the right singular vectors and singular values of A_b come from the
            // eigendecomposition of A_b^T A_b (FP64, cuSOLVER's batched symmetric eigensolver), in
            // batches of blocks whose formed A_b take about 2 GB.  Singular values carry an
            // absolute error of about eps s_1^2 / s, the kept subspace an angle of about
            // eps s_1^2 / (s_r^2 - s_{r+1}^2): adequate for FP32 handles at tolerances >= 1e-5.
            long long maxrows = 1;
            for (int b = 0; b < nn; ++b) maxrows = std::max(maxrows, (long long)sn[b] * tn[b]);
            const long long per = maxrows * Pn * (long long)sizeof(double);
            const int batch = (int)std::max(1LL, std::min((long long)nn, (2LL << 30) / per));
            double* d_A = (double*)dev_alloc(h, (size_t)batch * per);
            double* d_G = (double*)dev_alloc(h, (size_t)batch * Pn * Pn * sizeof(double));
            double* d_L = (double*)dev_alloc(h, (size_t)batch * Pn * sizeof(double));
            int* d_info = (int*)dev_alloc(h, (size_t)batch * sizeof(int));
            struct Libs {  // released on every exit path
                cublasHandle_t blas = nullptr;
                cusolverDnHandle_t sol = nullptr;
                cusolverDnParams_t prm = nullptr;
                ~Libs() {
                    if (prm) cusolverDnDestroyParams(prm);
                    if (sol) cusolverDnDestroy(sol);
                    if (blas) cublasDestroy(blas);
                }
            } lib;
            PH_BLAS(cublasCreate(&lib.blas));
            PH_SOLVER(cusolverDnCreate(&lib.sol));
            PH_SOLVER(cusolverDnCreateParams(&lib.prm));
            size_t wdev = 0, whost = 0;
            PH_SOLVER(cusolverDnXsyevBatched_bufferSize(lib.sol, lib.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                                        Pn, CUDA_R_64F, d_G, Pn, CUDA_R_64F, d_L, CUDA_R_64F, &wdev,
                                                        &whost, batch));
            void* d_work = dev_alloc(h, std::max<size_t>(wdev, 8));
            std::vector<unsigned char> h_work(std::max<size_t>(whost, 8));
            std::vector<double> lam((size_t)batch * Pn), vec((size_t)batch * Pn * Pn), s(Pn), V((size_t)Pn * Pn);
            std::vector<int> infos(batch);
            const double one = 1.0, zero = 0.0;
            for (int b0 = 0; b0 < nn; b0 += batch) {
                const int nb = std::min(batch, nn - b0);
                const long long total = (long long)nb * maxrows;
                near_form_kernel<<<(int)std::min<long long>(ceil_div(total, 256), 65535), 256>>>(nbld, b0, nb, maxrows, d_A);
                PH_LAUNCH("near_form_kernel");
                PH_BLAS(cublasDgemmStridedBatched(lib.blas, CUBLAS_OP_T, CUBLAS_OP_N, Pn, Pn, (int)maxrows, &one, d_A,
                                                  (int)maxrows, maxrows * Pn, d_A, (int)maxrows, maxrows * Pn, &zero, d_G,
                                                  Pn, (long long)Pn * Pn, nb));
                PH_SOLVER(cusolverDnXsyevBatched(lib.sol, lib.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, Pn,
                                                 CUDA_R_64F, d_G, Pn, CUDA_R_64F, d_L, CUDA_R_64F, d_work, wdev,
                                                 h_work.data(), whost, d_info, nb));
                PH_CUDA(cudaMemcpy(infos.data(), d_info, nb * sizeof(int), cudaMemcpyDeviceToHost));
                for (int i = 0; i < nb; ++i)
                    if (infos[i] != 0) throw Error(PH_ERR_CUDA, "batched symmetric eigensolver failed");
                PH_CUDA(cudaMemcpy(lam.data(), d_L, (size_t)nb * Pn * sizeof(double), cudaMemcpyDeviceToHost));
                PH_CUDA(cudaMemcpy(vec.data(), d_G, (size_t)nb * Pn * Pn * sizeof(double), cudaMemcpyDeviceToHost));
                for (int i = 0; i < nb; ++i) {
                    // eigenvalues ascending: reverse to singular values descending
                    for (int k = 0; k < Pn; ++k) {
                        const int src = Pn - 1 - k;
                        s[k] = std::sqrt(std::max(0.0, lam[(size_t)i * Pn + src]));
                        for (int t = 0; t < Pn; ++t) V[t + (size_t)Pn * k] = vec[(size_t)i * Pn * Pn + t + (size_t)Pn * src];
                    }
                    finish_block(b0 + i, s.data(), V.data());
                }
            }
            for (void* p : {(void*)d_A, (void*)d_G, (void*)d_L, (void*)d_info, d_work}) dev_free(h, p);
        }
        for (int b = 0; b < nnear; ++b) {
            const int src = h->nb_src[b];
            h->nb_rank[b] = h->nb_rank[src];
            h->nb_off[b] = h->nb_off[src];
            h->nb_toff[b] = h->nb_toff[src];
            h->nb_woff[b + 1] = h->nb_woff[b] + h->nb_rank[b];
        }
        h->near_elems = off;
        h->near_theta_elems = toff;
        h->w_elems = h->nb_woff[nnear];
        std::vector<int> qrank(nn);
        std::vector<long long> qoff(nn);
        for (int q = 0; q < nn; ++q) {
            qrank[q] = h->nb_rank[bl[q]];
            qoff[q] = h->nb_off[bl[q]];
        }
        int* d_rank = upload_vec(h, qrank);
        long long* d_off = upload_vec(h, qoff);
        double* d_vr = upload_vec(h, vr_pack);
        long long* d_voff = upload_vec(h, voff);
        h->d_near = dev_alloc(h, (size_t)off * h->scalar);
        // rows of A_b per projection chunk: shared memory chunk x Pn + Pn x r_max doubles within 96 KB
        const int rmax = *std::max_element(h->nb_rank.begin(), h->nb_rank.end());
        int chunk = 256;
        while (chunk > 16 && ((size_t)chunk * Pn + (size_t)Pn * rmax) * sizeof(double) > 160 * 1024) chunk /= 2;
        size_t smem2 = ((size_t)chunk * Pn + (size_t)Pn * rmax) * sizeof(double);
        if (o.prec == PH_FP32) {
            PH_CUDA(cudaFuncSetAttribute(near_project_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem2));
            near_project_kernel<float><<<nn, 256, smem2>>>(nbld, d_vr, d_voff, d_rank, d_off, (float*)h->d_near, chunk);
        } else {
            PH_CUDA(cudaFuncSetAttribute(near_project_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem2));
            near_project_kernel<double><<<nn, 256, smem2>>>(nbld, d_vr, d_voff, d_rank, d_off, (double*)h->d_near, chunk);
        }
        PH_LAUNCH("near_project_kernel");
        PH_CUDA(cudaDeviceSynchronize());
        for (void* p : {(void*)d_vr, (void*)d_voff}) dev_free(h, p);
    }
    h->d_near_theta = upload_vec(h, near_theta);

    // ------------------------------------------------------------------- far field
    const int nkeys = (int)plan.key_rep.size();
    const int Delta = h->Delta;
    h->key_ranks.assign((size_t)nkeys * (Delta + 1), 0);
    h->key_off.assign((size_t)nkeys * Delta, 0);
    h->key_hoff.assign(nkeys, 0);
    std::vector<std::vector<std::vector<double>>> key_cores(nkeys);
    std::vector<double> far_sp, far_th;
    long long hoff = 0;
    if (nkeys > 0 && o.compressor == 1) {
        // TT-cross + TT-rounding on the host (§2.1): the tensor M_k is never formed; its entries
        // are kernel values on the Chebyshev grids of the class's boxes and the theta grid
        const int kern = (int)h->kernel;
        std::atomic<int> next{0};
        std::vector<std::string> errors(nkeys);
        auto work = [&]() {
            for (int key = next++; key < nkeys; key = next++) {
                try {
                    const int fb = plan.key_rep[key];
                    const Node& s = plan.nodes[plan.far_s[fb]];
                    const Node& t = plan.nodes[plan.far_t[fb]];
                    std::vector<int> ranks;
                    far_cross(kern, d, dt, ps, pt, s.lo, s.hi, t.lo, t.hi, h->theta_nodes.data(), o.tol, o.rank_cap,
                              0x5eedull + (unsigned long long)key, key_cores[key], ranks);
                    for (int k = 0; k <= Delta; ++k) h->key_ranks[(size_t)key * (Delta + 1) + k] = ranks[k];
                } catch (const std::exception& e) {
                    errors[key] = e.what();
                }
            }
        };
        const int nthr = std::max(1, std::min(64, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int w = 0; w < nthr; ++w) pool.emplace_back(work);
        for (auto& th : pool) th.join();
        for (int key = 0; key < nkeys; ++key)
            if (!errors[key].empty()) throw Error(PH_ERR_CUDA, "TT-cross of a far-field tensor failed: " + errors[key]);
        for (int key = 0; key < nkeys; ++key) {
            const int* rk = &h->key_ranks[(size_t)key * (Delta + 1)];
            for (int k = 0; k < Delta; ++k) {
                auto& core = key_cores[key][k];
                bool theta_core = (k >= d && k < d + dt);
                auto& arena = theta_core ? far_th : far_sp;
                h->key_off[(size_t)key * Delta + k] = (long long)arena.size();
                arena.insert(arena.end(), core.begin(), core.end());
            }
            h->key_hoff[key] = hoff;
            hoff += (long long)rk[d] * rk[d + dt];
        }
    } else if (nkeys > 0) {
        TTEngine eng;
        eng.h = h;
        PH_BLAS(cublasCreate(&eng.blas));
        PH_SOLVER(cusolverDnCreate(&eng.solver));
        const long long PD = h->PD;
        const long long total = PD * P * PD;
        eng.reserve(total, (size_t)std::sqrt((double)total) + 2);
        double* d_nodes = (double*)dev_alloc(h, 2 * kMaxDim * kMaxPs * sizeof(double));
        double* d_tn = upload_vec(h, h->theta_nodes);
        int* d_pt = upload_vec(h, std::vector<int>(pt, pt + kMaxDim));
        std::vector<int> dims;
        for (int k = 0; k < d; ++k) dims.push_back(ps);
        for (int k = 0; k < dt; ++k) dims.push_back(pt[k]);
        for (int k = 0; k < d; ++k) dims.push_back(ps);
        for (int key = 0; key < nkeys; ++key) {
            const int fb = plan.key_rep[key];
            const Node& s = plan.nodes[plan.far_s[fb]];
            const Node& t = plan.nodes[plan.far_t[fb]];
            std::vector<double> nodes(2 * kMaxDim * kMaxPs, 0.0);
            for (int k = 0; k < d; ++k) {
                cheb_nodes(s.lo[k], s.hi[k], ps, &nodes[k * ps]);
                cheb_nodes(t.lo[k], t.hi[k], ps, &nodes[kMaxDim * kMaxPs + k * ps]);
            }
            PH_CUDA(cudaMemcpy(d_nodes, nodes.data(), nodes.size() * sizeof(double), cudaMemcpyHostToDevice));
            // the engine swaps its two buffers; the tensor is evaluated into the current one
            far_tensor_kernel<<<1024, 256>>>((int)h->kernel, d, dt, ps, d_pt, PD, P, d_nodes,
                                              d_nodes + kMaxDim * kMaxPs, d_tn, eng.C);
            PH_LAUNCH("far_tensor_kernel");
            std::vector<int> ranks;
            eng.run(dims, o.tol, o.rank_cap, key_cores[key], ranks);
            for (int k = 0; k <= Delta; ++k) h->key_ranks[(size_t)key * (Delta + 1) + k] = ranks[k];
            for (int k = 0; k < Delta; ++k) {
                auto& core = key_cores[key][k];
                bool theta_core = (k >= d && k < d + dt);
                auto& arena = theta_core ? far_th : far_sp;
                h->key_off[(size_t)key * Delta + k] = (long long)arena.size();
                arena.insert(arena.end(), core.begin(), core.end());
            }
            h->key_hoff[key] = hoff;
            hoff += (long long)ranks[d] * ranks[d + dt];
        }
    }
    // the online product of the d_theta > 1 parameter cores holds each factor in a 64 x 64 tile
    if (dt > 1)
        for (int key = 0; key < nkeys; ++key)
            for (int i = d; i <= d + dt; ++i)
                if (h->key_ranks[(size_t)key * (Delta + 1) + i] > 64)
                    throw Error(PH_ERR_UNSUPPORTED,
                                "with d_theta > 1 the far-field TT ranks around the parameter cores must be at most 64 "
                                "(set rank_cap <= 64)");
    // explicit factors per key (coupling mode 0, H^2): L_k^T and R_k^T, both r x PD row-major.
    // L[(i_1..i_k), s_k] = sum L[(i_1..i_{k-1}), s_{k-1}] G_k[s_{k-1}, i_k, s_k] from the left cores;
    // R[(j_1..j_d), s] from the right cores, innermost index first (App. A.4).
    std::vector<double> lr;
    h->key_lroff.assign(nkeys, 0);
    // the explicit coupling kernels tile r_d and r_{d+d_theta} by at most 64 rows; larger ranks
    // (only possible without a rank cap) use the TT chain
    for (int key = 0; key < nkeys && h->opts.coupling == 0; ++key) {
        const int* rk = &h->key_ranks[(size_t)key * (Delta + 1)];
        if (rk[d] > 64 || rk[d + dt] > 64) h->opts.coupling = 1;
    }
    if (o.fmt == PH_FMT_H2 && h->opts.coupling == 0) {
        for (int key = 0; key < nkeys; ++key) {
            const int* rk = &h->key_ranks[(size_t)key * (Delta + 1)];
            const auto& cores = key_cores[key];
            std::vector<double> L(1, 1.0);
            long long rows = 1;
            int rp = 1;
            for (int k = 0; k < d; ++k) {
                const int rn = rk[k + 1];
                const auto& G = cores[k];
                std::vector<double> Ln((size_t)rows * ps * rn, 0.0);
                for (int sn = 0; sn < rn; ++sn)
                    for (int i = 0; i < ps; ++i)
                        for (int a = 0; a < rp; ++a) {
                            const double g = G[a + (size_t)rp * (i + (size_t)ps * sn)];
                            if (g == 0.0) continue;
                            for (long long row = 0; row < rows; ++row)
                                Ln[(size_t)(row + rows * i) + (size_t)rows * ps * sn] += L[(size_t)row + rows * a] * g;
                        }
                L.swap(Ln);
                rows *= ps;
                rp = rn;
            }
            std::vector<double> Q(1, 1.0);
            rows = 1;
            int rr = 1;
            for (int k = d - 1; k >= 0; --k) {
                const int ci = d + dt + k;
                const int rl = rk[ci];
                const auto& G = cores[ci];
                std::vector<double> Qn((size_t)rows * ps * rl, 0.0);
                for (int a = 0; a < rl; ++a)
                    for (int j = 0; j < ps; ++j)
                        for (int c = 0; c < rr; ++c) {
                            const double g = G[a + (size_t)rl * (j + (size_t)ps * c)];
                            if (g == 0.0) continue;
                            for (long long rest = 0; rest < rows; ++rest)
                                Qn[(size_t)(j + ps * rest) + (size_t)rows * ps * a] += g * Q[(size_t)rest + rows * c];
                        }
                Q.swap(Qn);
                rows *= ps;
                rr = rl;
            }
            h->key_lroff[key] = (long long)lr.size();
            lr.insert(lr.end(), L.begin(), L.end());  // PD x r_d column-major == L^T row-major
            // R_k row-major, rows padded to a multiple of 4: [J * rp4 + s], zero beyond r_{d+1}
            const int rpr = rk[d + dt], rp4 = (rpr + 3) & ~3;
            const size_t base = lr.size();
            lr.resize(base + (size_t)h->PD * rp4, 0.0);
            for (int sidx = 0; sidx < rpr; ++sidx)
                for (long long J = 0; J < h->PD; ++J) lr[base + (size_t)J * rp4 + sidx] = Q[(size_t)J + (size_t)h->PD * sidx];
        }
    }
    h->lr_elems = (long long)lr.size();
    if (o.prec == PH_FP32) h->d_lr = upload_as<float>(h, lr);
    else h->d_lr = upload_as<double>(h, lr);
    // Tensor-core copy of R_k^T for phase 1 (FP32, p_s^d a multiple of 32, r' <= 64): rows s padded
    // to r'_16 = r' rounded up to 16, TF32 high and low parts (3xTF32), each 32-wide chunk of J in
    // the K-major core-matrix layout of tcgen05 operands (8 rows x 16 bytes per core matrix;
    // element (s, k) of a chunk at (k/8) r'_16 32 + (s/8) 256 + ((k%8)/4) 128 + (s%8) 16 + (k%4) 4 bytes).
    h->key_tcoff.assign(nkeys, 0);
    std::vector<float> tc;
    if (o.fmt == PH_FMT_H2 && h->opts.coupling == 0 && o.prec == PH_FP32 && h->PD % 32 == 0) {
        auto tf32_rna = [](float x) {
            // round to the nearest TF32 value (10 explicit mantissa bits), ties away from zero
            uint32_t u;
            std::memcpy(&u, &x, 4);
            if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xFFFFE000u;
            float y;
            std::memcpy(&y, &u, 4);
            return y;
        };
        for (int key = 0; key < nkeys; ++key) {
            const int* rk = &h->key_ranks[(size_t)key * (Delta + 1)];
            const int rpr = rk[d + dt], rp4 = (rpr + 3) & ~3, r16 = (rpr + 15) & ~15;
            const double* R = &lr[(size_t)h->key_lroff[key] + (size_t)rk[d] * h->PD];  // [J * rp4 + s]
            h->key_tcoff[key] = (long long)tc.size();
            const size_t chunk = (size_t)32 * r16;  // floats per chunk and part
            tc.resize(tc.size() + 2 * chunk * (h->PD / 32), 0.0f);
            float* base = &tc[(size_t)h->key_tcoff[key]];
            for (int c = 0; c < h->PD / 32; ++c)
                for (int sidx = 0; sidx < rpr; ++sidx)
                    for (int k = 0; k < 32; ++k) {
                        const float x = (float)R[(size_t)(32 * c + k) * rp4 + sidx];
                        const float hi = tf32_rna(x), lo = tf32_rna(x - hi);
                        const size_t off = ((size_t)(k / 8) * r16 * 32 + (sidx / 8) * 256 + ((k % 8) / 4) * 128 +
                                            (sidx % 8) * 16 + (k % 4) * 4) / 4;
                        base[(size_t)c * 2 * chunk + off] = hi;
                        base[(size_t)c * 2 * chunk + chunk + off] = lo;
                    }
        }
    }
    h->tc_elems = (long long)tc.size();
    h->d_tc = upload_vec(h, tc);
    h->far_elems = (long long)far_sp.size();
    h->far_theta_elems = (long long)far_th.size();
    h->H_elems = hoff;
    if (o.prec == PH_FP32) h->d_far = upload_as<float>(h, far_sp);
    else h->d_far = upload_as<double>(h, far_sp);
    h->d_far_theta = upload_vec(h, far_th);
    h->d_H = dev_alloc(h, std::max<long long>(1, hoff) * h->scalar);
    h->d_w = dev_alloc(h, std::max<long long>(1, h->w_elems) * h->scalar);

    // ---------------------------------------------------- leaf bases and transfers
    // U[(row * d + k) * p_s + j] = ell_j^{(B_leaf, k)}(x_row,k)   (§3.3)
    std::vector<double> U((size_t)n * d * ps);
    for (int leaf : plan.leaves) {
        const Node& c = plan.nodes[leaf];
        double nodes[kMaxPs], w[kMaxPs];
        for (int k = 0; k < d; ++k) {
            cheb_nodes(c.lo[k], c.hi[k], ps, nodes);
            bary_weights(nodes, ps, w);
            for (int row = c.begin; row < c.end; ++row)
                lagrange_bary(nodes, w, ps, pts[(size_t)row * d + k], &U[((size_t)row * d + k) * ps]);
        }
    }
    // E_lo / E_hi: [j * p_s + i] = ell_i^{parent}(eta_j^{child}) for the low / high half (§3.6.1)
    h->E64.assign(2 * ps * ps, 0.0);
    {
        double ref[kMaxPs], w[kMaxPs], half[kMaxPs];
        cheb_nodes(-1.0, 1.0, ps, ref);
        bary_weights(ref, ps, w);
        for (int hi = 0; hi < 2; ++hi) {
            cheb_nodes(hi ? 0.0 : -1.0, hi ? 1.0 : 0.0, ps, half);
            for (int j = 0; j < ps; ++j) lagrange_bary(ref, w, ps, half[j], &h->E64[(size_t)hi * ps * ps + j * ps]);
        }
    }
    if (o.prec == PH_FP32) {
        h->d_U = upload_as<float>(h, U);
        h->d_E = upload_as<float>(h, h->E64);
    } else {
        h->d_U = upload_as<double>(h, U);
        h->d_E = upload_as<double>(h, h->E64);
    }

    // --------------------------------------------- H format: S_b and T_b (Phase 3)
    const int nf = (int)plan.far_s.size();
    h->fb_soff.assign(nf, 0);
    h->fb_toff.assign(nf, 0);
    if (o.fmt == PH_FMT_H && nf > 0) {
        std::vector<double> st;
        for (int b = 0; b < nf; ++b) {
            const int key = plan.far_key[b];
            const int* rk = &h->key_ranks[(size_t)key * (Delta + 1)];
            const auto& cores = key_cores[key];
            const Node& s = plan.nodes[plan.far_s[b]];
            const Node& t = plan.nodes[plan.far_t[b]];
            // U factors of an arbitrary (possibly inner) node, evaluated on its own box
            auto factors = [&](const Node& c, int k, std::vector<double>& out) {
                double nodes[kMaxPs], w[kMaxPs];
                cheb_nodes(c.lo[k], c.hi[k], ps, nodes);
                bary_weights(nodes, ps, w);
                out.assign((size_t)c.size() * ps, 0.0);
                for (int row = c.begin; row < c.end; ++row)
                    lagrange_bary(nodes, w, ps, pts[(size_t)row * d + k], &out[(size_t)(row - c.begin) * ps]);
            };
            // S_b <- U_{s,1} G_1^{2};  S_b <- (U_{s,i} |x S_b) G_i^{2}
            const int ns = s.size();
            std::vector<double> S((size_t)ns * 1, 1.0), Uk;
            int rprev = 1;
            for (int k = 0; k < d; ++k) {
                factors(s, k, Uk);
                const int rn = rk[k + 1];
                const auto& G = cores[k];  // (rprev, ps, rn) Fortran
                std::vector<double> Sn((size_t)ns * rn, 0.0);
                for (int x = 0; x < ns; ++x)
                    for (int c = 0; c < rn; ++c) {
                        double acc = 0.0;
                        for (int j = 0; j < ps; ++j)
                            for (int a = 0; a < rprev; ++a)
                                acc += Uk[(size_t)x * ps + j] * S[(size_t)a * ns + x] * G[a + rprev * (j + ps * c)];
                        Sn[(size_t)c * ns + x] = acc;
                    }
                S.swap(Sn);
                rprev = rn;
            }
            // T_b from the right: Q <- sum_j U_{t,k}[y, j] G_{d+dt+k}[s, j, s'] Q[y, s']
            const int ntt = t.size();
            std::vector<double> Q((size_t)ntt, 1.0);
            int rnext = 1;
            for (int k = d - 1; k >= 0; --k) {
                factors(t, k, Uk);
                const int ci = d + dt + k;
                const int rl = rk[ci];
                const auto& G = cores[ci];  // (rl, ps, rnext)
                std::vector<double> Qn((size_t)ntt * rl, 0.0);
                for (int y = 0; y < ntt; ++y)
                    for (int a = 0; a < rl; ++a) {
                        double acc = 0.0;
                        for (int j = 0; j < ps; ++j)
                            for (int c = 0; c < rnext; ++c)
                                acc += Uk[(size_t)y * ps + j] * G[a + rl * (j + ps * c)] * Q[(size_t)c * ntt + y];
                        Qn[(size_t)a * ntt + y] = acc;
                    }
                Q.swap(Qn);
                rnext = rl;
            }
            h->fb_soff[b] = (long long)st.size();
            st.insert(st.end(), S.begin(), S.end());
            h->fb_toff[b] = (long long)st.size();
            st.insert(st.end(), Q.begin(), Q.end());
        }
        h->st_elems = (long long)st.size();
        if (o.prec == PH_FP32) h->d_st = upload_as<float>(h, st);
        else h->d_st = upload_as<double>(h, st);
    }

    h->offline_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return PH_OK;
}

}  // namespace ph
