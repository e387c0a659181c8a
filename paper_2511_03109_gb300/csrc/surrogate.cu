// Learned surrogate of the far-field cores H_k(theta) (an extension: the paper lists other
// parametric approximations as future work, §7).  In the explicit H^2 coupling C_k = L_k H_k(theta) R_k^T
// (§4.2, App. A.4) the spatial factors are fixed, so a network theta -> (H_k(theta))_k can replace
// the contraction of the stored theta cores.  This file holds
//   * the training targets: the exact cores in the gauge of L_k, R_k (least-squares projection of
//     the coupling matrix W_k(theta) of §3.6.2), evaluated on the GPU from the kernel;
//   * the perceptron's forward, backward and Adam kernels and the training loop;
//   * inference into the handle's H arena, used by ph_instantiate when the network is switched on.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace ph {

struct Surrogate {
    // projection (targets): per class [Lp^T (r_d x PD) | Rp (PD x r'_4)] at the offsets of the L/R
    // arena, Lp = L (L^T L)^{-1}, Rp = R (R^T R)^{-1}; Chebyshev nodes of each class's boxes
    void* proj = nullptr;
    double* geo = nullptr;  // [key][2][d][p_s]: target box nodes, then source box nodes
    // per class, FP64 row-major: [A_L | A_R | A_L^{-1} | A_R^{-1}], A the upper Cholesky factors of
    // L^T L and R^T R; K = A_L H A_R^T is the core in orthonormal bases (|L H R^T| = |K|)
    double* bal = nullptr;
    long long* bal_off = nullptr;
    float* kbuf = nullptr;  // inference: the network's balanced cores before the change of basis
    bool proj_ready = false;
    // network
    int n_in = 0, hidden = 0;
    long long n_out = 0;
    float* params = nullptr;           // FP32 master weights [W1 b1 W2 b2 W3 b3]
    __nv_bfloat16* wbf = nullptr;      // BF16 copies of W1, W2, W3 (same offsets minus the biases)
    float* scale = nullptr;            // per output: the class's target scale s_k
    float* work = nullptr;             // inference scratch: u, h1, h2
    bool accepted = false, use = false;
};

namespace {

constexpr int kT = 256;

// ------------------------------------------------------------------------------ kernel values

// kappa(x, y; theta) of the ph_kernel enumeration, in the arithmetic of T (the formulas of the
// kernel table in ph.h).
template <typename T>
__device__ __forceinline__ T kappa_t(int kernel, const T* x, const T* y, const T* th, int d) {
    T r2 = T(0);
    for (int k = 0; k < d; ++k) {
        const T df = x[k] - y[k];
        r2 += df * df;
    }
    const T l = th[0];
    switch (kernel) {
        case PH_KERNEL_GAUSS: return exp(-r2 / (T(2) * l * l));
        case PH_KERNEL_MATERN32: {
            const T s = sqrt(T(3) * r2) / l;
            return (T(1) + s) * exp(-s);
        }
        case PH_KERNEL_MATERN52: {
            const T s = sqrt(T(5) * r2) / l;
            return (T(1) + s + s * s / T(3)) * exp(-s);
        }
        case PH_KERNEL_ANISO_GAUSS: {
            T q = T(0);
            for (int k = 0; k < d; ++k) {
                const T df = x[k] - y[k];
                q += df * df / (T(2) * th[k] * th[k]);
            }
            return exp(-q);
        }
        case PH_KERNEL_SE: return exp(-r2 / (l * l));
        case PH_KERNEL_EXPONENTIAL: return exp(-sqrt(r2) / l);
        case PH_KERNEL_MULTIQUADRIC: return sqrt(T(1) + r2 / (l * l));
        case PH_KERNEL_POLY: return T(1) + l * r2 + l * l * r2 * r2;
        case PH_KERNEL_POLY2: return T(1) + th[0] * r2 + th[1] * th[1] * r2 * r2;
        case PH_KERNEL_POLYXY: {
            T dot = T(0);
            for (int k = 0; k < d; ++k) dot += x[k] * y[k];
            return (T(1) + dot) * (T(1) + dot) * (T(1) + l);
        }
    }
    return T(0);
}

// ---------------------------------------------------------------------------- the projection

// Right half of the projection for class `key` (blockIdx.x) and theta t (blockIdx.y of a batch):
// Tm[i][a] = sum_j W(theta)[i][j] Rp[j][a], W(theta)[i][j] = kappa(eta^s_i, eta^t_j; theta) with
// little-endian multi-indices i = i_1 + p i_2 + p^2 i_3 (§3.6.2).  Rp is staged in shared memory 16
// columns at a time; thread i keeps its row's 16 sums in registers and evaluates the kernel on the fly.
template <typename T>
__global__ void __launch_bounds__(kT) project_right_kernel(DevView<T> v, const T* proj, const double* geo,
                                                           const double* thetas, int t0, T* Tm, int tstride,
                                                           int kernel) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Rs = reinterpret_cast<T*>(smem_raw);  // PD x 16
    __shared__ T gs[2][kMaxDim][kMaxPs];
    __shared__ T th[kMaxDim];
    const int key = blockIdx.x, tt = blockIdx.y;
    const int d = v.d, ps = v.p_s, PD = v.PD, dt = v.dtheta;
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    const int rd = rk[d], rp = rk[d + dt], rp4 = (rp + 3) & ~3;
    for (int e = threadIdx.x; e < 2 * d * ps; e += blockDim.x)
        gs[e / (d * ps)][(e / ps) % d][e % ps] = (T)geo[(size_t)key * 2 * kMaxDim * kMaxPs + (e / (d * ps)) * kMaxDim * kMaxPs +
                                                          ((e / ps) % d) * kMaxPs + e % ps];
    if (threadIdx.x < dt) th[threadIdx.x] = (T)thetas[(size_t)(t0 + tt) * dt + threadIdx.x];
    const T* Rp = proj + v.key_lroff[key] + (long long)rd * PD;  // PD x rp4, row-major
    T* out = Tm + ((size_t)key * tstride + tt) * (size_t)PD * 64;  // PD x rp4 (leading dimension rp4)
    for (int a0 = 0; a0 < rp4; a0 += 16) {
        const int na = min(16, rp4 - a0);
        __syncthreads();
        for (int e = threadIdx.x; e < PD * 16; e += blockDim.x) {
            const int j = e / 16, a = e % 16;
            Rs[e] = (a < na) ? Rp[(long long)j * rp4 + a0 + a] : T(0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < PD; i += blockDim.x) {
            T x[kMaxDim];
            int rest = i;
            for (int k = 0; k < d; ++k) {
                x[k] = gs[0][k][rest % ps];
                rest /= ps;
            }
            T acc[16];
#pragma unroll
            for (int a = 0; a < 16; ++a) acc[a] = T(0);
            for (int j = 0; j < PD; ++j) {
                T y[kMaxDim];
                int rj = j;
                for (int k = 0; k < d; ++k) {
                    y[k] = gs[1][k][rj % ps];
                    rj /= ps;
                }
                const T w = kappa_t<T>(kernel, x, y, th, d);
                const T* r = Rs + j * 16;
#pragma unroll
                for (int a = 0; a < 16; ++a) acc[a] += w * r[a];
            }
            for (int a = 0; a < na; ++a) out[(size_t)i * rp4 + a0 + a] = acc[a];
        }
    }
}

// Left half: H*[t][key] (r_d x r', column-major at the class's H offset) = Lp^T Tm.
template <typename T>
__global__ void __launch_bounds__(kT) project_left_kernel(DevView<T> v, const T* proj, const T* Tm, int tstride,
                                                          T* out, long long out_stride) {
    const int key = blockIdx.x, tt = blockIdx.y;
    const int d = v.d, PD = v.PD, dt = v.dtheta;
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    const int rd = rk[d], rp = rk[d + dt], rp4 = (rp + 3) & ~3;
    const T* LpT = proj + v.key_lroff[key];  // rd x PD, row-major
    const T* Tk = Tm + ((size_t)key * tstride + tt) * (size_t)PD * 64;
    T* H = out + (long long)tt * out_stride + v.key_hoff[key];
    for (int e = threadIdx.x; e < rd * rp; e += blockDim.x) {
        const int q = e % rd, a = e / rd;
        T s = T(0);
        for (int i = 0; i < PD; ++i) s += LpT[(long long)q * PD + i] * Tk[(size_t)i * rp4 + a];
        H[e] = s;
    }
}

// Upper Cholesky factor A of an SPD r x r matrix G (row-major, G = A^T A), FP64.
std::vector<double> chol_upper(int r, const std::vector<double>& G) {
    std::vector<double> A((size_t)r * r, 0.0);
    for (int i = 0; i < r; ++i) {
        double dsum = G[(size_t)i * r + i];
        for (int k = 0; k < i; ++k) dsum -= A[(size_t)k * r + i] * A[(size_t)k * r + i];
        if (!(dsum > 0.0)) throw Error(PH_ERR_UNSUPPORTED, "singular Gram matrix of a far-field factor");
        const double aii = std::sqrt(dsum);
        A[(size_t)i * r + i] = aii;
        for (int j = i + 1; j < r; ++j) {
            double v = G[(size_t)i * r + j];
            for (int k = 0; k < i; ++k) v -= A[(size_t)k * r + i] * A[(size_t)k * r + j];
            A[(size_t)i * r + j] = v / aii;
        }
    }
    return A;
}

// Inverse of an upper-triangular r x r matrix (row-major), by back substitution per column.
std::vector<double> upper_inverse(int r, const std::vector<double>& A) {
    std::vector<double> X((size_t)r * r, 0.0);
    for (int c = 0; c < r; ++c)
        for (int i = c; i >= 0; --i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) v -= A[(size_t)i * r + k] * X[(size_t)k * r + c];
            X[(size_t)i * r + c] = v / A[(size_t)i * r + i];
        }
    return X;
}

// Per (class, theta): out = M1 in M2^T on the class's r_d x r' block (column-major at its H
// offset), with (M1, M2) = (A_L, A_R) (inverse = 0: a core into orthonormal bases) or
// (A_L^{-1}, A_R^{-1}) (inverse = 1: back); `in` optionally scaled per entry first.  FP64 in
// shared memory; in == out is allowed (each CTA reads its block before it writes it).
template <typename TI, typename TO>
__global__ void __launch_bounds__(kT) class_transform_kernel(DevView<TO> v, const TI* in, const float* in_scale,
                                                             TO* out, long long stride, const double* bal,
                                                             const long long* bal_off, int inverse) {
    extern __shared__ double tsm[];
    double* X = tsm;              // rd x rp, column-major (ld 64)
    double* T1 = tsm + 64 * 64;
    const int key = blockIdx.x, t = blockIdx.y;
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    const int rd = rk[v.d], rp = rk[v.d + v.dtheta];
    const long long base = (long long)t * stride + v.key_hoff[key];
    const double* AL = bal + bal_off[key];
    const double* AR = AL + (size_t)rd * rd;
    const double* M1 = inverse ? AR + (size_t)rp * rp : AL;
    const double* M2 = inverse ? M1 + (size_t)rd * rd : AR;
    for (int e = threadIdx.x; e < rd * rp; e += blockDim.x)
        X[(e % rd) + 64 * (e / rd)] = (double)in[base + e] * (in_scale ? (double)in_scale[v.key_hoff[key] + e] : 1.0);
    __syncthreads();
    for (int e = threadIdx.x; e < rd * rp; e += blockDim.x) {
        const int q = e % rd, a = e / rd;
        double acc = 0.0;
        for (int b = 0; b < rd; ++b) acc += M1[(size_t)q * rd + b] * X[b + 64 * a];
        T1[q + 64 * a] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rd * rp; e += blockDim.x) {
        const int q = e % rd, a = e / rd;
        double acc = 0.0;
        for (int c = 0; c < rp; ++c) acc += T1[q + 64 * c] * M2[(size_t)a * rp + c];
        out[base + e] = (TO)acc;
    }
}

template <typename TI, typename TO>
void class_transform(ph_handle* h, DevView<TO>& v, const TI* in, const float* in_scale, TO* out, long long stride,
                     int n_theta, int inverse, cudaStream_t s);

Surrogate& sur_of(ph_handle* h) {
    if (!h->sur) h->sur = new Surrogate();
    return *h->sur;
}

// The projection factors (orthonormal bases of the stored factors' column spaces), the changes of
// basis between H and the balanced core K, and the class geometry (once per handle; synchronous).
void build_projection(ph_handle* h) {
    Surrogate& S = sur_of(h);
    if (S.proj_ready) return;
    const Plan& plan = h->plan;
    if (h->opts.fmt != PH_FMT_H2 || h->opts.coupling != 0 || h->lr_elems <= 0)
        throw Error(PH_ERR_UNSUPPORTED, "the far-field surrogate needs the H^2 format with the explicit coupling");
    const int d = plan.d, dt = h->opts.dtheta, D = h->Delta, PD = h->PD, ps = h->opts.p_s;
    const int nk = (int)plan.key_rep.size();
    const size_t sc = h->scalar;
    std::vector<unsigned char> raw((size_t)h->lr_elems * sc);
    PH_CUDA(cudaMemcpy(raw.data(), h->d_lr, raw.size(), cudaMemcpyDeviceToHost));
    auto at = [&](size_t i) -> double {
        return sc == 4 ? (double)reinterpret_cast<const float*>(raw.data())[i] : reinterpret_cast<const double*>(raw.data())[i];
    };
    std::vector<double> out((size_t)h->lr_elems, 0.0), bal;
    std::vector<long long> bal_off;
    for (int k = 0; k < nk; ++k) {
        const int rd = h->key_ranks[(size_t)k * (D + 1) + d], rp = h->key_ranks[(size_t)k * (D + 1) + d + dt];
        const int rp4 = (rp + 3) & ~3;
        const size_t base = (size_t)h->key_lroff[k];
        // L^T L (rd x rd) from L^T (rd x PD, row-major); R^T R (rp x rp) from R (PD x rp4)
        std::vector<double> GL((size_t)rd * rd, 0.0), GR((size_t)rp * rp, 0.0);
        for (int a = 0; a < rd; ++a)
            for (int b = 0; b < rd; ++b) {
                double s = 0;
                for (int J = 0; J < PD; ++J) s += at(base + (size_t)a * PD + J) * at(base + (size_t)b * PD + J);
                GL[(size_t)a * rd + b] = s;
            }
        const size_t rb = base + (size_t)rd * PD;
        for (int a = 0; a < rp; ++a)
            for (int b = 0; b < rp; ++b) {
                double s = 0;
                for (int J = 0; J < PD; ++J) s += at(rb + (size_t)J * rp4 + a) * at(rb + (size_t)J * rp4 + b);
                GR[(size_t)a * rp + b] = s;
            }
        // L = Q_L A_L, R = Q_R A_R (A upper Cholesky factors of the Gram matrices): the targets are
        // computed in the orthonormal bases, K* = Q_L^T W(theta) Q_R = A_L H* A_R^T, which is well
        // conditioned however unevenly the stored factors scale their columns
        const std::vector<double> AL = chol_upper(rd, GL), AR = chol_upper(rp, GR);
        const std::vector<double> ALi = upper_inverse(rd, AL), ARi = upper_inverse(rp, AR);
        bal_off.push_back((long long)bal.size());
        for (const auto* m : {&AL, &AR, &ALi, &ARi}) bal.insert(bal.end(), m->begin(), m->end());
        // Q_L^T = A_L^{-T} L^T ; Q_R = R A_R^{-1}
        for (int a = 0; a < rd; ++a)
            for (int J = 0; J < PD; ++J) {
                double s = 0;
                for (int b = 0; b <= a; ++b) s += ALi[(size_t)b * rd + a] * at(base + (size_t)b * PD + J);
                out[base + (size_t)a * PD + J] = s;
            }
        for (int J = 0; J < PD; ++J)
            for (int a = 0; a < rp; ++a) {
                double s = 0;
                for (int b = 0; b <= a; ++b) s += at(rb + (size_t)J * rp4 + b) * ARi[(size_t)b * rp + a];
                out[rb + (size_t)J * rp4 + a] = s;
            }
    }
    S.bal = (double*)dev_alloc(h, std::max<size_t>(1, bal.size()) * sizeof(double));
    if (!bal.empty()) PH_CUDA(cudaMemcpy(S.bal, bal.data(), bal.size() * sizeof(double), cudaMemcpyHostToDevice));
    S.bal_off = (long long*)dev_alloc(h, std::max<size_t>(1, bal_off.size()) * sizeof(long long));
    if (!bal_off.empty())
        PH_CUDA(cudaMemcpy(S.bal_off, bal_off.data(), bal_off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    S.proj = dev_alloc(h, std::max<size_t>(1, out.size()) * sc);
    if (sc == 4) {
        std::vector<float> f(out.begin(), out.end());
        PH_CUDA(cudaMemcpy(S.proj, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    } else {
        PH_CUDA(cudaMemcpy(S.proj, out.data(), out.size() * 8, cudaMemcpyHostToDevice));
    }
    // Chebyshev nodes of the representative block's boxes of every class (target, then source)
    std::vector<double> geo((size_t)std::max(1, nk) * 2 * kMaxDim * kMaxPs, 0.0);
    for (int k = 0; k < nk; ++k) {
        const int fb = plan.key_rep[k];
        const Node* box[2] = {&plan.nodes[plan.far_s[fb]], &plan.nodes[plan.far_t[fb]]};
        for (int side = 0; side < 2; ++side)
            for (int a = 0; a < d; ++a)
                cheb_nodes(box[side]->lo[a], box[side]->hi[a], ps,
                           &geo[(size_t)k * 2 * kMaxDim * kMaxPs + side * kMaxDim * kMaxPs + a * kMaxPs]);
    }
    S.geo = (double*)dev_alloc(h, geo.size() * sizeof(double));
    PH_CUDA(cudaMemcpy(S.geo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice));
    S.proj_ready = true;
}

// The exact cores at n_theta parameters into out (n_theta x H_elems): H*_k, or with `balanced` the
// cores K*_k = Q_L^T W Q_R in the orthonormal bases.
template <typename T>
void far_project_typed(ph_handle* h, DevView<T>& v, const double* thetas_host, int n_theta, T* out,
                       cudaStream_t stream, bool balanced = false) {
    Surrogate& S = sur_of(h);
    const int nk = v.n_keys, dt = h->opts.dtheta;
    if (nk == 0 || n_theta == 0) return;
    // thetas to the device (synchronous: the host array may go once the call returns)
    double* d_th = (double*)dev_alloc(h, (size_t)n_theta * dt * sizeof(double));
    PH_CUDA(cudaMemcpy(d_th, thetas_host, (size_t)n_theta * dt * sizeof(double), cudaMemcpyHostToDevice));
    // batches of thetas whose intermediate PD x 64 products take about 256 MB
    const size_t per = (size_t)nk * v.PD * 64 * sizeof(T);
    const int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_theta, ((size_t)256 << 20) / per));
    T* Tm = (T*)dev_alloc(h, per * nb);
    const size_t smem = (size_t)v.PD * 16 * sizeof(T);
    PH_CUDA(cudaFuncSetAttribute(project_right_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int t0 = 0; t0 < n_theta; t0 += nb) {
        const int cnt = std::min(nb, n_theta - t0);
        project_right_kernel<T><<<dim3(nk, cnt), kT, smem, stream>>>(v, (const T*)S.proj, S.geo, d_th, t0, Tm, nb,
                                                                     (int)h->kernel);
        PH_LAUNCH("project_right_kernel");
        project_left_kernel<T><<<dim3(nk, cnt), kT, 0, stream>>>(v, (const T*)S.proj, Tm, nb, out + (size_t)t0 * h->H_elems,
                                                                 (long long)h->H_elems);
        PH_LAUNCH("project_left_kernel");
    }
    if (!balanced) class_transform<T, T>(h, v, out, nullptr, out, (long long)h->H_elems, n_theta, 1, stream);
    PH_CUDA(cudaStreamSynchronize(stream));
    dev_free(h, Tm);
    dev_free(h, d_th);
}

template <typename TI, typename TO>
void class_transform(ph_handle* h, DevView<TO>& v, const TI* in, const float* in_scale, TO* out, long long stride,
                     int n_theta, int inverse, cudaStream_t s) {
    Surrogate& S = *h->sur;
    const int nk = v.n_keys;
    if (nk == 0 || n_theta == 0) return;
    const size_t smem = (size_t)2 * 64 * 64 * sizeof(double);
    PH_CUDA(cudaFuncSetAttribute(class_transform_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int t0 = 0; t0 < n_theta; t0 += 65535) {
        const int cnt = std::min(65535, n_theta - t0);
        class_transform_kernel<TI, TO><<<dim3(nk, cnt), kT, smem, s>>>(v, in + (long long)t0 * stride, in_scale,
                                                                      out + (long long)t0 * stride, stride, S.bal,
                                                                      S.bal_off, inverse);
        PH_LAUNCH("class_transform_kernel");
    }
}

// ------------------------------------------------------------------------------- the network

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// C[m][n] = beta C[m][n] + sum_k A(m, k) B(k, n) (+ bias[n]) with A(m, k) = A[m as0 + k as1],
// B(k, n) = B[k bs0 + n bs1], C row-major (ldc); FP32 accumulation.  64 x 64 tiles, 16-deep
// slices of A and B in shared memory (loaded along whichever index is contiguous), 4 x 4 outputs
// per thread.  The network's products: the weights enter as BF16, activations as FP32.  With
// gridDim.z > 1 the K range is split (kchunk per CTA) and the partial sums are added atomically
// into C, which the caller has zeroed (beta = 0): the products whose K is the network's output
// dimension would otherwise run on a few CTAs only.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kT) gemm_kernel(int M, int N, int K, const TA* __restrict__ A, long long as0,
                                                  long long as1, const TB* __restrict__ B, long long bs0,
                                                  long long bs1, float* __restrict__ C, long long ldc, float beta,
                                                  const float* __restrict__ bias, int kchunk) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int kb0 = blockIdx.z * kchunk, ke = min(K, kb0 + kchunk);
    float acc[4][4] = {};
    const bool a_k_fast = (as1 == 1), b_k_fast = (bs0 == 1);
    for (int k0 = kb0; k0 < ke; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += kT) {
            int mm, kk;
            if (a_k_fast) { kk = e % 16; mm = e / 16; } else { mm = e % 64; kk = e / 64; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < ke) ? to_f(A[(long long)m * as0 + (long long)k * as1]) : 0.f;
            int nn, kb;
            if (b_k_fast) { kb = e % 16; nn = e / 16; } else { nn = e % 64; kb = e / 64; }
            const int n = n0 + nn, kq = k0 + kb;
            Bs[kb][nn] = (n < N && kq < ke) ? to_f(B[(long long)kq * bs0 + (long long)n * bs1]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty * 4 + u];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int m = m0 + ty * 4 + u;
        if (m >= M) continue;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int n = n0 + tx * 4 + w;
            if (n >= N) continue;
            float* c = C + (long long)m * ldc + n;
            if (gridDim.z > 1) {
                atomicAdd(c, acc[u][w] + ((bias && blockIdx.z == 0) ? bias[n] : 0.f));
            } else {
                const float val = acc[u][w] + (bias ? bias[n] : 0.f);
                *c = (beta != 0.f) ? beta * *c + val : val;
            }
        }
    }
}

template <typename TA, typename TB>
void gemm(cudaStream_t s, int M, int N, int K, const TA* A, long long as0, long long as1, const TB* B, long long bs0,
          long long bs1, float* C, long long ldc, float beta, const float* bias) {
    if (M <= 0 || N <= 0) return;
    const long long tiles = ceil_div(N, 64) * ceil_div(M, 64);
    int splits = 1;
    if (beta == 0.f && ldc == N && tiles < 296 && K >= 8192)
        splits = (int)std::max<long long>(1, std::min<long long>(ceil_div(K, 2048), 1184 / tiles));
    const int kchunk = (int)(ceil_div(ceil_div(K, splits), 16) * 16);
    splits = (int)ceil_div(K, kchunk);
    if (splits > 1) PH_CUDA(cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), s));
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64), (unsigned)splits);
    gemm_kernel<TA, TB><<<grid, kT, 0, s>>>(M, N, K, A, as0, as1, B, bs0, bs1, C, ldc, beta, bias, kchunk);
    PH_LAUNCH("gemm_kernel");
}

// gelu(x) = x Phi(x), Phi(x) = erfc(-x / sqrt 2) / 2 (exact GELU); gelu'(x) = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_f(float x) { return x * 0.5f * erfcf(-x * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_grad_f(float x) {
    return 0.5f * erfcf(-x * 0.70710678118654752f) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void gelu_kernel(const float* a, float* h, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        h[i] = gelu_f(a[i]);
}

// dA = dH * gelu'(A), in place in dH
__global__ void gelu_back_kernel(const float* a, float* dh, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dh[i] *= gelu_grad_f(a[i]);
}

// dY = (Y - T) / (B n_out) in place of Y (after the loss sum(Y - T)^2 / (2 B n_out) is accumulated)
__global__ void loss_kernel(float* Y, const float* T, long long n, double inv, double* loss) {
    double part = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float r = Y[i] - T[i];
        part += (double)r * r;
        Y[i] = (float)(r * inv);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __shared__ double red[kT / 32];
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kT / 32; ++w) s += red[w];
        atomicAdd(loss, 0.5 * s * inv);
    }
}

// out[n] = sum_b G[b][n] (bias gradients; G row-major rows x cols)
__global__ void colsum_kernel(const float* G, int rows, long long cols, float* out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cols; c += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < rows; ++r) s += G[(long long)r * cols + c];
        out[c] = s;
    }
}

// Adam (Kingma & Ba 2015, Alg. 1) on every parameter, FP32 moments; the BF16 copy of each weight
// (biases excluded: wmap[i] < 0) is refreshed from the updated master value.
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                            float c1, float c2, float eps, __nv_bfloat16* wbf, const long long* seg, int nseg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        // seg: [start, end, bf16 offset] of each weight matrix in the parameter vector
        for (int s = 0; s < nseg; ++s)
            if (i >= seg[3 * s] && i < seg[3 * s + 1]) wbf[seg[3 * s + 2] + (i - seg[3 * s])] = __float2bfloat16_rn(pi);
    }
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* q, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        q[i] = __float2bfloat16_rn(p[i]);
}

// U[b][k] = 2 (theta - lo) / (hi - lo) - 1 for the batch's samples idx[b] of thetas (n x dt)
__global__ void inputs_kernel(const double* thetas, const int* idx, int B, int dt, double lo0, double lo1, double lo2,
                              double hi0, double hi1, double hi2, float* U) {
    const double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * dt; e += gridDim.x * blockDim.x) {
        const int b = e / dt, k = e % dt;
        const int s = idx ? idx[b] : b;
        U[e] = (float)(2.0 * (thetas[(size_t)s * dt + k] - lo[k]) / (hi[k] - lo[k]) - 1.0);
    }
}

// rows of the scaled targets: T[b][o] = Hstar[idx[b]][o] / scale[o]
template <typename TS>
__global__ void targets_kernel(const TS* Hs, const int* idx, int B, long long n_out, const float* scale, float* T) {
    const long long total = (long long)B * n_out;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / n_out, o = e % n_out;
        T[e] = (float)Hs[(long long)idx[b] * n_out + o] / scale[o];
    }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(ceil_div(n, kT), 148 * 8)); }

// Parameter layout [W1 b1 W2 b2 W3 b3] and the BF16 layout [W1 W2 W3].
struct Layout {
    long long w1, b1, w2, b2, w3, b3, total;
    long long q1, q2, q3, qtotal;
    Layout(int n_in, int H, long long n_out) {
        w1 = 0;
        b1 = w1 + (long long)H * n_in;
        w2 = b1 + H;
        b2 = w2 + (long long)H * H;
        w3 = b2 + H;
        b3 = w3 + n_out * H;
        total = b3 + n_out;
        q1 = 0;
        q2 = (long long)H * n_in;
        q3 = q2 + (long long)H * H;
        qtotal = q3 + n_out * H;
    }
};

// Device buffers of one forward / backward pass over B samples.
struct Pass {
    float *U, *A1, *H1, *A2, *H2, *Y;
};

void forward(cudaStream_t s, const Layout& L, int n_in, int H, long long n_out, const float* P, const __nv_bfloat16* Q,
             int B, Pass& x) {
    // A1 = U W1^T + b1, H1 = gelu(A1), A2 = H1 W2^T + b2, H2 = gelu(A2), Y = H2 W3^T + b3
    gemm(s, B, H, n_in, x.U, n_in, 1, Q + L.q1, 1, n_in, x.A1, H, 0.f, P + L.b1);
    gelu_kernel<<<grid_for((long long)B * H), kT, 0, s>>>(x.A1, x.H1, (long long)B * H);
    gemm(s, B, H, H, x.H1, H, 1, Q + L.q2, 1, H, x.A2, H, 0.f, P + L.b2);
    gelu_kernel<<<grid_for((long long)B * H), kT, 0, s>>>(x.A2, x.H2, (long long)B * H);
    gemm(s, B, (int)n_out, H, x.H2, H, 1, Q + L.q3, 1, H, x.Y, n_out, 0.f, P + L.b3);
    PH_LAUNCH("mlp forward");
}

// Gradients into G (layout of the parameters) from dY (in x.Y); x.A1 / x.A2 hold the
// pre-activations, dH1 / dH2 scratch B x H each.
void backward(cudaStream_t s, const Layout& L, int n_in, int H, long long n_out, const __nv_bfloat16* Q, int B,
              Pass& x, float* dH1, float* dH2, float* G) {
    // dW3 = dY^T H2 (n_out x H), db3 = sum_b dY, dH2 = dY W3
    gemm(s, (int)n_out, H, B, x.Y, 1, n_out, x.H2, H, 1, G + L.w3, H, 0.f, nullptr);
    colsum_kernel<<<grid_for(n_out), kT, 0, s>>>(x.Y, B, n_out, G + L.b3);
    gemm(s, B, H, (int)n_out, x.Y, n_out, 1, Q + L.q3, H, 1, dH2, H, 0.f, nullptr);
    gelu_back_kernel<<<grid_for((long long)B * H), kT, 0, s>>>(x.A2, dH2, (long long)B * H);
    // dW2 = dA2^T H1, db2, dH1 = dA2 W2
    gemm(s, H, H, B, dH2, 1, H, x.H1, H, 1, G + L.w2, H, 0.f, nullptr);
    colsum_kernel<<<grid_for(H), kT, 0, s>>>(dH2, B, H, G + L.b2);
    gemm(s, B, H, H, dH2, H, 1, Q + L.q2, H, 1, dH1, H, 0.f, nullptr);
    gelu_back_kernel<<<grid_for((long long)B * H), kT, 0, s>>>(x.A1, dH1, (long long)B * H);
    // dW1 = dA1^T U, db1
    gemm(s, H, n_in, B, dH1, 1, H, x.U, n_in, 1, G + L.w1, n_in, 0.f, nullptr);
    colsum_kernel<<<grid_for(H), kT, 0, s>>>(dH1, B, H, G + L.b1);
    PH_LAUNCH("mlp backward");
}

}  // namespace

namespace {

// One theta through the hidden layers (one CTA, hidden <= 1024): h1 = gelu(W1 u + b1),
// h2 = gelu(W2 h1 + b2) into work[0 .. hidden).
__global__ void infer_hidden_kernel(const float* P, const __nv_bfloat16* Q, long long b1, long long q2, long long b2,
                                    int n_in, int H, double th0, double th1, double th2, double lo0, double lo1,
                                    double lo2, double hi0, double hi1, double hi2, float* work) {
    extern __shared__ float h1[];
    const double th[3] = {th0, th1, th2}, lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    for (int o = threadIdx.x; o < H; o += blockDim.x) {
        float a = P[b1 + o];
        for (int k = 0; k < n_in; ++k)
            a = fmaf(__bfloat162float(Q[(long long)o * n_in + k]), (float)(2.0 * (th[k] - lo[k]) / (hi[k] - lo[k]) - 1.0), a);
        h1[o] = gelu_f(a);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < H; o += blockDim.x) {
        float a = P[b2 + o];
        const __nv_bfloat16* w = Q + q2 + (long long)o * H;
        for (int k = 0; k < H; ++k) a = fmaf(__bfloat162float(w[k]), h1[k], a);
        work[o] = gelu_f(a);
    }
}

// Output layer into the H arena: H[o] = scale[o] (W3[o] . h2 + b3[o]); one warp per output row,
// each lane reading 8 consecutive BF16 weights (16 bytes) per step: a streaming read of W3.
template <typename T>
__global__ void __launch_bounds__(kT) infer_out_kernel(const float* P, const __nv_bfloat16* Q, long long b3,
                                                       long long q3, int H, long long n_out, const float* work,
                                                       const float* scale, T* out) {
    extern __shared__ float h2[];
    for (int k = threadIdx.x; k < H; k += blockDim.x) h2[k] = work[k];
    __syncthreads();
    const int lane = threadIdx.x % 32;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long o = blockIdx.x * (long long)(blockDim.x / 32) + threadIdx.x / 32; o < n_out; o += warps) {
        const __nv_bfloat16* w = Q + q3 + o * H;
        float s = 0.f;
        for (int k0 = 8 * lane; k0 < H; k0 += 256) {
            const uint4 raw = *reinterpret_cast<const uint4*>(w + k0);
            const __nv_bfloat162* p2 = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 f = __bfloat1622float2(p2[u]);
                s = fmaf(f.x, h2[k0 + 2 * u], s);
                s = fmaf(f.y, h2[k0 + 2 * u + 1], s);
            }
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) out[o] = (T)(scale[o] * (s + P[b3 + o]));
    }
}

// Per output over n rows of targets (n x n_out, type TS): sum of squares and the mean of the
// scaled values (pass 2, with scale known).
template <typename TS>
__global__ void target_stats_kernel(const TS* Hs, int n, long long n_out, const float* scale, double* out) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n_out; o += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < n; ++t) {
            const double x = (double)Hs[(long long)t * n_out + o];
            s += scale ? x / scale[o] : x * x;
        }
        out[o] = scale ? s / n : s;
    }
}

// Per theta t: sum (A - B)^2 and sum B^2 over the n_out entries (A from the network's scaled
// outputs or the polynomial cores, B the projected ones), accumulated in FP64.
template <typename TA, typename TB>
__global__ void err_kernel(const TA* A, const float* ascale, const TB* B, long long n_out, double* out) {
    const int t = blockIdx.y;
    double num = 0.0, den = 0.0;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n_out; o += (long long)gridDim.x * blockDim.x) {
        const double a = (double)A[(long long)t * n_out + o] * (ascale ? (double)ascale[o] : 1.0);
        const double b = (double)B[(long long)t * n_out + o];
        num += (a - b) * (a - b);
        den += b * b;
    }
    for (int off = 16; off > 0; off >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
    }
    if (threadIdx.x % 32 == 0) {
        atomicAdd(out + 2 * t, num);
        atomicAdd(out + 2 * t + 1, den);
    }
}

// RAII device buffer for the standalone network check (no handle involved).
struct DevBuf {
    void* p = nullptr;
    explicit DevBuf(size_t bytes) {
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            throw Error(PH_ERR_OOM, "device allocation failed");
        }
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <typename T> T* as() { return static_cast<T*>(p); }
};

std::vector<float> init_params(const Layout& L, int n_in, int H, long long n_out, unsigned long long seed) {
    std::vector<float> p((size_t)L.total, 0.f);
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    auto fill = [&](long long off, long long count, int fan_in) {
        const double sd = 1.0 / std::sqrt((double)fan_in);
        for (long long i = 0; i < count; ++i) p[(size_t)(off + i)] = (float)(sd * nd(gen));
    };
    fill(L.w1, (long long)H * n_in, n_in);
    fill(L.w2, (long long)H * H, H);
    fill(L.w3, n_out * H, H);
    return p;
}

void weights_to_bf16(cudaStream_t s, const Layout& L, int n_in, int H, long long n_out, const float* P,
                     __nv_bfloat16* Q) {
    to_bf16_kernel<<<grid_for((long long)H * n_in), kT, 0, s>>>(P + L.w1, Q + L.q1, (long long)H * n_in);
    to_bf16_kernel<<<grid_for((long long)H * H), kT, 0, s>>>(P + L.w2, Q + L.q2, (long long)H * H);
    to_bf16_kernel<<<grid_for(n_out * H), kT, 0, s>>>(P + L.w3, Q + L.q3, n_out * H);
    PH_LAUNCH("to_bf16_kernel");
}

template <typename T>
void train_typed(ph_handle* h, DevView<T>& v, const double* th_train, int n_train, const double* th_val, int n_val,
                 const ph_surrogate_opts& o, ph_surrogate_report& rep, cudaStream_t s) {
    Surrogate& S = sur_of(h);
    const int dt = h->opts.dtheta, H = o.hidden, B = std::min(o.batch, n_train);
    const long long n_out = h->H_elems;
    const Layout L(dt, H, n_out);
    auto t0 = std::chrono::steady_clock::now();
    build_projection(h);
    // targets: the projected cores of the training and validation thetas
    T* Ht = (T*)dev_alloc(h, (size_t)n_train * n_out * sizeof(T));
    T* Hv = (T*)dev_alloc(h, (size_t)n_val * n_out * sizeof(T));
    // the network learns the cores in orthonormal bases (K = A_L H A_R^T): there the squared error
    // of a core is the squared error of its coupling matrix L H R^T
    far_project_typed<T>(h, v, th_train, n_train, Ht, s, true);
    far_project_typed<T>(h, v, th_val, n_val, Hv, s, true);
    auto t1 = std::chrono::steady_clock::now();
    rep.targets_seconds = std::chrono::duration<double>(t1 - t0).count();
    // class scales s_k (RMS of the class's training targets) and the initial output bias (mean)
    double* d_stats = (double*)dev_alloc(h, (size_t)n_out * sizeof(double));
    target_stats_kernel<T><<<grid_for(n_out), kT, 0, s>>>(Ht, n_train, n_out, nullptr, d_stats);
    std::vector<double> ss((size_t)n_out);
    PH_CUDA(cudaMemcpyAsync(ss.data(), d_stats, ss.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    std::vector<float> scale((size_t)n_out, 1.f);
    const int nk = (int)h->plan.key_rep.size();
    for (int k = 0; k < nk; ++k) {
        const int* rk = &h->key_ranks[(size_t)k * (h->Delta + 1)];
        const long long a = h->key_hoff[k], cnt = (long long)rk[h->plan.d] * rk[h->plan.d + dt];
        double sum = 0;
        for (long long e = 0; e < cnt; ++e) sum += ss[(size_t)(a + e)];
        const double rms = std::sqrt(sum / std::max(1.0, (double)cnt * n_train));
        for (long long e = 0; e < cnt; ++e) scale[(size_t)(a + e)] = rms > 0 ? (float)rms : 1.f;
    }
    if (!S.scale) S.scale = (float*)dev_alloc(h, (size_t)n_out * sizeof(float));
    PH_CUDA(cudaMemcpy(S.scale, scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice));
    target_stats_kernel<T><<<grid_for(n_out), kT, 0, s>>>(Ht, n_train, n_out, S.scale, d_stats);
    std::vector<double> mean((size_t)n_out);
    PH_CUDA(cudaMemcpyAsync(mean.data(), d_stats, mean.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    dev_free(h, d_stats);
    // the network
    if (S.params) dev_free(h, S.params);
    if (S.wbf) dev_free(h, S.wbf);
    if (S.work) dev_free(h, S.work);
    S.params = nullptr;
    S.wbf = nullptr;
    S.work = nullptr;
    S.n_in = dt;
    S.hidden = H;
    S.n_out = n_out;
    S.accepted = S.use = false;
    std::vector<float> p0 = init_params(L, dt, H, n_out, o.seed);
    for (long long e = 0; e < n_out; ++e) p0[(size_t)(L.b3 + e)] = (float)mean[(size_t)e];
    S.params = (float*)dev_alloc(h, (size_t)L.total * sizeof(float));
    S.wbf = (__nv_bfloat16*)dev_alloc(h, (size_t)L.qtotal * sizeof(__nv_bfloat16));
    S.work = (float*)dev_alloc(h, (size_t)std::max(H, 32) * sizeof(float));
    if (S.kbuf) dev_free(h, S.kbuf);
    S.kbuf = (float*)dev_alloc(h, (size_t)std::max<long long>(1, n_out) * sizeof(float));
    PH_CUDA(cudaMemcpy(S.params, p0.data(), p0.size() * sizeof(float), cudaMemcpyHostToDevice));
    weights_to_bf16(s, L, dt, H, n_out, S.params, S.wbf);
    float* G = (float*)dev_alloc(h, (size_t)L.total * sizeof(float));
    float* Mm = (float*)dev_alloc(h, (size_t)L.total * sizeof(float));
    float* Vm = (float*)dev_alloc(h, (size_t)L.total * sizeof(float));
    PH_CUDA(cudaMemsetAsync(Mm, 0, (size_t)L.total * sizeof(float), s));
    PH_CUDA(cudaMemsetAsync(Vm, 0, (size_t)L.total * sizeof(float), s));
    // activations for batches of up to max(B, 256) rows (validation reuses them)
    const int BR = std::max(B, std::min(256, std::max(1, n_val)));
    Pass x;
    x.U = (float*)dev_alloc(h, (size_t)BR * dt * sizeof(float));
    x.A1 = (float*)dev_alloc(h, (size_t)BR * H * sizeof(float));
    x.H1 = (float*)dev_alloc(h, (size_t)BR * H * sizeof(float));
    x.A2 = (float*)dev_alloc(h, (size_t)BR * H * sizeof(float));
    x.H2 = (float*)dev_alloc(h, (size_t)BR * H * sizeof(float));
    x.Y = (float*)dev_alloc(h, (size_t)BR * n_out * sizeof(float));
    float* Tb = (float*)dev_alloc(h, (size_t)B * n_out * sizeof(float));
    float* dH1 = (float*)dev_alloc(h, (size_t)B * H * sizeof(float));
    float* dH2 = (float*)dev_alloc(h, (size_t)B * H * sizeof(float));
    double* d_loss = (double*)dev_alloc(h, (size_t)std::max(1, o.steps) * sizeof(double));
    PH_CUDA(cudaMemsetAsync(d_loss, 0, (size_t)std::max(1, o.steps) * sizeof(double), s));
    double* d_tht = (double*)dev_alloc(h, (size_t)n_train * dt * sizeof(double));
    PH_CUDA(cudaMemcpy(d_tht, th_train, (size_t)n_train * dt * sizeof(double), cudaMemcpyHostToDevice));
    // batch order: a fresh permutation of the training set per epoch (from the seed)
    std::vector<int> order;
    {
        std::mt19937_64 gen(o.seed ^ 0x9e3779b97f4a7c15ull);
        std::vector<int> perm(n_train);
        for (int i = 0; i < n_train; ++i) perm[i] = i;
        size_t pos = perm.size();
        for (long long k = 0; k < (long long)o.steps * B; ++k) {
            if (pos == perm.size()) {
                std::shuffle(perm.begin(), perm.end(), gen);
                pos = 0;
            }
            order.push_back(perm[pos++]);
        }
    }
    int* d_order = (int*)dev_alloc(h, std::max<size_t>(1, order.size()) * sizeof(int));
    if (!order.empty()) PH_CUDA(cudaMemcpy(d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
    const long long segs[9] = {L.w1, L.b1, L.q1, L.w2, L.b2, L.q2, L.w3, L.b3, L.q3};
    long long* d_seg = (long long*)dev_alloc(h, sizeof(segs));
    PH_CUDA(cudaMemcpy(d_seg, segs, sizeof(segs), cudaMemcpyHostToDevice));
    const double* lo = h->opts.theta_lo;
    const double* hi = h->opts.theta_hi;
    const double lr_min = o.lr / 100.0;
    for (int step = 0; step < o.steps; ++step) {
        const int* idx = d_order + (size_t)step * B;
        inputs_kernel<<<grid_for((long long)B * dt), kT, 0, s>>>(d_tht, idx, B, dt, lo[0], lo[1], lo[2], hi[0], hi[1],
                                                                 hi[2], x.U);
        targets_kernel<T><<<grid_for((long long)B * n_out), kT, 0, s>>>(Ht, idx, B, n_out, S.scale, Tb);
        forward(s, L, dt, H, n_out, S.params, S.wbf, B, x);
        loss_kernel<<<grid_for((long long)B * n_out), kT, 0, s>>>(x.Y, Tb, (long long)B * n_out,
                                                                  1.0 / ((double)B * n_out), d_loss + step);
        backward(s, L, dt, H, n_out, S.wbf, B, x, dH1, dH2, G);
        const double lr = lr_min + 0.5 * (o.lr - lr_min) * (1.0 + std::cos(M_PI * step / std::max(1, o.steps)));
        const int t = step + 1;
        adam_kernel<<<grid_for(L.total), kT, 0, s>>>(S.params, G, Mm, Vm, L.total, (float)lr, 0.9f, 0.999f,
                                                     (float)(1.0 - std::pow(0.9, t)), (float)(1.0 - std::pow(0.999, t)),
                                                     1e-8f, S.wbf, d_seg, 3);
        PH_LAUNCH("mlp training step");
    }
    std::vector<double> losses((size_t)std::max(1, o.steps));
    PH_CUDA(cudaMemcpyAsync(losses.data(), d_loss, losses.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    rep.loss_first = o.steps > 0 ? losses.front() : 0.0;
    rep.loss_last = o.steps > 0 ? losses.back() : 0.0;
    auto t2 = std::chrono::steady_clock::now();
    rep.train_seconds = std::chrono::duration<double>(t2 - t1).count();
    // validation: the network's cores and the polynomial path's against the projected ones
    float* Yv = (float*)dev_alloc(h, (size_t)n_val * n_out * sizeof(float));
    T* Hp = (T*)dev_alloc(h, (size_t)n_val * n_out * sizeof(T));
    double* d_thv = (double*)dev_alloc(h, (size_t)n_val * dt * sizeof(double));
    PH_CUDA(cudaMemcpy(d_thv, th_val, (size_t)n_val * dt * sizeof(double), cudaMemcpyHostToDevice));
    for (int v0 = 0; v0 < n_val; v0 += BR) {
        const int cnt = std::min(BR, n_val - v0);
        inputs_kernel<<<grid_for((long long)cnt * dt), kT, 0, s>>>(d_thv + (size_t)v0 * dt, nullptr, cnt, dt, lo[0], lo[1],
                                                                   lo[2], hi[0], hi[1], hi[2], x.U);
        forward(s, L, dt, H, n_out, S.params, S.wbf, cnt, x);
        PH_CUDA(cudaMemcpyAsync(Yv + (size_t)v0 * n_out, x.Y, (size_t)cnt * n_out * sizeof(float),
                                cudaMemcpyDeviceToDevice, s));
    }
    for (int t = 0; t < n_val; ++t) {
        online_instantiate(h, th_val + (size_t)t * dt, s, -1);  // the polynomial path (the network is off)
        PH_CUDA(cudaMemcpyAsync(Hp + (size_t)t * n_out, h->d_H, (size_t)n_out * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    h->instantiated = false;  // the handle's cores were overwritten by the validation
    class_transform<T, T>(h, v, Hp, nullptr, Hp, n_out, n_val, 0, s);  // polynomial cores into the same bases
    double* d_err = (double*)dev_alloc(h, (size_t)4 * std::max(1, n_val) * sizeof(double));
    PH_CUDA(cudaMemsetAsync(d_err, 0, (size_t)4 * std::max(1, n_val) * sizeof(double), s));
    const dim3 eg((unsigned)std::min<long long>(ceil_div(n_out, kT), 64), (unsigned)std::max(1, n_val));
    if (n_val > 0) {
        err_kernel<float, T><<<eg, kT, 0, s>>>(Yv, S.scale, Hv, n_out, d_err);
        err_kernel<T, T><<<eg, kT, 0, s>>>(Hp, nullptr, Hv, n_out, d_err + 2 * n_val);
        PH_LAUNCH("err_kernel");
    }
    std::vector<double> err((size_t)4 * std::max(1, n_val));
    PH_CUDA(cudaMemcpyAsync(err.data(), d_err, err.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    // rms = sqrt(sum_t E_t^2 / sum_t |H*_t|^2), max = max_t E_t / sqrt(mean_t |H*_t|^2)
    double sn = 0, sp = 0, sref = 0, mn = 0, mp = 0;
    for (int t = 0; t < n_val; ++t) {
        sn += err[2 * t];
        sp += err[2 * n_val + 2 * t];
        sref += err[2 * t + 1];
        mn = std::max(mn, err[2 * t]);
        mp = std::max(mp, err[2 * n_val + 2 * t]);
    }
    sref = std::max(sref, 1e-300);
    rep.val_err_net_rms = std::sqrt(sn / sref);
    rep.val_err_poly_rms = std::sqrt(sp / sref);
    rep.val_err_net_max = std::sqrt(mn / (sref / std::max(1, n_val)));
    rep.val_err_poly_max = std::sqrt(mp / (sref / std::max(1, n_val)));
    rep.params = (long)L.total;
    rep.out_dim = (long)n_out;
    S.accepted = n_val > 0 && (o.accept_tol > 0 ? rep.val_err_net_rms <= o.accept_tol
                                                : rep.val_err_net_rms <= rep.val_err_poly_rms);
    rep.accepted = S.accepted ? 1 : 0;
    for (void* p : {(void*)Ht, (void*)Hv, (void*)G, (void*)Mm, (void*)Vm, (void*)x.U, (void*)x.A1, (void*)x.H1,
                    (void*)x.A2, (void*)x.H2, (void*)x.Y, (void*)Tb, (void*)dH1, (void*)dH2, (void*)d_loss,
                    (void*)d_tht, (void*)d_order, (void*)d_seg, (void*)Yv, (void*)Hp, (void*)d_thv, (void*)d_err})
        dev_free(h, p);
}

template <typename T>
DevView<T>& view_of(ph_handle* h);
template <>
DevView<float>& view_of<float>(ph_handle* h) { return h->vf; }
template <>
DevView<double>& view_of<double>(ph_handle* h) { return h->vd; }

template <typename T>
void infer_typed(ph_handle* h, const double* theta, cudaStream_t s) {
    Surrogate& S = *h->sur;
    const Layout L(S.n_in, S.hidden, S.n_out);
    const double* lo = h->opts.theta_lo;
    const double* hi = h->opts.theta_hi;
    double th[3] = {0, 0, 0};
    for (int k = 0; k < S.n_in; ++k) th[k] = theta[k];
    infer_hidden_kernel<<<1, kT, (size_t)S.hidden * sizeof(float), s>>>(S.params, S.wbf, L.b1, L.q2, L.b2, S.n_in,
                                                                        S.hidden, th[0], th[1], th[2], lo[0], lo[1],
                                                                        lo[2], hi[0], hi[1], hi[2], S.work);
    const int grid = (int)std::max<long long>(1, std::min<long long>(ceil_div(S.n_out, kT / 32), (long long)h->num_sms * 8));
    infer_out_kernel<float><<<grid, kT, (size_t)S.hidden * sizeof(float), s>>>(S.params, S.wbf, L.b3, L.q3, S.hidden,
                                                                              S.n_out, S.work, S.scale, S.kbuf);
    PH_LAUNCH("surrogate inference");
    DevView<T>& v = view_of<T>(h);
    class_transform<float, T>(h, v, S.kbuf, nullptr, (T*)h->d_H, S.n_out, 1, 1, s);  // K -> H
    if (h->adj_ready) transpose_H(h, s);
}

}  // namespace

bool surrogate_instantiate_far(ph_handle* h, const double* theta, cudaStream_t stream) {
    if (!h->sur || !h->sur->use || !h->sur->accepted) return false;
    ProfScope ps(h, 0, stream);
    if (h->opts.prec == PH_FP32) infer_typed<float>(h, theta, stream);
    else infer_typed<double>(h, theta, stream);
    return true;
}

void surrogate_free(ph_handle* h) {
    delete h->sur;  // device buffers belong to h->buffers
    h->sur = nullptr;
}

}  // namespace ph

// ------------------------------------------------------------------------------------ C ABI

namespace {

ph_status check_thetas(ph_handle* h, const double* th, int n) {
    for (int t = 0; t < n; ++t)
        for (int k = 0; k < h->opts.dtheta; ++k) {
            const double x = th[(size_t)t * h->opts.dtheta + k];
            if (!std::isfinite(x)) return ph::fail(h, PH_ERR_NONFINITE, "theta is not finite");
            if (x < h->opts.theta_lo[k] || x > h->opts.theta_hi[k])
                return ph::fail(h, PH_ERR_THETA_OUT_OF_BOX, "theta outside the parameter box");
        }
    return PH_OK;
}

ph_status need_explicit_h2(ph_handle* h) {
    if (h->opts.fmt != PH_FMT_H2 || h->opts.coupling != 0 || h->plan.key_rep.empty())
        return ph::fail(h, PH_ERR_UNSUPPORTED,
                        "the far-field surrogate needs the H^2 format with the explicit coupling and a far field");
    return PH_OK;
}

}  // namespace

extern "C" ph_status ph_far_project(ph_handle* h, const double* thetas, int n_theta, void* out, void* stream) {
    if (!h) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_far_project: NULL handle");
    if (!thetas || !out || n_theta < 0) return ph::fail(h, PH_ERR_INVALID_ARG, "ph_far_project: invalid argument");
    ph_status st = need_explicit_h2(h);
    if (st != PH_OK) return st;
    if ((st = check_thetas(h, thetas, n_theta)) != PH_OK) return st;
    if (ph::take_timeout(h) != PH_OK) return PH_ERR_TIMEOUT;
    return ph::guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ph::build_projection(h);
        if (h->opts.prec == PH_FP32) ph::far_project_typed<float>(h, h->vf, thetas, n_theta, (float*)out, s);
        else ph::far_project_typed<double>(h, h->vd, thetas, n_theta, (double*)out, s);
        return PH_OK;
    });
}

extern "C" ph_status ph_instantiate_cores(ph_handle* h, const double* theta, const void* cores, void* stream) {
    if (!h) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_instantiate_cores: NULL handle");
    if (!theta || !cores) return ph::fail(h, PH_ERR_INVALID_ARG, "ph_instantiate_cores: NULL argument");
    ph_status st = check_thetas(h, theta, 1);
    if (st != PH_OK) return st;
    if (ph::take_timeout(h) != PH_OK) return PH_ERR_TIMEOUT;
    return ph::guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ph::online_instantiate_near(h, theta, s);
        if (h->H_elems > 0) {
            PH_CUDA(cudaMemcpyAsync(h->d_H, cores, (size_t)h->H_elems * h->scalar, cudaMemcpyDeviceToDevice, s));
            if (h->adj_ready) ph::transpose_H(h, s);
        }
        h->instantiated = true;
        return PH_OK;
    });
}

extern "C" ph_status ph_surrogate_train(ph_handle* h, const double* thetas_train, int n_train,
                                        const double* thetas_val, int n_val, const ph_surrogate_opts* opts,
                                        ph_surrogate_report* rep, void* stream) {
    if (!h) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_surrogate_train: NULL handle");
    if (!thetas_train || n_train < 1 || !thetas_val || n_val < 1)
        return ph::fail(h, PH_ERR_INVALID_ARG, "ph_surrogate_train: needs training and validation thetas");
    ph_status st = need_explicit_h2(h);
    if (st != PH_OK) return st;
    if ((st = check_thetas(h, thetas_train, n_train)) != PH_OK) return st;
    if ((st = check_thetas(h, thetas_val, n_val)) != PH_OK) return st;
    ph_surrogate_opts o{};
    if (opts) o = *opts;
    if (o.hidden == 0) o.hidden = 256;
    if (o.steps == 0) o.steps = 2000;
    if (o.batch == 0) o.batch = 256;
    if (o.lr == 0) o.lr = 1e-3;
    if (o.hidden < 8 || o.hidden > 1024 || o.hidden % 8 != 0 || o.steps < 0 || o.batch < 1 || !(o.lr > 0) ||
        o.accept_tol < 0)
        return ph::fail(h, PH_ERR_INVALID_ARG, "ph_surrogate_train: option out of range (hidden: 8..1024, a multiple of 8)");
    if (ph::take_timeout(h) != PH_OK) return PH_ERR_TIMEOUT;
    return ph::guarded(h, [&]() -> ph_status {
        PH_CUDA(cudaSetDevice(h->device));
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ph_surrogate_report r{};
        if (h->sur) h->sur->use = false;
        if (h->opts.prec == PH_FP32) ph::train_typed<float>(h, h->vf, thetas_train, n_train, thetas_val, n_val, o, r, s);
        else ph::train_typed<double>(h, h->vd, thetas_train, n_train, thetas_val, n_val, o, r, s);
        if (rep) *rep = r;
        return PH_OK;
    });
}

extern "C" ph_status ph_surrogate_use(ph_handle* h, int enable) {
    if (!h) return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_surrogate_use: NULL handle");
    if (!enable) {
        if (h->sur) h->sur->use = false;
        return PH_OK;
    }
    if (!h->sur || !h->sur->accepted)
        return ph::fail(h, PH_ERR_UNSUPPORTED, "no accepted surrogate network: the polynomial path stays in use");
    h->sur->use = true;
    return PH_OK;
}

extern "C" ph_status ph_mlp_check(int n_in, int hidden, int n_out, const float* params, int batch, const float* U,
                                  const float* T, float* Y, float* grads, double* loss) {
    if (n_in < 1 || n_in > 3 || hidden < 8 || hidden > 1024 || hidden % 8 != 0 || n_out < 1 || batch < 1 || !params ||
        !U || !T || !Y || !grads || !loss)
        return ph::fail(nullptr, PH_ERR_INVALID_ARG, "ph_mlp_check: invalid argument");
    return ph::guarded(nullptr, [&]() -> ph_status {
        using namespace ph;
        const Layout L(n_in, hidden, n_out);
        DevBuf P((size_t)L.total * 4), Q((size_t)L.qtotal * 2), G((size_t)L.total * 4), dU((size_t)batch * n_in * 4),
            A1((size_t)batch * hidden * 4), H1((size_t)batch * hidden * 4), A2((size_t)batch * hidden * 4),
            H2((size_t)batch * hidden * 4), dY((size_t)batch * n_out * 4), dT((size_t)batch * n_out * 4),
            dH1((size_t)batch * hidden * 4), dH2((size_t)batch * hidden * 4), dl(8);
        cudaStream_t s = nullptr;
        PH_CUDA(cudaMemcpy(P.p, params, (size_t)L.total * 4, cudaMemcpyHostToDevice));
        PH_CUDA(cudaMemcpy(dU.p, U, (size_t)batch * n_in * 4, cudaMemcpyHostToDevice));
        PH_CUDA(cudaMemcpy(dT.p, T, (size_t)batch * n_out * 4, cudaMemcpyHostToDevice));
        PH_CUDA(cudaMemset(dl.p, 0, 8));
        weights_to_bf16(s, L, n_in, hidden, n_out, P.as<float>(), Q.as<__nv_bfloat16>());
        Pass x{dU.as<float>(), A1.as<float>(), H1.as<float>(), A2.as<float>(), H2.as<float>(), dY.as<float>()};
        forward(s, L, n_in, hidden, n_out, P.as<float>(), Q.as<__nv_bfloat16>(), batch, x);
        PH_CUDA(cudaMemcpy(Y, dY.p, (size_t)batch * n_out * 4, cudaMemcpyDeviceToHost));
        loss_kernel<<<grid_for((long long)batch * n_out), kT>>>(dY.as<float>(), dT.as<float>(), (long long)batch * n_out,
                                                                1.0 / ((double)batch * n_out), dl.as<double>());
        backward(s, L, n_in, hidden, n_out, Q.as<__nv_bfloat16>(), batch, x, dH1.as<float>(), dH2.as<float>(),
                 G.as<float>());
        PH_CUDA(cudaDeviceSynchronize());
        PH_CUDA(cudaMemcpy(grads, G.p, (size_t)L.total * 4, cudaMemcpyDeviceToHost));
        PH_CUDA(cudaMemcpy(loss, dl.p, 8, cudaMemcpyDeviceToHost));
        return PH_OK;
    });
}
