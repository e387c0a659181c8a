// Online stage (Alg. "Online Stage", §4.4) and MVM (§4.5) of the parametric
// H / H^2 matrix.  Every step runs in the kernels below; the host only
// sequences launches.
//
//   ph_instantiate:  instantiate_kernel   v_i(theta_i) (App. A.4, FP64 barycentric),
//                                         w_b = G_{b,2} x_2 v (§4.3), H_k(theta) (Alg. PTTK online)
//   ph_matvec:       gather_kernel        X -> cluster order
//                    near_kernel          Y_s += reshape(G_{b,1} w_b) X_t, D_b never formed (§4.3)
//                    upsweep_leaf_kernel  xhat_s = U_s^T X_s          (Alg. FastForward)
//                    transfer_kernel      xhat_s += E_s'^T xhat_s'    (FastKron, up)
//                    coupling_kernel      yhat_s += L_b H_b R_b^T xhat_t as a TT chain (Alg. Modified H^2 MVM)
//                    transfer_kernel      yhat_s' += E_s' yhat_s      (FastKron, down)
//                    far_h_kernel         y_s += S_b (H_b (T_b^T x_t)) (H format, §4.5)
//                    combine_kernel       Y = Y_near + U_s yhat_s (Alg. FastBackward) -> original order
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "handle.h"

namespace ph {

namespace {

constexpr int kThreads = 256;

// ----------------------------------------------------------------------------- instantiate

// v_k(theta) = (w_k / (theta - eta_k)) / sum_j w_j / (theta - eta_j) with the
// barycentric weights w (Berrut & Trefethen, SIAM Review 2004, eq. 4.2); an
// exact node gives the exact unit vector.  For dimension `deriv` the derivatives
// v_k'(theta) instead (the instantiated matrix is linear in each v_i, so this gives
// dK_hat/dtheta_deriv).  One warp per parameter dimension.
// One warp: out[k] = ell_k(theta) (or ell_k'(theta) with deriv) for the p nodes / barycentric
// weights given; lanes >= p write nothing.  Every lane of the warp must call it.
__device__ void lagrange_weights_warp(const double* nodes, const double* bw, int p, double th, bool deriv,
                                      double* out) {
    const int lane = threadIdx.x % 32;
    const double x = (lane < p) ? nodes[lane] : 0.0;
    const double w = (lane < p) ? bw[lane] : 0.0;
    const double diff = th - x;
    const bool hit = (lane < p) && (diff == 0.0);
    const unsigned any = __ballot_sync(0xffffffffu, hit);
    auto warp_sum = [](double s) {
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
    };
    if (!deriv) {
        const double num = (lane < p && !hit) ? w / diff : 0.0;
        const double den = warp_sum(num);
        if (lane < p) out[lane] = any ? (hit ? 1.0 : 0.0) : num / den;
    } else if (any) {
        // theta at node k: ell_j'(x_k) = (w_j / w_k) / (x_k - x_j) for j != k, and the
        // derivatives sum to zero (the differentiation matrix of Berrut & Trefethen, §9)
        const int k = __ffs(any) - 1;
        const double xk = __shfl_sync(0xffffffffu, x, k), wk = __shfl_sync(0xffffffffu, w, k);
        const double dj = (lane < p && lane != k) ? (w / wk) / (xk - x) : 0.0;
        const double sum = warp_sum(dj);
        if (lane < p) out[lane] = (lane == k) ? -sum : dj;
    } else {
        // a_j = w_j / (theta - x_j), S = sum a_j, T = sum a_j / (theta - x_j):
        // ell_j' = (ell_j T - a_j / (theta - x_j)) / S; the nearest node's entry is taken as
        // minus the sum of the others, which avoids its cancellation
        const double a = (lane < p) ? w / diff : 0.0;
        const double S = warp_sum(a);
        const double T = warp_sum((lane < p) ? a / diff : 0.0);
        const double dj = (lane < p) ? ((a / S) * T - a / diff) / S : 0.0;
        double best = (lane < p) ? fabs(a) : -1.0;
        int kmax = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ok = __shfl_xor_sync(0xffffffffu, kmax, o);
            if (ob > best || (ob == best && ok < kmax)) {
                best = ob;
                kmax = ok;
            }
        }
        const double others = warp_sum(lane == kmax ? 0.0 : dj);
        if (lane < p) out[lane] = (lane == kmax) ? -others : dj;
    }
}

__device__ void parametric_vectors(const double* nodes, const double* bw, const int* pt, int dt,
                                   const double* theta, int deriv, double (*out)[kMaxPTheta]) {
    const int warp = threadIdx.x / 32;
    if (warp < dt)
        lagrange_weights_warp(nodes + warp * kMaxPTheta, bw + warp * kMaxPTheta, pt[warp], theta[warp],
                              warp == deriv, out[warp]);
}

// Online stage for one theta (Alg. "Online Stage", §4.4).  Near block b (CTA < near_ctas, one
// thread per block): w_b = W_b (v_1 (x) .. (x) v_dtheta), W_b the stored r_{b,1} x P theta matrix
// (for d_theta = 1 the core G_{b,2} = V_r^T itself; §4.3).  Far class k (one CTA per class):
// H_k = prod_i G_{k,d+i} x_2 v_i (Alg. PTTK online, App. A.4), for d_theta > 1 as the product of
// the d_theta matrices M_i = G_{k,d+i} x_2 v_i formed in shared memory (ranks <= 64).
template <typename T>
__global__ void instantiate_kernel(DevView<T> v, double th0, double th1, double th2, int near_ctas, int deriv) {
    __shared__ double sv[kMaxDim][kMaxPTheta];
    __shared__ double vprod[kMaxThetaGrid];
    extern __shared__ double dsm[];  // far classes with d_theta > 1: three 64 x 64 matrices
    const double th[3] = {th0, th1, th2};
    parametric_vectors(v.theta_nodes, v.theta_bw, v.p_theta, v.dtheta, th, deriv, sv);
    __syncthreads();
    __shared__ double svn[kMaxDim][kMaxPTheta];  // the near field's own grid
    if ((int)blockIdx.x < near_ctas) parametric_vectors(v.theta_nodes_near, v.theta_bw_near, v.p_theta_near, v.dtheta, th, deriv, svn);
    __syncthreads();
    const int dt = v.dtheta;
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < dt * kMaxPTheta; e += blockDim.x)
            v.v64[e] = ((e % kMaxPTheta) < v.p_theta[e / kMaxPTheta]) ? sv[e / kMaxPTheta][e % kMaxPTheta] : 0.0;
    int P = 1;
    for (int i = 0; i < dt; ++i) P *= v.p_theta_near[i];
    if ((int)blockIdx.x < near_ctas) {
        // tensor-product weights of the near grid, theta-grid index t = k_1 + p_1 (k_2 + p_2 k_3)
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
            double w = 1.0;
            int rest = t;
            for (int i = 0; i < dt; ++i) {
                w *= svn[i][rest % v.p_theta_near[i]];
                rest /= v.p_theta_near[i];
            }
            vprod[t] = w;
        }
        __syncthreads();
        const int b = blockIdx.x * blockDim.x + threadIdx.x;
        if (b < v.n_near) {
            const int r = v.nb_rank[b];
            const double* G = v.near_theta + v.nb_toff[b];
            T* w = v.w + v.nb_woff[b];
            for (int c = 0; c < r; ++c) {
                double s = 0.0;
                for (int t = 0; t < P; ++t) s += G[c + r * t] * vprod[t];
                w[c] = (T)s;
            }
        }
        return;
    }
    const int key = blockIdx.x - near_ctas;
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    T* H = v.H + v.key_hoff[key];
    if (dt == 1) {
        // H_k = G_{k,d+1} x_2 v  (r_d x r_{d+1}, column-major)
        const int P0 = v.p_theta[0];
        const int ra = rk[v.d], rb = rk[v.d + 1];
        const double* G = v.far_theta + v.key_off[(size_t)key * v.Delta + v.d];
        for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) {
            const int a = e % ra, bb = e / ra;
            double s = 0.0;
            for (int t = 0; t < P0; ++t) s += G[a + ra * (t + P0 * bb)] * sv[0][t];
            H[e] = (T)s;
            if (v.HT) v.HT[v.key_hoff[key] + bb + rb * a] = (T)s;
        }
        return;
    }
    double* Tm = dsm;             // running product, column-major, leading dimension 64
    double* Mi = dsm + 64 * 64;   // M_i
    double* Tn = dsm + 2 * 64 * 64;
    const int ra = rk[v.d];
    int rc = 0;  // columns of the running product
    for (int i = 0; i < dt; ++i) {
        const int r0 = rk[v.d + i], r1 = rk[v.d + i + 1], p = v.p_theta[i];
        const double* G = v.far_theta + v.key_off[(size_t)key * v.Delta + v.d + i];
        double* dst = (i == 0) ? Tm : Mi;
        for (int e = threadIdx.x; e < r0 * r1; e += blockDim.x) {
            const int a = e % r0, bb = e / r0;
            double s = 0.0;
            for (int t = 0; t < p; ++t) s += G[a + r0 * (t + p * bb)] * sv[i][t];
            dst[a + 64 * bb] = s;
        }
        __syncthreads();
        if (i > 0) {
            for (int e = threadIdx.x; e < ra * r1; e += blockDim.x) {
                const int a = e % ra, bb = e / ra;
                double s = 0.0;
                for (int q = 0; q < r0; ++q) s += Tm[a + 64 * q] * Mi[q + 64 * bb];
                Tn[a + 64 * bb] = s;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < ra * r1; e += blockDim.x) Tm[(e % ra) + 64 * (e / ra)] = Tn[(e % ra) + 64 * (e / ra)];
            __syncthreads();
        }
        rc = r1;
    }
    for (int e = threadIdx.x; e < ra * rc; e += blockDim.x) {
        const T hv = (T)Tm[(e % ra) + 64 * (e / ra)];
        H[e] = hv;
        if (v.HT) v.HT[v.key_hoff[key] + e / ra + rc * (e % ra)] = hv;
    }
}

// Many theta, one X: the instantiated matrix is linear in the parametric vector (§4.3 weights,
// App. A.4 H_b), so K_hat(theta) X = sum_q ell_q(theta) K_hat(eta_q) X exactly, with eta_q the
// theta nodes; likewise its derivative with ell_q'.  Yq holds the p products K_hat(eta_q) X
// (n x m each, leading dimension n).  CTA (x, y): a range of the n m entries for up to 32
// values of theta, whose weights one warp each forms in FP64 (cast to T for the sums).
template <typename T>
__global__ void __launch_bounds__(kThreads) node_combine_kernel(DevView<T> v, const T* __restrict__ Yq, int n, int m,
                                                               const double* __restrict__ thetas, int n_theta,
                                                               int deriv, T* __restrict__ Y, long long ldy,
                                                               long long stride_y) {
    constexpr int TB = 32;
    __shared__ double Wd[TB][kMaxPTheta];
    __shared__ T W[TB][kMaxPTheta];
    const int p = v.p_theta[0];
    const int t0 = blockIdx.y * TB;
    const int tc = min(TB, n_theta - t0);
    const int warp = threadIdx.x / 32;
    for (int tt = warp; tt < tc; tt += kThreads / 32)
        lagrange_weights_warp(v.theta_nodes, v.theta_bw, p, thetas[t0 + tt], deriv >= 0, Wd[tt]);
    __syncthreads();
    for (int e = threadIdx.x; e < TB * kMaxPTheta; e += blockDim.x) {
        const int tt = e / kMaxPTheta, q = e % kMaxPTheta;
        W[tt][q] = (tt < tc && q < p) ? (T)Wd[tt][q] : T(0);
    }
    __syncthreads();
    const long long nel = (long long)n * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nel;
         e += (long long)gridDim.x * blockDim.x) {
        T yq[kMaxPTheta];
#pragma unroll
        for (int q = 0; q < kMaxPTheta; ++q) yq[q] = (q < p) ? Yq[(long long)q * nel + e] : T(0);
        const long long i = e % n, c = e / n;
        for (int tt = 0; tt < tc; ++tt) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < kMaxPTheta; ++q) acc += W[tt][q] * yq[q];
            Y[(long long)(t0 + tt) * stride_y + i + c * ldy] = acc;
        }
    }
}

// ------------------------------------------------------------------------- gather / scatter

// Xc[i * S + c] = X[perm[i] + c * ldx] for c < m; zero for m <= c < S.
template <typename T>
__global__ void gather_kernel(DevView<T> v, const T* __restrict__ X, long long ldx, int m, int S,
                              int check) {
    const long long total = (long long)v.n * S;
    int bad = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / S), c = (int)(e % S);
        T x = (c < m) ? X[v.perm[i] + (long long)c * ldx] : T(0);
        if (check && !isfinite((double)x)) bad = 1;
        v.Xc[e] = x;
    }
    if (check && bad) atomicAdd(v.flags, 1);
}

// -------------------------------------------------------------------------------- near field

// One CTA per near work item (up to four consecutive near blocks (s, t) of one target leaf s).
// Thread (row i, group g) walks the columns j = g, g + G, ... of each block:
//   d_ij = sum_k w_k G_{b,1}[(j r + k) n_s + i]   (r loads, coalesced over i)
//   acc[c] += d_ij x_t[j][c]                      (x_t staged in shared memory)
// so the instantiated block D_b(theta) never exists in memory.  Groups are reduced in shared
// memory and the item's partial sum Y_s^{item} is written once; combine_kernel adds the
// partials of a leaf in a fixed order.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads, 3) near_kernel(DevView<T> v, int S, int c0, int maxleaf) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int RK = 8;                                 // ranks up to RK use the unrolled path
    T* xs = reinterpret_cast<T*>(smem_raw);              // maxleaf x MC
    T* red = xs + (size_t)maxleaf * MC;                   // kThreads x MC
    T* sw = red + (size_t)kThreads * MC;                  // kMaxNearRank
    const int item = blockIdx.x;
    const int leaf = v.item_leaf[item];
    const int snode = v.leaf_node[leaf];
    const int ns = v.node_end[snode] - v.node_begin[snode];
    const int b0 = v.item_first[item], b1 = b0 + v.item_count[item];
    T* part = v.partials + (long long)item * v.part_stride * S;
    for (int rbase = 0; rbase < ns; rbase += kThreads) {
        const int nrows = min(kThreads, ns - rbase);
        const int RP = (nrows + 31) & ~31;
        const int G = kThreads / RP;
        const int i = threadIdx.x % RP, g = threadIdx.x / RP;
        const bool active = (g < G) && (i < nrows);
        T acc[MC];
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[c] = T(0);
        for (int b = b0; b < b1; ++b) {
            const int tnode = v.nb_t[b];
            const int tb = v.node_begin[tnode];
            const int nt = v.node_end[tnode] - tb;
            const int r = v.nb_rank[b];
            __syncthreads();
            for (int e = threadIdx.x; e < nt * MC; e += blockDim.x) {
                const int j = e / MC, c = e % MC;
                xs[e] = v.Xc[(long long)(tb + j) * S + c0 + c];
            }
            if (threadIdx.x < r) sw[threadIdx.x] = v.w[v.nb_woff[b] + threadIdx.x];
            __syncthreads();
            if (!active) continue;
            const T* Gb = v.near_cores + v.nb_off[b] + (rbase + i);
            const long long cstride = (long long)r * ns;  // one column j of all r slabs
            if (r <= RK) {
                T wr[RK];
#pragma unroll
                for (int k = 0; k < RK; ++k) wr[k] = (k < r) ? sw[k] : T(0);
                int j = g;
                for (; j + 3 * G < nt; j += 4 * G) {
                    T val[4][RK];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int k = 0; k < RK; ++k)
                            val[u][k] = (k < r) ? __ldg(Gb + (j + u * G) * cstride + (long long)k * ns) : T(0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        T dij = T(0);
#pragma unroll
                        for (int k = 0; k < RK; ++k) dij += wr[k] * val[u][k];
                        const T* xj = xs + (j + u * G) * MC;
#pragma unroll
                        for (int c = 0; c < MC; ++c) acc[c] += dij * xj[c];
                    }
                }
                for (; j < nt; j += G) {
                    T dij = T(0);
#pragma unroll
                    for (int k = 0; k < RK; ++k)
                        if (k < r) dij += wr[k] * __ldg(Gb + j * cstride + (long long)k * ns);
#pragma unroll
                    for (int c = 0; c < MC; ++c) acc[c] += dij * xs[j * MC + c];
                }
            } else {
                for (int j = g; j < nt; j += G) {
                    T dij = T(0);
                    for (int k = 0; k < r; ++k) dij += sw[k] * __ldg(Gb + j * cstride + (long long)k * ns);
#pragma unroll
                    for (int c = 0; c < MC; ++c) acc[c] += dij * xs[j * MC + c];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < MC; ++c) red[threadIdx.x * MC + c] = acc[c];
        __syncthreads();
        if (g == 0 && i < nrows) {
            for (int gg = 1; gg < G; ++gg)
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[c] += red[(gg * RP + i) * MC + c];
#pragma unroll
            for (int c = 0; c < MC; ++c) part[(long long)(rbase + i) * S + c0 + c] = acc[c];
        }
    }
}

// --------------------------------------------------------------------------------- H^2 sweeps

template <typename T, int MC>
__device__ void mode_product(const T* z, T* out, const T* E, int p, int PD, int stride, bool transpose,
                             bool accumulate);

// xhat_s[I][c] = sum_{j in s} prod_k U_k[j][i_k] X[j][c]  (leaf stage of Alg. FastForward)
// Adds val into *p atomically (vector form for float x 4 on global memory).
template <typename T, int CT>
__device__ __forceinline__ void atomic_add_ct(T* p, const T (&val)[CT]) {
#pragma unroll
    for (int c = 0; c < CT; ++c) atomicAdd(p + c, val[c]);
}
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
template <>
__device__ __forceinline__ void atomic_add_ct<float, 4>(float* p, const float (&val)[4]) {
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(val[0], val[1], val[2], val[3]));
}
#endif

// Leaf stage of Alg. FastForward: xhat_s[I][c] = sum_{j in s} prod_k U_k[j][i_k] X[j][c].  When
// `push` is set the leaf also applies its transfer matrix, (E_{s,d} (x) .. (x) E_{s,1})^T xhat_s,
// and adds the result into its parent's xhat (which starts at zero), so the up-sweep needs no
// separate pass over the leaves' parents.  One CTA per leaf.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) upsweep_leaf_kernel(DevView<T> v, int S, int c0, int push_level) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int CH = 32;
    T* su = reinterpret_cast<T*>(smem_raw);               // CH x d x p_s
    T* sx = su + CH * kMaxDim * kMaxPs;                    // CH x MC
    T* sE = sx + CH * MC;                                  // 2 p^2 (padded to 4)
    const int leaf = blockIdx.x;
    const int node = v.leaf_node[leaf];
    const int row0 = v.node_begin[node], ns = v.node_end[node] - row0;
    const int ps = v.p_s, d = v.d, PD = v.PD;
    T* b0 = sE + ((2 * ps * ps + 3) & ~3);                 // PD x MC
    T* b1 = b0 + (size_t)PD * MC;                          // PD x MC
    constexpr int OPT = 4;  // outputs per thread: PD <= 4 * kThreads
    T acc[OPT][MC];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[o][c] = T(0);
    int idx[OPT][kMaxDim];
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        int I = threadIdx.x + o * kThreads;
        for (int k = 0; k < kMaxDim; ++k) {
            idx[o][k] = (k < d) ? I % ps : 0;
            I /= (k < d) ? ps : 1;
        }
    }
    for (int j0 = 0; j0 < ns; j0 += CH) {
        const int nj = min(CH, ns - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < nj * d * ps; e += blockDim.x)
            su[e] = v.U[(long long)(row0 + j0) * d * ps + e];
        for (int e = threadIdx.x; e < nj * MC; e += blockDim.x)
            sx[e] = v.Xc[(long long)(row0 + j0 + e / MC) * S + c0 + e % MC];
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
            const T* uj = su + j * d * ps;
#pragma unroll
            for (int o = 0; o < OPT; ++o) {
                if (threadIdx.x + o * kThreads < PD) {
                    T u = uj[idx[o][0]];
                    if (d > 1) u *= uj[ps + idx[o][1]];
                    if (d > 2) u *= uj[2 * ps + idx[o][2]];
#pragma unroll
                    for (int c = 0; c < MC; ++c) acc[o][c] += u * sx[j * MC + c];
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        const int I = threadIdx.x + o * kThreads;
        if (I < PD)
#pragma unroll
            for (int c = 0; c < MC; ++c) v.xhat[((long long)node * PD + I) * S + c0 + c] = acc[o][c];
    }
    const int parent = v.node_parent[node];
    if (parent < 0 || v.node_level[parent] < push_level) return;
    for (int e = threadIdx.x; e < 2 * ps * ps; e += blockDim.x) sE[e] = v.E[e];
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
        const int I = threadIdx.x + o * kThreads;
        if (I < PD)
#pragma unroll
            for (int c = 0; c < MC; ++c) b0[I * MC + c] = acc[o][c];
    }
    const int halves = v.node_halves[node];
    T* in = b0;
    T* out = b1;
    int stride = 1;
    for (int k = 0; k < d; ++k) {
        __syncthreads();
        mode_product<T, MC>(in, out, sE + ((halves >> k) & 1) * ps * ps, ps, PD, stride, true, false);
        T* t = in; in = out; out = t;
        stride *= ps;
    }
    __syncthreads();
    constexpr int CT = MC < 4 ? MC : 4;
    T* dst = v.xhat + (long long)parent * PD * S + c0;
    for (int e = threadIdx.x; e < PD * (MC / CT); e += blockDim.x) {
        const int I = e / (MC / CT), cq = e % (MC / CT);
        T val[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) val[c] = in[I * MC + cq * CT + c];
        atomic_add_ct<T, CT>(dst + (long long)I * S + cq * CT, val);
    }
}

// Loads CT consecutive values starting at p (p aligned to CT * sizeof(T) when CT is 2 or 4).
template <typename T, int CT>
__device__ __forceinline__ void load_ct(const T* p, T (&x)[CT]) {
#pragma unroll
    for (int c = 0; c < CT; ++c) x[c] = p[c];
}
template <>
__device__ __forceinline__ void load_ct<float, 4>(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
template <>
__device__ __forceinline__ void load_ct<double, 4>(const double* p, double (&x)[4]) {
    const double2 v0 = reinterpret_cast<const double2*>(p)[0];
    const double2 v1 = reinterpret_cast<const double2*>(p)[1];
    x[0] = v0.x; x[1] = v0.y; x[2] = v1.x; x[3] = v1.y;
}

// d0 += a0 b0, d1 += a1 b1 as one packed FP32 FMA (same rounding as two fmaf); FP64: two fma.
__device__ __forceinline__ void fma_pair(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), make_float2(d0, d1));
    d0 = r.x;
    d1 = r.y;
}
__device__ __forceinline__ void fma_pair(double& d0, double& d1, double a0, double a1, double b0, double b1) {
    d0 = fma(a0, b0, d0);
    d1 = fma(a1, b1, d1);
}

// One mode-k product of the tensor z (p^d x MC, little-endian) with a p x p matrix:
// out[.., a, ..] = sum_b A(a, b) z[.., b, ..] with A(a, b) = E[b p + a] (transposed, up-sweep)
// or E[a p + b] (down-sweep).  Each thread owns whole fibres along mode k: it loads the p
// inputs of a fibre once and writes its p outputs.
template <typename T, int MC>
__device__ void mode_product(const T* z, T* out, const T* E, int p, int PD, int stride, bool transpose,
                             bool accumulate) {
    const int nfib = PD / p;
    for (int e = threadIdx.x; e < nfib * MC; e += blockDim.x) {
        const int c = e % MC, f = e / MC;
        const int inner = f % stride, outer = f / stride;
        const int base = inner + stride * p * outer;
        T in[kMaxPs];
#pragma unroll
        for (int b = 0; b < kMaxPs; ++b)
            if (b < p) in[b] = z[(base + b * stride) * MC + c];
        for (int a = 0; a < p; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < kMaxPs; ++b)
                if (b < p) s += (transpose ? E[b * p + a] : E[a * p + b]) * in[b];
            T* o = out + (base + a * stride) * MC + c;
            if (accumulate) *o += s;
            else *o = s;
        }
    }
}

// Block-wide copy of n consecutive values from global to shared memory: 16-byte vectors when
// both ends allow it, several loads in flight per thread.
template <typename T>
__device__ __forceinline__ void block_copy(T* __restrict__ dst, const T* __restrict__ src, int n) {
    constexpr int EV = 16 / sizeof(T);
    if (((uintptr_t)dst % 16 == 0) && ((uintptr_t)src % 16 == 0) && n % EV == 0) {
        const int nv = n / EV;
        const int4* s4 = reinterpret_cast<const int4*>(src);
        int4* d4 = reinterpret_cast<int4*>(dst);
#pragma unroll 4
        for (int e = threadIdx.x; e < nv; e += blockDim.x) d4[e] = __ldg(s4 + e);
    } else {
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
    }
}

// Leaf stage of Alg. FastForward, register-tiled: xhat_s[I][c] = sum_{j in s} U_s[j][I] X[j][c]
// with U_s[j][I] = prod_k U_{s,k}[j][i_k] (face-splitting, §3.3) formed on the fly.  For
// p_s a multiple of 4 and p_s^d = 4 NT with NT dividing kThreads: thread (tile, group) owns
// 4 consecutive i_1 of one (i_2, .., i_d) and all MC right-hand sides, and sums the points
// j = group, group + JS, ... (JS = kThreads / NT groups, combined in shared memory at the end).
// Per point the thread reads 4 factor values and the point's MC values of X (broadcast within
// the warp) and issues 4 MC FMAs.  With `push` the leaf then applies its transfer matrix and
// adds the result into its parent's xhat, as upsweep_leaf_kernel does.  One CTA per leaf.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) upsweep_leaf_tiled_kernel(DevView<T> v, int S, int c0, int push_level) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int CH = 64;  // points staged per chunk
    const int ps = v.p_s, d = v.d, PD = v.PD;
    const int NT = PD / 4, JS = kThreads / NT;
    T* su = reinterpret_cast<T*>(smem_raw);              // CH x d x p_s
    T* sx = su + CH * d * ps;                             // CH x MC
    T* red = sx + CH * MC;                                // JS x PD x MC (slot 0 then holds the sum)
    T* b1 = red + (size_t)JS * PD * MC;                   // PD x MC
    T* sE = b1 + (size_t)PD * MC;                         // 2 p^2
    const int leaf = blockIdx.x;
    const int node = v.leaf_node[leaf];
    const int row0 = v.node_begin[node], ns = v.node_end[node] - row0;
    const int tile = threadIdx.x % NT, g = threadIdx.x / NT;
    const int q4 = tile % (ps / 4), rest = tile / (ps / 4);
    const int I0 = 4 * q4 + ps * rest;
    const int i2 = (d > 1) ? rest % ps : 0, i3 = (d > 2) ? rest / ps : 0;
    T acc[4][MC];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[e][c] = T(0);
    for (int j0 = 0; j0 < ns; j0 += CH) {
        const int nj = min(CH, ns - j0);
        __syncthreads();
        block_copy(su, v.U + (long long)(row0 + j0) * d * ps, nj * d * ps);
        if (S == MC) {
            block_copy(sx, v.Xc + (long long)(row0 + j0) * S, nj * MC);
        } else {
            for (int e = threadIdx.x; e < nj * MC; e += blockDim.x)
                sx[e] = v.Xc[(long long)(row0 + j0 + e / MC) * S + c0 + e % MC];
        }
        __syncthreads();
        for (int j = g; j < nj; j += JS) {
            const T* uj = su + j * d * ps;
            T u1[4];
            load_ct<T, 4>(uj + 4 * q4, u1);
            T ur = T(1);
            if (d > 1) ur = uj[ps + i2];
            if (d > 2) ur *= uj[2 * ps + i3];
            T x[MC];
            if constexpr (MC >= 4) {
#pragma unroll
                for (int c = 0; c < MC; c += 4) load_ct<T, 4>(sx + j * MC + c, *reinterpret_cast<T(*)[4]>(&x[c]));
            } else {
#pragma unroll
                for (int c = 0; c < MC; ++c) x[c] = sx[j * MC + c];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T u = u1[e] * ur;
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[e][c] += u * x[c];
            }
        }
    }
    // combine the JS point groups: slot g holds group g's sums, slot 0 receives the total
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int c = 0; c < MC; ++c) red[((size_t)g * PD + I0 + e) * MC + c] = acc[e][c];
    __syncthreads();
    for (int e = threadIdx.x; e < PD * MC; e += blockDim.x) {
        T s = red[e];
        for (int gg = 1; gg < JS; ++gg) s += red[(size_t)gg * PD * MC + e];
        red[e] = s;
        v.xhat[((long long)node * PD + e / MC) * S + c0 + e % MC] = s;
    }
    const int parent = v.node_parent[node];
    if (parent < 0 || v.node_level[parent] < push_level) return;
    for (int e = threadIdx.x; e < 2 * ps * ps; e += blockDim.x) sE[e] = v.E[e];
    const int halves = v.node_halves[node];
    T* in = red;
    T* out = b1;
    int stride = 1;
    for (int k = 0; k < d; ++k) {
        __syncthreads();
        mode_product<T, MC>(in, out, sE + ((halves >> k) & 1) * ps * ps, ps, PD, stride, true, false);
        T* t = in; in = out; out = t;
        stride *= ps;
    }
    __syncthreads();
    constexpr int CT = MC < 4 ? MC : 4;
    T* dst = v.xhat + (long long)parent * PD * S + c0;
    for (int e = threadIdx.x; e < PD * (MC / CT); e += blockDim.x) {
        const int I = e / (MC / CT), cq = e % (MC / CT);
        T val[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) val[c] = in[I * MC + cq * CT + c];
        atomic_add_ct<T, CT>(dst + (long long)I * S + cq * CT, val);
    }
}

// Up-sweep (up = true): xhat_s += sum over inner children s' of (E_{s',d} (x) .. (x) E_{s',1})^T xhat_s'.
// Down-sweep (up = false): yhat_s' += (E_{s',d} (x) .. (x) E_{s',1}) yhat_s for each inner child s'.
// Leaf children are handled by upsweep_leaf_kernel and combine_kernel.
// FastKron (§3.6.3) applies the Kronecker factors one mode at a time.  One CTA per node.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) transfer_kernel(DevView<T> v, const int* nodes, int S, int c0,
                                                            bool up, T* src_all, T* dst_all) {
    extern __shared__ unsigned char smem_raw[];
    const int PD = v.PD, p = v.p_s, d = v.d;
    T* sE = reinterpret_cast<T*>(smem_raw);  // 2 p^2, padded to 4
    T* b0 = sE + ((2 * p * p + 3) & ~3);
    T* b1 = b0 + (size_t)PD * MC;
    T* sacc = b1 + (size_t)PD * MC;
    for (int e = threadIdx.x; e < 2 * p * p; e += blockDim.x) sE[e] = v.E[e];
    const int node = nodes[blockIdx.x];
    const int cb = v.node_child_off[node], ce = v.node_child_off[node + 1];
    if (up) {
        // leaf children have already added their share (upsweep_leaf_kernel)
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            sacc[e] = dst_all[((long long)node * PD + e / MC) * S + c0 + e % MC];
        for (int q = cb; q < ce; ++q) {
            const int ch = v.node_children[q];
            if (v.node_leaf[ch] >= 0) continue;
            const int halves = v.node_halves[ch];
            __syncthreads();
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
                b0[e] = src_all[((long long)ch * PD + e / MC) * S + c0 + e % MC];
            T* in = b0;
            T* out = b1;
            int stride = 1;
            for (int k = 0; k < d; ++k) {
                __syncthreads();
                const bool last = (k == d - 1);
                mode_product<T, MC>(in, last ? sacc : out, sE + ((halves >> k) & 1) * p * p, p, PD, stride, true,
                                    last);
                T* t = in; in = out; out = t;
                stride *= p;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            dst_all[((long long)node * PD + e / MC) * S + c0 + e % MC] = sacc[e];
    } else {
        __syncthreads();
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            sacc[e] = src_all[((long long)node * PD + e / MC) * S + c0 + e % MC];
        for (int q = cb; q < ce; ++q) {
            const int ch = v.node_children[q];
            if (v.node_leaf[ch] >= 0) continue;  // leaves pull their share in combine_kernel
            const int halves = v.node_halves[ch];
            T* in = sacc;
            T* out = b0;
            int stride = 1;
            for (int k = 0; k < d; ++k) {
                __syncthreads();
                mode_product<T, MC>(in, out, sE + ((halves >> k) & 1) * p * p, p, PD, stride, false, false);
                in = out;
                out = (out == b0) ? b1 : b0;
                stride *= p;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
                dst_all[((long long)ch * PD + e / MC) * S + c0 + e % MC] += in[e];
        }
    }
}

// Row stride (in elements) of the chain's shared-memory buffers: MC values padded by 4 when
// MC >= 8, so that row-strided 16-byte accesses of a quarter warp fall in distinct banks.
template <int MC>
struct ChainRow {
    static constexpr int value = (MC >= 8) ? MC + 4 : MC;
};

// Stores CT consecutive values (one 16-byte store for float x 4).
template <typename T, int CT>
__device__ __forceinline__ void store_ct(T* p, const T (&x)[CT]) {
#pragma unroll
    for (int c = 0; c < CT; ++c) p[c] = x[c];
}
template <>
__device__ __forceinline__ void store_ct<float, 4>(float* p, const float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}

// Split of the contraction dimension over 1, 2, 4 or 8 adjacent lanes so that narrow steps still
// occupy the CTA; the lanes' partial sums are combined with warp shuffles.
__device__ __forceinline__ int split_for(int items, int K) {
    int s = 1;
    while (s < 8 && items * s < kThreads && K >= 16 * s) s <<= 1;
    return s;
}

template <typename T, int CT>
__device__ __forceinline__ void reduce_split(T (&acc)[4][CT], int split) {
    for (int o = 1; o < split; o <<= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[j][c] += __shfl_xor_sync(0xffffffffu, acc[j][c], o);
}

// Right-core step of the chain: out[A + a s'][c] = sum_{K < p r_in} in[(A + a K) istride + c] G[s' + r_out K]
// (istride = the shared row stride, or the workspace row stride for the first step, which
// reads xhat_t straight from global memory).  Work item = (A, quad of s', CT columns); the
// K loop is split over adjacent lanes when there are few items.
template <typename T, int MC>
__device__ void chain_rstep(const T* in, int istride, T* out, const T* __restrict__ G, int a, int K, int rout) {
    constexpr int CT = MC < 4 ? MC : 4, CQ = MC / CT, RS = ChainRow<MC>::value;
    const int SQ = (rout + 3) >> 2;
    const int items = a * SQ * CQ;
    const int split = split_for(items, K);
    const int kc = (K + split - 1) / split;
    const int total = ((items * split + 31) / 32) * 32;  // whole warps, so shuffles see every lane
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int ks = w % split, item = w / split;
        const bool live = item < items;
        const int cq = item % CQ, rest = item / CQ;
        const int A = rest % a, sq = rest / a;
        const int k0 = ks * kc, k1 = live ? min(K, k0 + kc) : k0;
        const int nso = min(4, rout - 4 * sq);
        T acc[4][CT];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[j][c] = T(0);
        const T* ip = in + (long long)A * istride + cq * CT;
        const T* gp = G + 4 * sq;
        for (int k = k0; k < k1; ++k) {
            T x[CT];
            load_ct<T, CT>(ip + (long long)a * k * istride, x);
            const T* gk = gp + (long long)rout * k;
            T g[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j] = (j < nso) ? __ldg(gk + j) : T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int c = 0; c < CT; ++c) acc[j][c] += g[j] * x[c];
        }
        if (split > 1) reduce_split<T, CT>(acc, split);
        if (live && ks == 0)
            for (int j = 0; j < nso; ++j) store_ct<T, CT>(out + (long long)(A + a * (4 * sq + j)) * RS + cq * CT, acc[j]);
    }
}

// Left-core (and H) step: out[row + rows B][c] = sum_{s < r_in} G[row + rows s] in[s + r_in B][c].
// Work item = (quad of rows, B, CT columns).
template <typename T, int MC>
__device__ void chain_lstep(const T* in, T* out, const T* __restrict__ G, int rows, int rin, int bsz) {
    constexpr int CT = MC < 4 ? MC : 4, CQ = MC / CT, RS = ChainRow<MC>::value;
    const int RQ = (rows + 3) >> 2;
    const int items = RQ * bsz * CQ;
    const int split = split_for(items, rin);
    const int kc = (rin + split - 1) / split;
    const int total = ((items * split + 31) / 32) * 32;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int ks = w % split, item = w / split;
        const bool live = item < items;
        const int cq = item % CQ, rest = item / CQ;
        const int B = rest % bsz, rq = rest / bsz;
        const int k0 = ks * kc, k1 = live ? min(rin, k0 + kc) : k0;
        const int nr = min(4, rows - 4 * rq);
        T acc[4][CT];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[j][c] = T(0);
        const T* ip = in + (long long)rin * B * RS + cq * CT;
        const T* gp = G + 4 * rq;
        for (int k = k0; k < k1; ++k) {
            T x[CT];
            load_ct<T, CT>(ip + (long long)k * RS, x);
            const T* gk = gp + (long long)rows * k;
            T g[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j] = (j < nr) ? __ldg(gk + j) : T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int c = 0; c < CT; ++c) acc[j][c] += g[j] * x[c];
        }
        if (split > 1) reduce_split<T, CT>(acc, split);
        if (live && ks == 0)
            for (int j = 0; j < nr; ++j) store_ct<T, CT>(out + (long long)(4 * rq + j + rows * B) * RS + cq * CT, acc[j]);
    }
}

// Multiplication stage of Alg. "Modified H^2-Matrix MVM": for every far block (s, t) with
// compressed class k, z = xhat_t; d right-core steps z <- reshape(z, [p^{d-i-1}, p r]) G^{1}^T
// (the first reads xhat_t from global memory); z <- H_k z; d - 1 left-core steps
// z <- G^{2} reshape(z, [r, p^i]); the last left-core step (G_1, r_0 = 1) is accumulated in
// registers.  The far blocks of a target are split over `nsplit` CTAs whose sums meet in
// yhat_s through atomic adds (yhat is cleared before the launch).
template <typename T, int MC, int NI>
__global__ void __launch_bounds__(kThreads, 3) coupling_kernel(DevView<T> v, int S, int c0, int zmax, int nsplit) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int CT = MC < 4 ? MC : 4, CQ = MC / CT, RS = ChainRow<MC>::value;
    const int PD = v.PD, p = v.p_s, d = v.d, Delta = v.Delta;
    T* z0 = reinterpret_cast<T*>(smem_raw);
    T* z1 = z0 + (size_t)zmax * RS;
    const int ti = blockIdx.x / nsplit, part = blockIdx.x % nsplit;
    const int s = v.far_targets[ti];
    const int RQ0 = (p + 3) >> 2;
    const int bsz_last = PD / p;
    const int items_last = RQ0 * bsz_last * CQ;
    T yreg[NI][4][CT];
#pragma unroll
    for (int u = 0; u < NI; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < CT; ++c) yreg[u][j][c] = T(0);
    const int fb0 = v.far_by_target[ti], fb1 = v.far_by_target[ti + 1];
    const int per = (fb1 - fb0 + nsplit - 1) / nsplit;
    const int my0 = fb0 + part * per, my1 = min(fb1, my0 + per);
    for (int fb = my0; fb < my1; ++fb) {
        const int t = v.fb_t[fb], key = v.fb_key[fb];
        const int* rk = v.key_ranks + (size_t)key * (Delta + 1);
        const long long* off = v.key_off + (size_t)key * Delta;
        const T* xin = v.xhat + (long long)t * PD * S + c0;
        T* in = z1;
        T* out = z0;
        int a = PD / p;
        for (int i = 0; i < d; ++i) {  // right cores G_Delta, ..., G_{Delta-d+1}
            const int core = Delta - 1 - i;
            __syncthreads();
            if (i == 0) chain_rstep<T, MC>(xin, S, out, v.far_cores + off[core], a, p * rk[core + 1], rk[core]);
            else chain_rstep<T, MC>(in, RS, out, v.far_cores + off[core], a, p * rk[core + 1], rk[core]);
            T* tmp = in; in = out; out = tmp;
            a /= p;
        }
        __syncthreads();
        chain_lstep<T, MC>(in, out, v.H + v.key_hoff[key], rk[d], rk[d + v.dtheta], 1);  // H_k
        { T* tmp = in; in = out; out = tmp; }
        int bsz = 1;
        for (int i = 0; i + 1 < d; ++i) {  // left cores G_d, ..., G_2
            const int core = d - 1 - i;
            __syncthreads();
            chain_lstep<T, MC>(in, out, v.far_cores + off[core], rk[core] * p, rk[core + 1], bsz);
            T* tmp = in; in = out; out = tmp;
            bsz *= p;
        }
        __syncthreads();
        // last left core G_1 (1 x p x r_1): fixed items per thread, accumulated in registers
        {
            const T* G = v.far_cores + off[0];
            const int rin = rk[1];
#pragma unroll
            for (int u = 0; u < NI; ++u) {
                const int item = threadIdx.x + u * kThreads;
                if (item < items_last) {
                    const int cq = item % CQ, rest = item / CQ;
                    const int B = rest % bsz_last, rq = rest / bsz_last;
                    const int nr = min(4, p - 4 * rq);
                    const T* ip = in + (long long)rin * B * RS + cq * CT;
                    for (int k = 0; k < rin; ++k) {
                        T x[CT];
                        load_ct<T, CT>(ip + (long long)k * RS, x);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const T g = (j < nr) ? __ldg(G + 4 * rq + j + p * k) : T(0);
#pragma unroll
                            for (int c = 0; c < CT; ++c) yreg[u][j][c] += g * x[c];
                        }
                    }
                }
            }
        }
    }
    if (my0 >= my1) return;
    T* dst = v.yhat + (long long)s * PD * S + c0;
#pragma unroll
    for (int u = 0; u < NI; ++u) {
        const int item = threadIdx.x + u * kThreads;
        if (item < items_last) {
            const int cq = item % CQ, rest = item / CQ;
            const int B = rest % bsz_last, rq = rest / bsz_last;
            const int nr = min(4, p - 4 * rq);
            for (int j = 0; j < nr; ++j)
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    T* o = dst + (long long)(4 * rq + j + p * B) * S + cq * CT + c;
                    if (nsplit > 1) atomicAdd(o, yreg[u][j][c]);
                    else *o = yreg[u][j][c];
                }
        }
    }
}

// Explicit coupling, phase 1 (grouped by translation class k): for the far blocks b of one item
// (up to four blocks of class k), P = R_k^T xhat_t(b) and z_b = H_k P.  R_k^T is the
// p_s^d-long side of C_k = L_k H_k R_k^T (§4.2), so this is a matrix product with K = p_s^d
// whose A operand is shared by all N = blocks x MC columns of the item.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads, 2) coupling_a_kernel(DevView<T> v, int S, int c0) {
    constexpr int KC = 32, NMAX = 64, BS = NMAX + 4, AS = KC + 1;
    extern __shared__ unsigned char smem_raw[];
    T* As = reinterpret_cast<T*>(smem_raw);  // 64 x AS
    T* Bs = As + 64 * AS;                     // KC x BS
    T* Ps = Bs + KC * BS;                     // 64 x BS
    const int item = blockIdx.x;
    const int key = v.citem_key[item], first = v.citem_first[item], cnt = v.citem_count[item];
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    const int rd = rk[v.d], rp = rk[v.d + v.dtheta];
    const int PD = v.PD, Ntot = cnt * MC;
    const int rp4 = (rp + 3) & ~3;
    const T* Rk = v.far_lr + v.key_lroff[key] + (long long)rd * PD;  // R_k row-major [J * rp4 + s]
    const T* H = v.H + v.key_hoff[key];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int n0 = 0; n0 < Ntot; n0 += NMAX) {  // columns in passes of 64
        const int N = min(NMAX, Ntot - n0);
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[u][j] = T(0);
        for (int k0 = 0; k0 < PD; k0 += KC) {
            const int kn = min(KC, PD - k0);
            __syncthreads();
            for (int e = threadIdx.x; e < rp * KC; e += blockDim.x) {
                const int row = e / KC, kk = e % KC;
                As[row * AS + kk] = (kk < kn) ? Rk[(long long)(k0 + kk) * rp4 + row] : T(0);
            }
            for (int e = threadIdx.x; e < KC * N; e += blockDim.x) {
                const int kk = e / N, col = n0 + e % N;
                const int b = col / MC, c = col % MC;
                const int t = v.fb_t[v.kb_list[first + b]];
                Bs[kk * BS + (col - n0)] = (kk < kn) ? v.xhat[((long long)t * PD + k0 + kk) * S + c0 + c] : T(0);
            }
            __syncthreads();
            if (4 * tx < N) {
#pragma unroll 4
                for (int kk = 0; kk < KC; ++kk) {
                    T bv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) bv[j] = Bs[kk * BS + 4 * tx + j];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const T av = As[(ty + 16 * u) * AS + kk];
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[u][j] += av * bv[j];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ty + 16 * u < rp)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (4 * tx + j < N) Ps[(ty + 16 * u) * BS + 4 * tx + j] = acc[u][j];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = ty + 16 * u;
            if (r >= rd) continue;
            T z[4] = {T(0), T(0), T(0), T(0)};
            for (int q = 0; q < rp; ++q) {
                const T hv = H[r + rd * q];
#pragma unroll
                for (int j = 0; j < 4; ++j) z[j] += hv * Ps[q * BS + 4 * tx + j];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = 4 * tx + j;
                if (col < N) {
                    const int gcol = n0 + col;
                    const int fb = v.kb_list[first + gcol / MC];
                    v.zbuf[((long long)fb * v.zstride + r) * S + c0 + gcol % MC] = z[j];
                }
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Phase 1 of the explicit coupling (§4.5, App. A.4), staged path (p_s^d a multiple of 32, MC >= 4):
// for an item of nb far blocks of class k (nb chosen so that r'_4 x nb MC ~ 8192 outputs,
// r'_4 = r_{d+1} rounded up to 4), P = R_k^T X with X the items' xhat_t columns, then z_b = H_k P.  Chunks of
// R_k (32 x r'_4, row-major) and of X (32 x N) are copied into shared memory with 16-byte
// asynchronous copies, two chunks in flight, so the copy of chunk c + 1 overlaps the products of
// chunk c.  Thread tile: 4 rows of P x 4 columns.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads, 2) coupling_a_staged_kernel(DevView<T> v, int S, int c0) {
    constexpr int KC = 32, NMAX = 256, BS = NMAX + 4;
    constexpr int EV = 16 / sizeof(T);  // elements per 16-byte copy
    extern __shared__ unsigned char smem_raw[];
    T* As = reinterpret_cast<T*>(smem_raw);  // 2 x KC x 64
    T* Bs = As + 2 * KC * 64;                 // 2 x KC x BS; reused for P (64 x BS) after the K loop
    __shared__ long long colbase[16];
    const int item = blockIdx.x;
    const int key = v.citem_key[item], first = v.citem_first[item], cnt = v.citem_count[item];
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    const int rd = rk[v.d], rp = rk[v.d + v.dtheta], rp4 = (rp + 3) & ~3;
    const int PD = v.PD, N = cnt * MC;
    const T* Rk = v.far_lr + v.key_lroff[key] + (long long)rd * PD;  // [J * rp4 + s]
    if (threadIdx.x < cnt) colbase[threadIdx.x] = (long long)v.fb_t[v.kb_list[first + threadIdx.x]] * PD * S + c0;
    __syncthreads();
    auto issue = [&](int chunk, int buf) {
        const int k0 = chunk * KC;
        T* A = As + buf * KC * 64;
        T* B = Bs + buf * KC * BS;
        const T* src = Rk + (long long)k0 * rp4;  // KC x rp4 contiguous
        for (int e = threadIdx.x; e < KC * rp4 / EV; e += blockDim.x) {
            const int kk = (e * EV) / rp4, q = (e * EV) % rp4;
            cp_async16(A + kk * 64 + q, src + e * EV);
        }
        for (int e = threadIdx.x; e < cnt * KC * (MC / EV); e += blockDim.x) {
            const int b = e / (KC * (MC / EV)), rest = e % (KC * (MC / EV));
            const int kk = rest / (MC / EV), q = rest % (MC / EV);
            cp_async16(B + kk * BS + b * MC + q * EV, v.xhat + colbase[b] + (long long)(k0 + kk) * S + q * EV);
        }
        cp_async_commit();
    };
    constexpr int CW = (MC >= 8) ? 8 : 4;  // columns of P per thread (N is a multiple of CW)
    const int TR = rp4 / 4;              // row quads of P
    const int TC = (N + CW - 1) / CW;    // column groups
    const int tr = threadIdx.x % TR, tc = threadIdx.x / TR;
    const bool active = tc < TC;
    T acc[4][CW];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[u][j] = T(0);
    const int nchunks = PD / KC;
    issue(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks) {
            issue(c + 1, (c + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T* A = As + (c & 1) * KC * 64 + 4 * tr;
        const T* B = Bs + (c & 1) * KC * BS + CW * tc;
        if (active) {
#pragma unroll 8
            for (int kk = 0; kk < KC; ++kk) {
                T av[4], bv[CW];
                load_ct<T, 4>(A + kk * 64, av);
#pragma unroll
                for (int h = 0; h < CW; h += 4) load_ct<T, 4>(B + kk * BS + h, *reinterpret_cast<T(*)[4]>(&bv[h]));
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int j = 0; j < CW; j += 2) fma_pair(acc[u][j], acc[u][j + 1], av[u], av[u], bv[j], bv[j + 1]);
            }
        }
        __syncthreads();  // the buffer of chunk c is refilled by the issue of chunk c + 2
    }
    T* Ps = Bs;  // 64 x BS
    if (active)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int h = 0; h < CW; h += 4)
                store_ct<T, 4>(Ps + (4 * tr + u) * BS + CW * tc + h, *reinterpret_cast<T(*)[4]>(&acc[u][h]));
    __syncthreads();
    const T* H = v.H + v.key_hoff[key];
    const int TQ = (N + 3) / 4;  // column quads of z
    for (int e = threadIdx.x; e < rd * TQ; e += blockDim.x) {
        const int r = e / TQ, cq = e % TQ;
        T z[4] = {T(0), T(0), T(0), T(0)};
        for (int q = 0; q < rp; ++q) {
            const T hv = H[r + rd * q];
            T pv[4];
            load_ct<T, 4>(Ps + q * BS + 4 * cq, pv);
#pragma unroll
            for (int j = 0; j < 4; ++j) z[j] += hv * pv[j];
        }
        const int col = 4 * cq;
        if (col < N) {
            const int fb = v.kb_list[first + col / MC];
            store_ct<T, 4>(v.zbuf + ((long long)fb * v.zstride + r) * S + c0 + col % MC, z);
        }
    }
}

// ------------------------------------------------------------------ tcgen05 (5th-generation tensor cores)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }



__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase `parity` of an mbarrier: gives up after about one second (global
// timer), or after 2^28 polls should the timer not advance, and returns false then.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    for (int it = 0; !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity));
        if (!done && (it & 63) == 63 && (global_ns() - t0 > 1000000000ull || it >= (1 << 28) - 1)) break;
    }
    return done != 0;
}

// One CTA waits on an mbarrier that nothing arrives on, with the bounded wait of the bulk-copy and
// tensor-core kernels: out[0] = 1 if the wait ended by the phase completing (it cannot), out[1] =
// nanoseconds waited.
__global__ void wait_bound_kernel(unsigned long long* out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const uint64_t t0 = global_ns();
    const bool done = mbar_wait(&bar, 0);
    const uint64_t t1 = global_ns();
    if (threadIdx.x == 0) {
        out[0] = done ? 1ull : 0ull;
        out[1] = t1 - t0;
    }
}

// The bounded wait of wait_bound_kernel on behalf of a handle: when it runs out it is counted in
// the handle's flags[1] exactly as a production kernel counts a wait that ran out.
__global__ void handle_timeout_kernel(int* flags) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool done = mbar_wait(&bar, 0);
    if (threadIdx.x == 0 && !done) atomicAdd(flags + 1, 1);
}


__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}


__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing
// on an mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bounded wait for phase `parity` of an mbarrier that also gives up as soon as *abort is set
// (another role of the CTA stopped).  Returns true when the phase completed.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort) {
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    for (int it = 0; !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity));
        if (!done && (it & 63) == 63 &&
            (*abort || global_ns() - t0 > 1000000000ull || it >= (1 << 28) - 1))
            break;
    }
    return done != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16 bytes,
// `lbo` bytes apart along K and `sbo` bytes apart along M / N; descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// D (tensor memory) [+]= A (shared memory) x B (shared memory), kind::tf32, one CTA.
__device__ __forceinline__ void umma_tf32_ss(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}



// Each thread of the warp reads 32 consecutive 32-bit columns of its own lane (load and wait in
// one statement).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}



// Phase 1 of the explicit coupling, z_b = H_k R_k^T xhat_t (§4.5; R_k from the right cores,
// App. A.4), on the tensor cores: FP32 data, one chunk of 16 right-hand sides, p_s^d a multiple
// of 32, r_d, r' <= 64.  Persistent: CTA i takes items i, i + G, ... (G = grid size) of up to 8
// far blocks of one class k; the item's 128 (block, right-hand side) pairs are the rows of
//     P^T = X^T R_k,   X = [xhat_t(b)] (p_s^d x 128),  R_k (p_s^d x r'),
// formed by tcgen05.mma kind::tf32 with split operands (3xTF32: x = x_hi + x_lo, products
// hi*hi + hi*lo + lo*hi, so the result keeps FP32 accuracy).  K = p_s^d runs in chunks of 32;
// a task is one chunk of one item.  Warp roles:
//   * warp 0 (producer): bulk copies of each task's inputs into a ring of NS stages: the raw
//     2 KB xhat slices of the item's blocks, and the chunk of R_k stored split (hi, lo) in the
//     K-major no-swizzle operand layout (8-row x 16-byte core matrices, 128 bytes apart along K,
//     256 bytes apart along N, K slices of 8 r'_16 * 32 bytes apart);
//   * warps 2-9 (workers, two per 32-lane quarter of tensor memory): each thread owns one row
//     (block b, right-hand side c) and one half of the chunk's K values; it splits its 16 xhat
//     values and writes hi / lo into one of NA shared-memory A buffers in the same K-major
//     operand layout as B (an MMA that reads A from tensor memory cost several times more per
//     instruction at these small shapes, measured); LAG tasks after a group of KACC
//     chunks it reads its half of the group's product columns back and adds them to P in FP32
//     registers, so the tensor cores never accumulate more than KACC chunks (accumulating all
//     of K on the tensor cores lost accuracy); after an item's last chunk it hands its half of
//     P to the epilogue warps through a shared buffer;
//   * warp 1 (MMA): one thread issues the 12 MMAs of each chunk (4 K slices of 8 x 3 products)
//     into one of NACC accumulator regions (KACC consecutive chunks of an item share one) and
//     commits them to mbarriers that free the stage, the A buffer and, after a region's last
//     chunk, hand the region to the workers;
//   * warps 10-13 (epilogue): stage H_k in shared memory, then z_b[s][c] = sum_q H_k[s, q]
//     P^T[(b, c), q] for one row each, stored to the far blocks' z buffer, overlapped with the
//     next item's MMAs.  The epilogue warps decide together (a barrier reduction) whether to go
//     on, so their barriers never diverge; no other role waits on them except through the P
//     buffers, so no wait can close a cycle.
// Every wait is bounded (about a second): the role that runs out counts it in flags[1] and sets
// a shared abort flag; every role stops issuing work, waits (bounded) for the copies and MMAs it
// started, and the CTA frees its tensor memory before it exits.
namespace tc2 {
constexpr int NS = 3;                          // stages of the bulk-copy ring
constexpr int NA = 2;                          // shared-memory A buffers (hi + lo, 128 x 32 each)
constexpr int NACC = 4;                        // tensor-memory accumulator regions (64 columns each)
constexpr int KACC = 2;                        // chunks of 32 accumulated in one region before it is read
constexpr int LAG = 3;                         // a group is drained after the A operand LAG tasks later is stored
constexpr int NW = 8;                          // worker warps
constexpr int XROW = 2048 + 64;                // bytes per block slice in a stage (bank padding)
constexpr int XS_BYTES = 8 * XROW;             // raw xhat slices of one stage
constexpr int BS_BYTES = 2 * 32 * 64 * 4;      // R_k chunk, hi + lo, r'_16 <= 64
constexpr int STAGE = XS_BYTES + BS_BYTES;
constexpr int PROW = 65;                       // floats per row of a P hand-off buffer (bank padding)
constexpr int PS_BYTES = 128 * PROW * 4;
constexpr int HS_BYTES = 64 * 64 * 4;          // H_k staged by the epilogue: [q][s], s padded to 64
constexpr int APART = 128 * 32 * 4;            // one part (hi or lo) of an A buffer
constexpr int SMEM = NS * STAGE + NA * 2 * APART + PS_BYTES + HS_BYTES;
constexpr int EPI0 = 2 + NW;                   // first epilogue warp
constexpr int THREADS = 32 * (EPI0 + 4);
constexpr uint32_t ACC_COL = 0;                // accumulators at columns [0, 256)
constexpr int TMEM_COLS = 256;
}  // namespace tc2

// Barrier `id` over `n` threads that also returns the AND of every participant's `v`.
__device__ __forceinline__ bool bar_and(bool v, int id, int n) {
    int r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 q, %1, 0;\n bar.red.and.pred p, %2, %3, q;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(r)
                 : "r"((int)v), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(tc2::THREADS, 1) coupling_a_umma_kernel(DevView<float> v) {
    using namespace tc2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* abuf = smem_raw + NS * STAGE;                         // NA x (hi, lo)
    float* pbuf = reinterpret_cast<float*>(abuf + NA * 2 * APART);       // 128 x PROW
    float* hs = pbuf + 128 * PROW;                                       // 64 x 64
    __shared__ __align__(8) uint64_t full[NS], sempty[NS], aready[NA], aempty[NA], accfull[NACC], accempty[NACC];
    __shared__ __align__(8) uint64_t pfull, pempty;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int PD = v.PD, nchunks = PD / 32, ngroups = (nchunks + KACC - 1) / KACC;
    const int G = gridDim.x;
    const int my_items = (v.n_tcitems - (int)blockIdx.x + G - 1) / G;
    const int T = my_items * nchunks;
    volatile int* abortp = &abort_flag;

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&sempty[i], 1 + NW);  // MMA commit (B read) + the worker warps (xhat read)
        }
        for (int i = 0; i < NA; ++i) {
            mbar_init(&aready[i], NW);
            mbar_init(&aempty[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accempty[i], NW);
        }
        mbar_init(&pfull, NW);
        mbar_init(&pempty, 4);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;

    // the item of local index j and its class data (every role loads the next item's data one
    // item ahead, so that these dependent global loads never stall the pipeline)
    struct Item {
        int key, first, cnt, rd, rp;
        long long hoff, tcoff;
    };
    auto item_at = [&](int j) {
        Item it;
        const int idx = (int)blockIdx.x + min(j, my_items - 1) * G;
        it.key = v.tcitem_key[idx];
        it.first = v.tcitem_first[idx];
        it.cnt = v.tcitem_count[idx];
        const int* rk = v.key_ranks + (size_t)it.key * (v.Delta + 1);
        it.rd = rk[v.d];
        it.rp = rk[v.d + v.dtheta];
        it.hoff = v.key_hoff[it.key];
        it.tcoff = v.key_tcoff[it.key];
        return it;
    };
    auto fail = [&]() {
        if (atomicExch(&abort_flag, 1) == 0) atomicAdd(v.flags + 1, 1);
    };
    auto group_of = [&](int t) { return (t / nchunks) * ngroups + (t % nchunks) / KACC; };
    auto group_end = [&](int t) {
        const int ch = t % nchunks;
        return (ch % KACC == KACC - 1) || ch == nchunks - 1;
    };

    if (warp == 0) {
        // ------------------------------------------------------------------ producer
        if (lane == 0) {
            int issued = 0;
            Item it{}, nxt = item_at(0);
            int src[8], nsrc[8];
            auto load_src = [&](const Item& x, int (&o)[8]) {
#pragma unroll
                for (int i = 0; i < 8; ++i) o[i] = (i < x.cnt) ? v.kb_list[x.first + i] : 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) o[i] = (i < x.cnt) ? v.fb_t[o[i]] : 0;
            };
            load_src(nxt, nsrc);
            for (int t = 0; t < T; ++t) {
                const int st = t % NS, ch = t % nchunks;
                if (ch == 0) {
                    it = nxt;
#pragma unroll
                    for (int i = 0; i < 8; ++i) src[i] = nsrc[i];
                    nxt = item_at(t / nchunks + 1);
                    load_src(nxt, nsrc);
                }
                if (t >= NS && !mbar_wait_ab(&sempty[st], (uint32_t)((t / NS - 1) & 1), abortp)) {
                    fail();
                    break;
                }
                if (*abortp) break;
                const int r16 = (it.rp + 15) & ~15;
                const uint32_t bbytes = 2u * 32u * (uint32_t)r16 * 4u;
                unsigned char* stg = smem_raw + st * STAGE;
                mbar_expect_tx(&full[st], (uint32_t)it.cnt * 2048u + bbytes);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i < it.cnt)
                        bulk_g2s(stg + i * XROW, v.xhat + (long long)src[i] * PD * 16 + (long long)ch * 512, 2048u,
                                 &full[st]);
                bulk_g2s(stg + XS_BYTES, v.far_tc + it.tcoff + (size_t)ch * 2 * 32 * r16, bbytes, &full[st]);
                issued = t + 1;
            }
            // before the shared memory goes: wait (bounded) for the copies still in flight
            for (int u = max(0, issued - NS); u < issued; ++u) mbar_wait(&full[u % NS], (uint32_t)((u / NS) & 1));
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int issued = 0, gdone = 0;
            uint32_t idesc = 0, r16 = 16;
            Item nxt = item_at(0);
            for (int t = 0; t < T; ++t) {
                const int st = t % NS, a = t % NA, ch = t % nchunks;
                const int g = group_of(t), r = g % NACC;
                const bool gfirst = ch % KACC == 0, glast = group_end(t);
                if (ch == 0) {
                    const Item it = nxt;
                    nxt = item_at(t / nchunks + 1);
                    r16 = (uint32_t)((it.rp + 15) & ~15);
                    idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((r16 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
                }
                bool ok = mbar_wait_ab(&full[st], (uint32_t)((t / NS) & 1), abortp);
                ok = ok && mbar_wait_ab(&aready[a], (uint32_t)((t / NA) & 1), abortp);
                if (ok && gfirst && g >= NACC)
                    ok = mbar_wait_ab(&accempty[r], (uint32_t)((g / NACC - 1) & 1), abortp);
                if (!ok || *abortp) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t b_hi = smem_u32(smem_raw + st * STAGE + XS_BYTES);
                const uint32_t b_lo = b_hi + 32u * r16 * 4u;
                const uint32_t a_hi = smem_u32(abuf + a * 2 * APART), a_lo = a_hi + APART;
                const uint32_t d = tmem + ACC_COL + (uint32_t)r * 64u;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const uint32_t bo = (uint32_t)s * r16 * 32u, ao = (uint32_t)s * 128u * 32u;
                    umma_tf32_ss(d, umma_desc2(a_hi + ao, 128, 256), umma_desc2(b_hi + bo, 128, 256), idesc,
                                 (s == 0 && gfirst) ? 0u : 1u);
                    umma_tf32_ss(d, umma_desc2(a_hi + ao, 128, 256), umma_desc2(b_lo + bo, 128, 256), idesc, 1u);
                    umma_tf32_ss(d, umma_desc2(a_lo + ao, 128, 256), umma_desc2(b_hi + bo, 128, 256), idesc, 1u);
                }
                umma_commit(&sempty[st]);
                umma_commit(&aempty[a]);
                if (glast) {
                    umma_commit(&accfull[r]);
                    gdone = g + 1;
                }
                issued = t + 1;
            }
            // the MMAs issued last complete before the tensor memory is freed: after an abort in
            // the middle of a group, commit what was issued to that group's region first
            if (issued > 0) {
                const int gl = group_of(issued - 1);
                if (gdone <= gl) umma_commit(&accfull[gl % NACC]);
                mbar_wait(&accfull[gl % NACC], (uint32_t)((gl / NACC) & 1));
            }
        }
    } else if (warp < EPI0) {
        // ------------------------------------------------------------------ workers
        const int q = warp & 3;              // tensor-memory lane quarter of this warp
        const int hh = (warp - 2) / 4;       // half of the K values (split) and of the columns (drain)
        const int row = 32 * q + lane;       // (block b, right-hand side c)
        const int b = row / 16, c = row % 16;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        float P[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) P[jj] = 0.0f;
        bool ok = true;
        Item cur{}, nxt = item_at(0);  // item of the task being split, and the one after it
        Item drn{}, dnxt = nxt;        // item of the group being drained, and the one after it
        // adds this warp's half of the product columns of the group ending with task u to P;
        // after an item's last chunk, hands P to the epilogue warps
        auto drain = [&](int u) -> bool {
            const int ch = u % nchunks, j = u / nchunks;
            const int g = group_of(u), r = g % NACC;
            if (!mbar_wait_ab(&accfull[r], (uint32_t)((g / NACC) & 1), abortp)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (ch < KACC) {
                drn = dnxt;
                dnxt = item_at(j + 1);
            }
            if (32 * hh < drn.rp) {  // warp-uniform
                float pv[32];
                tmem_ld32(tmem + lane_base + ACC_COL + (uint32_t)r * 64u + 32u * hh, pv);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) P[jj] += (32 * hh + jj < drn.rp) ? pv[jj] : 0.0f;
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[r]);
            if (ch != nchunks - 1) return true;
            if (j >= 1 && !mbar_wait_ab(&pempty, (uint32_t)((j - 1) & 1), abortp)) return false;
            float* dst = pbuf + row * PROW + 32 * hh;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                dst[jj] = P[jj];
                P[jj] = 0.0f;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&pfull);
            return true;
        };
        for (int t = 0; t < T && ok; ++t) {
            const int st = t % NS, a = t % NA;
            if (t % nchunks == 0) {
                cur = nxt;
                nxt = item_at(t / nchunks + 1);
            }
            ok = mbar_wait_ab(&full[st], (uint32_t)((t / NS) & 1), abortp);
            if (ok && t >= NA) ok = mbar_wait_ab(&aempty[a], (uint32_t)((t / NA - 1) & 1), abortp);
            if (!ok) break;
            const float* xs = reinterpret_cast<const float*>(smem_raw + st * STAGE + b * XROW) + 16 * 16 * hh + c;
            float hi[16], lo[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float x = (b < cur.cnt) ? xs[i * 16] : 0.0f;
                hi[i] = tf32_rna(x);
                lo[i] = tf32_rna(x - hi[i]);
            }
            // element (row, k) of a part at (k / 8) 4096 + (row / 8) 256 + ((k % 8) / 4) 128 +
            // (row % 8) 16 + (k % 4) 4 bytes: 8-row x 16-byte core matrices, 128 bytes apart along
            // K, 256 bytes apart along M, K slices of 8 4096 bytes apart
            unsigned char* ahi = abuf + a * 2 * APART;
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4) {
                const int k = 16 * hh + 4 * g4;
                const uint32_t off = (k / 8) * 4096 + (row / 8) * 256 + ((k % 8) / 4) * 128 + (row % 8) * 16;
                *reinterpret_cast<float4*>(ahi + off) = make_float4(hi[4 * g4], hi[4 * g4 + 1], hi[4 * g4 + 2], hi[4 * g4 + 3]);
                *reinterpret_cast<float4*>(ahi + APART + off) =
                    make_float4(lo[4 * g4], lo[4 * g4 + 1], lo[4 * g4 + 2], lo[4 * g4 + 3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&aready[a]);
                mbar_arrive(&sempty[st]);
            }
            // drain the group that ended LAG tasks ago, so that the MMAs of the last few tasks run
            // while this warp splits the next operands (LAG < NA keeps the A buffers flowing)
            if (t >= LAG && group_end(t - LAG)) {
                ok = drain(t - LAG);
                if (!ok) break;
            }
        }
        for (int u = max(0, T - LAG); u < T && ok; ++u)
            if (group_end(u)) ok = drain(u);
        if (!ok) fail();
    } else {
        // ------------------------------------------------------------------ epilogue
        const int row = tid - 32 * EPI0;
        const int b = row / 16, c = row % 16;
        Item nxt = item_at(0);
        int nfb = (b < nxt.cnt) ? v.kb_list[nxt.first + b] : 0;
        for (int j = 0; j < my_items; ++j) {
            const Item it = nxt;
            const int fb = nfb;
            nxt = item_at(j + 1);
            nfb = (b < nxt.cnt) ? v.kb_list[nxt.first + b] : 0;
            // one decision for all epilogue warps (a barrier that also guarantees that every
            // epilogue thread is done with the previous item's H_k)
            const bool ok = bar_and(mbar_wait_ab(&pfull, (uint32_t)(j & 1), abortp), 1, 128);
            if (!ok) {
                fail();
                break;
            }
            // H_k (r_d x r', column-major in global memory) into hs[q][s], s padded to 64
            const float* H = v.H + it.hoff;
            for (int e = row; e < it.rd * it.rp; e += 128) {
                const int s = e % it.rd, qq = e / it.rd;
                hs[qq * 64 + s] = H[e];
            }
            float Pr[64];
            const float* pr = pbuf + row * PROW;
#pragma unroll
            for (int qq = 0; qq < 64; ++qq) Pr[qq] = (qq < it.rp) ? pr[qq] : 0.0f;
            __syncwarp();
            if (lane == 0) mbar_arrive(&pempty);
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (b < it.cnt) {
                float* dst = v.zbuf + (long long)fb * v.zstride * 16 + c;
                for (int s0 = 0; s0 < it.rd; s0 += 4) {
                    // four rows s0..s0+3 of H_k per shared-memory vector read
                    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int qq = 0; qq < 64; ++qq) {
                        if (qq < it.rp) {
                            const float4 h4 = *reinterpret_cast<const float4*>(hs + qq * 64 + s0);
                            z[0] = fmaf(h4.x, Pr[qq], z[0]);
                            z[1] = fmaf(h4.y, Pr[qq], z[1]);
                            z[2] = fmaf(h4.z, Pr[qq], z[2]);
                            z[3] = fmaf(h4.w, Pr[qq], z[3]);
                        }
                    }
                    const int ns = min(4, it.rd - s0);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (e < ns) dst[(long long)(s0 + e) * 16] = z[e];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Near field Y_s += reshape(G_{b,1} w_b) X_t (§4.3, applied as in §4.5), bulk-copy pipelined
// (FP32 / FP64, chunks of MC right-hand sides with S == MC, leaves of at most kThreads points,
// r ns <= the stage size).  One CTA per near work item, as near_kernel, with a producer warp: the
// cores G_{b,1} of the item's blocks are streamed in chunks of whole columns j (each chunk
// contiguous in memory: [(j r + k) ns + i]) by 1-D bulk copies into a ring of NS stages, together
// with the rows x_t of each block (into one buffer per block).  The eight consumer warps form
// d_ij = sum_k w_k G[(j r + k) ns + i] from shared memory and accumulate d_ij x_t[j][c] as
// near_kernel does; a stage is handed back through an mbarrier arrival per consumer warp, so the
// CTA never stops at a full barrier while the cores stream.
//
// Mirror sharing: a stored block (s, t) with s != t also stands for the block (t, s), whose
// matrix is D_st^T.  The consumers then also write d_ij into a slice of up to JBM columns of D_st
// in shared memory, and when the slice is full every warp takes a pair of its columns: lane
// (segment, column group) sums d_ij x_s[i][c] over its segment of rows i, a butterfly over the
// segments completes (D_st^T x_s)[j][c], and the result goes to the block's mirror slot, from
// which combine_kernel adds it to leaf t.  One read of G_{b,1} serves both blocks.  A slice costs
// two consumer barriers: slice complete (which also carries the abort vote) and slice read.
//
// Every wait is bounded: after a timeout the CTA counts it in flags[1], stops issuing copies and
// waits (bounded) for those in flight before it exits.
namespace nt1 {
constexpr int NS = 4;                    // stages
constexpr int STAGE = 16384;             // bytes of cores per stage
constexpr int STB = STAGE + 32;          // plus the 16-byte rounding of a chunk's start and end
constexpr int kConsumers = kThreads / 32;
constexpr int JBM = 2 * kConsumers;      // columns of a D slice (one pair per consumer warp)
}  // namespace nt1

// Columns of a block per stage chunk (at most `cap`).
template <typename T>
__device__ __forceinline__ int near_chunk_cols(int r, int ns, int cap) {
    const long long colf = (long long)r * ns;
    const int J = (int)(nt1::STAGE / (colf * (long long)sizeof(T)));
    return J < 1 ? 1 : (J > cap ? cap : J);
}

// Shared memory of near_tma_kernel: the stages, the x_t buffers (4, or 2 with mirror sharing),
// and with sharing x_s and a D slice of JBM columns.
template <typename T>
__host__ __device__ inline size_t near_tma_smem(int maxleaf, int mc, bool share) {
    size_t b = (size_t)nt1::NS * nt1::STB + (size_t)(share ? 2 : 4) * maxleaf * mc * sizeof(T);
    if (share) b += ((size_t)maxleaf * mc + (size_t)nt1::JBM * maxleaf) * sizeof(T);
    return b;
}

template <typename T, int MC>
__global__ void __launch_bounds__(kThreads + 32, 2) near_tma_kernel(DevView<T> v, int maxleaf) {
    using namespace nt1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool share = v.near_share != 0;
    const int XB = share ? 2 : 4;                               // x_t buffers
    unsigned char* stg = smem_raw;                              // NS x STB
    T* xs = reinterpret_cast<T*>(smem_raw + NS * STB);          // XB x maxleaf x MC (one per block)
    T* xsrc = xs + (size_t)XB * maxleaf * MC;                   // maxleaf x MC: x_s (sharing)
    T* dcur = xsrc + (size_t)maxleaf * MC;                      // JBM x maxleaf: the D slice
    T* red = reinterpret_cast<T*>(smem_raw);                    // kThreads x MC, after the stream
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int item = blockIdx.x;
    const int leaf = v.item_leaf[item];
    const int snode = v.leaf_node[leaf];
    const int sbeg = v.node_begin[snode];
    const int ns = v.node_end[snode] - sbeg;
    const int b0 = v.item_first[item], b1 = b0 + v.item_count[item];
    const int jcap = share ? JBM : 1 << 20;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumers);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumers) {
        // ---------------- producer warp: lane 0 issues the copies of every chunk of the item
        if (lane == 0) {
            int t = 0;
            bool ok = true;
            for (int b = b0; b < b1 && ok; ++b) {
                const int r = v.nb_rank[b];
                const int tnode = v.nb_t[b];
                const int tb = v.node_begin[tnode], nt = v.node_end[tnode] - tb;
                const long long colf = (long long)r * ns;
                const int J = near_chunk_cols<T>(r, ns, jcap);
                for (int j0 = 0; j0 < nt; j0 += J, ++t) {
                    const int st = t % NS;
                    if (t >= NS) ok = mbar_wait(&empty[st], (uint32_t)(((t / NS) - 1) & 1));
                    if (!ok || *(volatile int*)&abort_flag) {
                        ok = false;
                        break;
                    }
                    const int jn = min(J, nt - j0);
                    const uintptr_t a0 = (uintptr_t)(v.near_cores + v.nb_off[b] + j0 * colf);
                    const uintptr_t a1 = a0 + (uintptr_t)(jn * colf) * sizeof(T);
                    const uintptr_t s0 = a0 & ~(uintptr_t)15, e0 = (a1 + 15) & ~(uintptr_t)15;
                    uint32_t bytes = (uint32_t)(e0 - s0);
                    const uint32_t xbytes = (j0 == 0) ? (uint32_t)(nt * MC * sizeof(T)) : 0u;
                    const uint32_t sbytes = (share && t == 0) ? (uint32_t)(ns * MC * sizeof(T)) : 0u;
                    mbar_expect_tx(&full[st], bytes + xbytes + sbytes);
                    bulk_g2s(stg + st * STB, (const void*)s0, bytes, &full[st]);
                    if (xbytes)
                        bulk_g2s(xs + (size_t)(b - b0) * maxleaf * MC, v.Xc + (long long)tb * MC, xbytes, &full[st]);
                    if (sbytes) bulk_g2s(xsrc, v.Xc + (long long)sbeg * MC, sbytes, &full[st]);
                }
            }
            if (!ok) {
                atomicAdd(v.flags + 1, 1);
                abort_flag = 1;
            }
            // before the CTA's shared memory goes: wait (bounded) for the copies still in flight,
            // i.e. the last NS chunks issued
            for (int u = max(0, t - NS); u < t; ++u) mbar_wait(&full[u % NS], (uint32_t)((u / NS) & 1));
        }
        return;
    }

    // ---------------- consumer warps
    const int RP = (ns + 31) & ~31;
    const int G = kThreads / RP;
    const int i = tid % RP, g = tid / RP;
    const bool active = (g < G) && (i < ns);
    // mirror product lanes: lane = cg + CG * seg; rows of segment seg start seglen apart (odd, so
    // the segments of one load fall in distinct banks)
    constexpr int VW = 16 / (int)sizeof(T);
    constexpr int CG = MC >= VW ? MC / VW : 1, SEGS = 32 / CG;  // (launched only for MC >= VW)
    const int seg = lane / CG, cg = lane % CG;
    const int seglen = ((ns + SEGS - 1) / SEGS) | 1;
    T acc[MC];
#pragma unroll
    for (int c = 0; c < MC; ++c) acc[c] = T(0);
    bool ok = true;
    int t = 0;
    for (int b = b0; b < b1; ++b) {
        const int r = v.nb_rank[b];
        const int tnode = v.nb_t[b];
        const int nt = v.node_end[tnode] - v.node_begin[tnode];
        const long long colf = (long long)r * ns;
        const int J = near_chunk_cols<T>(r, ns, jcap);
        const int mslot = share ? v.nb_mslot[b] : -1;
        constexpr int RK = 8;  // ranks up to RK use the unrolled path
        T wr[RK];
        const T* wb = v.w + v.nb_woff[b];
#pragma unroll
        for (int k = 0; k < RK; ++k) wr[k] = (k < r) ? wb[k] : T(0);
        const T* xsb = xs + (size_t)(b - b0) * maxleaf * MC;
        int fbase = 0;  // first column of the current D slice
        for (int j0 = 0; j0 < nt; j0 += J, ++t) {
            const int st = t % NS;
            if (ok) ok = mbar_wait(&full[st], (uint32_t)((t / NS) & 1)) && !*(volatile int*)&abort_flag;
            const int jn = min(J, nt - j0);
            if (ok) {
                const uintptr_t a0 = (uintptr_t)(v.near_cores + v.nb_off[b] + j0 * colf);
                const T* Gs = reinterpret_cast<const T*>(stg + st * STB + (a0 & 15)) + i;
                if (active) {
                    for (int jj = g; jj < jn; jj += G) {
                        const T* gj = Gs + jj * colf;
                        T dij = T(0);
                        if (r <= RK) {
#pragma unroll
                            for (int k = 0; k < RK; ++k)
                                if (k < r) dij += wr[k] * gj[(long long)k * ns];
                        } else {
                            for (int k = 0; k < r; ++k) dij += wb[k] * gj[(long long)k * ns];
                        }
                        const T* xj = xsb + (j0 + jj) * MC;
#pragma unroll
                        for (int c = 0; c < MC; c += 2) fma_pair(acc[c], acc[c + 1], dij, dij, xj[c], xj[c + 1]);
                        if (mslot >= 0) dcur[(size_t)(j0 + jj - fbase) * maxleaf + i] = dij;
                    }
                }
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[st])) : "memory");
            }
            if (mslot < 0) continue;
            // mirror product of the slice once it is full (block-uniform decision)
            const int jend = j0 + jn;
            if (jend < nt && jend + min(J, nt - jend) - fbase <= JBM) continue;
            ok = bar_and(ok, 1, kThreads);  // the slice is complete in every warp
            const int ncols = jend - fbase, jc = 2 * warp;
            if (ok && jc < ncols) {
                T a0[VW], a1[VW];
#pragma unroll
                for (int e = 0; e < VW; ++e) a0[e] = a1[e] = T(0);
                const T* D0 = dcur + (size_t)jc * maxleaf;
                const T* D1 = D0 + maxleaf;  // a column past ncols holds stale values: never stored
                const int i0 = seg * seglen, i1 = min(ns, i0 + seglen);
                for (int ii = i0; ii < i1; ++ii) {
                    const T d0 = D0[ii], d1 = D1[ii];
                    T xv[VW];
                    load_ct<T, VW>(xsrc + (size_t)ii * MC + cg * VW, xv);
#pragma unroll
                    for (int e = 0; e < VW; e += 2) {
                        fma_pair(a0[e], a0[e + 1], d0, d0, xv[e], xv[e + 1]);
                        fma_pair(a1[e], a1[e + 1], d1, d1, xv[e], xv[e + 1]);
                    }
                }
#pragma unroll
                for (int off = CG; off < 32; off <<= 1)
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        a0[e] += __shfl_xor_sync(0xffffffffu, a0[e], off);
                        a1[e] += __shfl_xor_sync(0xffffffffu, a1[e], off);
                    }
                if (seg < 2 && jc + seg < ncols) {
                    T* dst = v.partials + ((long long)(v.n_items + mslot) * v.part_stride + fbase + jc + seg) * MC + cg * VW;
#pragma unroll
                    for (int e = 0; e < VW; ++e) dst[e] = seg == 0 ? a0[e] : a1[e];
                }
            }
            fbase = jend;
            asm volatile("bar.sync 1, %0;" ::"r"(kThreads) : "memory");  // the slice was read
        }
    }
    if (!ok && lane == 0) atomicExch(&abort_flag, 1);
    // reduce the column groups (the stages are no longer written: every chunk was consumed)
    asm volatile("bar.sync 1, %0;" ::"r"(kThreads) : "memory");
    if (ok) {
#pragma unroll
        for (int c = 0; c < MC; ++c) red[tid * MC + c] = acc[c];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kThreads) : "memory");
    if (ok && g == 0 && i < ns) {
        for (int gg = 1; gg < G; ++gg)
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[c] += red[(gg * RP + i) * MC + c];
        T* part = v.partials + (long long)item * v.part_stride * MC;
#pragma unroll
        for (int c = 0; c < MC; ++c) part[(long long)i * MC + c] = acc[c];
    }
}

// Explicit coupling, phase 2 (grouped by target s): yhat_s += sum over far blocks b of s of
// L_k z_b, L_k = (I (x) G_1^{2}) ... G_d^{2} formed offline (App. A.4).  Thread tile: 8
// consecutive rows of yhat_s x CT right-hand sides; z_b staged in shared memory eight blocks at a
// time.  The far blocks of a target are split over `nsplit` CTAs that meet in yhat via atomics.
template <typename T, int MC, int NIB>
__global__ void __launch_bounds__(kThreads, 2) coupling_b_kernel(DevView<T> v, int S, int c0, int nsplit) {
    constexpr int CT = MC < 4 ? MC : 4, CQ = MC / CT, RPT = 8, ZB = 8;
    extern __shared__ unsigned char smem_raw[];
    T* zs = reinterpret_cast<T*>(smem_raw);  // ZB x zstride x MC
    const int PD = v.PD, zst = v.zstride;
    const int ti = blockIdx.x / nsplit, part = blockIdx.x % nsplit;
    const int s = v.far_targets[ti];
    const int fb0 = v.far_by_target[ti], fb1 = v.far_by_target[ti + 1];
    const int per = (fb1 - fb0 + nsplit - 1) / nsplit;
    const int my0 = fb0 + part * per, my1 = min(fb1, my0 + per);
    if (my0 >= my1) return;
    const int RG = (PD + RPT - 1) / RPT;
    const int items = RG * CQ;
    const bool vec = (PD % 4) == 0;
    T acc[NIB][RPT][CT];
#pragma unroll
    for (int u = 0; u < NIB; ++u)
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[u][i][c] = T(0);
    for (int g0 = my0; g0 < my1; g0 += ZB) {
        const int nb = min(ZB, my1 - g0);
        __syncthreads();
        for (int e = threadIdx.x; e < nb * zst * MC; e += blockDim.x) {
            const int bi = e / (zst * MC), rest = e % (zst * MC);
            zs[e] = v.zbuf[((long long)(g0 + bi) * zst + rest / MC) * S + c0 + rest % MC];
        }
        __syncthreads();
        for (int bi = 0; bi < nb; ++bi) {
            const int key = v.fb_key[g0 + bi];
            const int rd = v.key_ranks[(size_t)key * (v.Delta + 1) + v.d];
            const T* Lt = v.far_lr + v.key_lroff[key];
            const T* zb = zs + bi * zst * MC;
#pragma unroll
            for (int u = 0; u < NIB; ++u) {
                const int it = threadIdx.x + u * kThreads;
                if (it >= items) continue;
                const int cq = it % CQ, rg = it / CQ;
                const int I0 = rg * RPT;
                const bool full = vec && (I0 + RPT <= PD);
                int q = 0;
                if (NIB == 1 && full) {
                    // four columns of L_k per step, all loads issued before the products
                    for (; q + 4 <= rd; q += 4) {
                        T l[4][RPT];
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const T* lp = Lt + (long long)(q + w) * PD + I0;
                            load_ct<T, 4>(lp, *reinterpret_cast<T(*)[4]>(&l[w][0]));
                            load_ct<T, 4>(lp + 4, *reinterpret_cast<T(*)[4]>(&l[w][4]));
                        }
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            T x[CT];
                            load_ct<T, CT>(zb + (q + w) * MC + cq * CT, x);
#pragma unroll
                            for (int i = 0; i < RPT; ++i)
#pragma unroll
                                for (int c = 0; c < CT; ++c) acc[u][i][c] += l[w][i] * x[c];
                        }
                    }
                }
                for (; q < rd; ++q) {
                    T l[RPT];
                    const T* lp = Lt + (long long)q * PD + I0;
                    if (full) {
                        load_ct<T, 4>(lp, *reinterpret_cast<T(*)[4]>(&l[0]));
                        load_ct<T, 4>(lp + 4, *reinterpret_cast<T(*)[4]>(&l[4]));
                    } else {
#pragma unroll
                        for (int i = 0; i < RPT; ++i) l[i] = (I0 + i < PD) ? lp[i] : T(0);
                    }
                    T x[CT];
                    load_ct<T, CT>(zb + q * MC + cq * CT, x);
#pragma unroll
                    for (int i = 0; i < RPT; ++i)
#pragma unroll
                        for (int c = 0; c < CT; ++c) acc[u][i][c] += l[i] * x[c];
                }
            }
        }
    }
    T* dst = v.yhat + (long long)s * PD * S + c0;
#pragma unroll
    for (int u = 0; u < NIB; ++u) {
        const int it = threadIdx.x + u * kThreads;
        if (it >= items) continue;
        const int cq = it % CQ, rg = it / CQ;
        for (int i = 0; i < RPT; ++i) {
            const int I = rg * RPT + i;
            if (I >= PD) break;
            T* o = dst + (long long)I * S + cq * CT;
            if (nsplit > 1) atomic_add_ct<T, CT>(o, acc[u][i]);
            else store_ct<T, CT>(o, acc[u][i]);
        }
    }
}

// H format far field (§4.5): y_s += S_b (H_k (T_b^T x_t)) for every far block of target s.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) far_h_kernel(DevView<T> v, int S, int c0, int rmax) {
    extern __shared__ unsigned char smem_raw[];
    const int ti = blockIdx.x;
    const int s = v.far_targets[ti];
    const int row0 = v.node_begin[s], ns = v.node_end[s] - row0;
    T* ys = reinterpret_cast<T*>(smem_raw);   // ns x MC
    T* tv = ys + (size_t)ns * MC;             // rmax x MC
    T* uv = tv + (size_t)rmax * MC;           // rmax x MC
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
    for (int e = threadIdx.x; e < ns * MC; e += blockDim.x) ys[e] = T(0);
    for (int fb = v.far_by_target[ti]; fb < v.far_by_target[ti + 1]; ++fb) {
        const int t = v.fb_t[fb], key = v.fb_key[fb];
        const int tb = v.node_begin[t], nt = v.node_end[t] - tb;
        const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
        const int ra = rk[v.d], rb = rk[v.d + v.dtheta];
        const T* Sb = v.st + v.fb_soff[fb];
        const T* Tb = v.st + v.fb_toff[fb];
        const T* H = v.H + v.key_hoff[key];
        __syncthreads();
        for (int q = warp; q < rb; q += nwarps) {  // tv[q] = T_b[:, q]^T x_t
            T acc[MC];
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[c] = T(0);
            for (int j = lane; j < nt; j += 32) {
                const T tj = Tb[(long long)q * nt + j];
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[c] += tj * v.Xc[(long long)(tb + j) * S + c0 + c];
            }
#pragma unroll
            for (int c = 0; c < MC; ++c) {
                T x = acc[c];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) tv[q * MC + c] = x;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ra * MC; e += blockDim.x) {  // uv = H tv
            const int x = e / MC, c = e % MC;
            T acc = T(0);
            for (int y = 0; y < rb; ++y) acc += H[x + ra * y] * tv[y * MC + c];
            uv[e] = acc;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {  // ys += S_b uv
            T acc[MC];
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[c] = T(0);
            for (int x = 0; x < ra; ++x) {
                const T sv = Sb[(long long)x * ns + i];
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[c] += sv * uv[x * MC + c];
            }
#pragma unroll
            for (int c = 0; c < MC; ++c) ys[i * MC + c] += acc[c];
        }
    }
    __syncthreads();
    T* dst = v.yfar + (long long)v.level_slot[v.node_level[s]] * v.n * S;
    for (int e = threadIdx.x; e < ns * MC; e += blockDim.x)
        dst[(long long)(row0 + e / MC) * S + c0 + e % MC] = ys[e];
}

// Y[perm[i] + c ldy] = sum of the leaf's near partials + (U_s yhat_s)[i][c] (H^2, leaf stage of
// FastBackward) or + sum over levels of y_far (H).  One CTA per leaf.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) combine_kernel(DevView<T> v, T* __restrict__ Y, long long ldy,
                                                           int m, int S, int c0, int h2, int pull_level) {
    extern __shared__ unsigned char smem_raw[];
    T* sy = reinterpret_cast<T*>(smem_raw);  // PD x MC
    const int leaf = blockIdx.x;
    const int node = v.leaf_node[leaf];
    const int row0 = v.node_begin[node], ns = v.node_end[node] - row0;
    const int ps = v.p_s, d = v.d, PD = v.PD;
    if (h2) {
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            sy[e] = v.yhat[((long long)node * PD + e / MC) * S + c0 + e % MC];
        const int parent = v.node_parent[node];
        if (parent >= 0 && v.node_level[parent] >= pull_level) {
            // last level of Alg. FastBackward: yhat_s += (E_{s,d} (x) .. (x) E_{s,1}) yhat_parent
            T* sE = sy + (size_t)PD * MC;
            T* b0 = sE + ((2 * ps * ps + 3) & ~3);
            T* b1 = b0 + (size_t)PD * MC;
            for (int e = threadIdx.x; e < 2 * ps * ps; e += blockDim.x) sE[e] = v.E[e];
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
                b0[e] = v.yhat[((long long)parent * PD + e / MC) * S + c0 + e % MC];
            const int halves = v.node_halves[node];
            T* in = b0;
            T* out = b1;
            int stride = 1;
            for (int k = 0; k < d; ++k) {
                __syncthreads();
                const bool last = (k == d - 1);
                mode_product<T, MC>(in, last ? sy : out, sE + ((halves >> k) & 1) * ps * ps, ps, PD, stride, false,
                                    last);
                T* t = in; in = out; out = t;
                stride *= ps;
            }
        }
        __syncthreads();
    }
    constexpr int CT = MC < 4 ? MC : 4, CQ = MC / CT;
    // thread item = (row i, CT columns); U factors of the rows staged per chunk of rows
    T* su = sy + (size_t)PD * MC;  // reuses the transfer scratch: kThreads rows x d x p_s
    const int p1 = ps, p2 = d > 1 ? ps : 1, p3 = d > 2 ? ps : 1;
    for (int r0 = 0; r0 < ns; r0 += kThreads) {
        const int nr = min(kThreads, ns - r0);
        if (h2) {
            __syncthreads();
            for (int e = threadIdx.x; e < nr * d * ps; e += blockDim.x)
                su[e] = v.U[(long long)(row0 + r0) * d * ps + e];
            __syncthreads();
        }
        for (int it = threadIdx.x; it < nr * CQ; it += blockDim.x) {
            const int i = r0 + it / CQ, cq = it % CQ;
            const long long row = row0 + i;
            T acc[CT];
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[c] = T(0);
            for (int q = v.items_by_leaf[leaf]; q < v.items_by_leaf[leaf + 1]; ++q) {
                T x[CT];
                load_ct<T, CT>(v.partials + ((long long)q * v.part_stride + i) * S + c0 + cq * CT, x);
#pragma unroll
                for (int c = 0; c < CT; ++c) acc[c] += x[c];
            }
            for (int q = v.mirror_by_leaf[leaf]; q < v.mirror_by_leaf[leaf + 1]; ++q) {  // D_st^T x_s
                T x[CT];
                load_ct<T, CT>(v.partials + ((long long)(v.n_items + q) * v.part_stride + i) * S + c0 + cq * CT, x);
#pragma unroll
                for (int c = 0; c < CT; ++c) acc[c] += x[c];
            }
            if (h2) {
                const T* u = su + (it / CQ) * d * ps;
                int I = 0;
                for (int i3 = 0; i3 < p3; ++i3) {
                    const T w3 = d > 2 ? u[2 * ps + i3] : T(1);
                    for (int i2 = 0; i2 < p2; ++i2) {
                        const T w23 = d > 1 ? w3 * u[ps + i2] : w3;
                        for (int i1 = 0; i1 < p1; ++i1, ++I) {
                            const T w = w23 * u[i1];
                            T yv[CT];
                            load_ct<T, CT>(sy + I * MC + cq * CT, yv);
#pragma unroll
                            for (int c = 0; c < CT; ++c) acc[c] += w * yv[c];
                        }
                    }
                }
            } else {
                for (int sl = 0; sl < v.n_far_levels; ++sl)
#pragma unroll
                    for (int c = 0; c < CT; ++c) acc[c] += v.yfar[((long long)sl * v.n + row) * S + c0 + cq * CT + c];
            }
            const int orig = v.perm[row];
#pragma unroll
            for (int c = 0; c < CT; ++c)
                if (c0 + cq * CT + c < m) Y[orig + (long long)(c0 + cq * CT + c) * ldy] = acc[c];
        }
    }
}

// Y[perm[i] + c ldy] = sum of the leaf's near partials + (U_s yhat_s)[i][c] for the H^2 format,
// register-tiled (MC a multiple of 4, d = 2 or 3): yhat_s first receives its parent's share
// (E_{s,d} (x) .. (x) E_{s,1}) yhat_parent (last level of Alg. FastBackward) as in
// combine_kernel; then thread (row i, part) sums U_s[i][I] yhat_s[I][0..MC) over the I whose
// outermost index falls in its part (two parts, combined in shared memory), with
// U_s[i][I] = prod_k U_{s,k}[i][i_k] formed on the fly and yhat_s read as broadcast vectors.
// One CTA per leaf, rows in passes of 128.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) combine_tiled_kernel(DevView<T> v, T* __restrict__ Y, long long ldy,
                                                                 int m, int S, int c0, int pull_level) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int RB = kThreads / 2;
    const int ps = v.p_s, d = v.d, PD = v.PD;
    const int US = d * ps + 1;                              // padded factor row (bank spread)
    T* sy = reinterpret_cast<T*>(smem_raw);                 // PD x MC
    T* sE = sy + (size_t)PD * MC;                           // 2 p^2 (padded to 4)
    T* b0 = sE + ((2 * ps * ps + 3) & ~3);                  // PD x MC (pull scratch)
    T* b1 = b0 + (size_t)PD * MC;                           // PD x MC
    T* su = b0;                                             // RB x US (reuses the pull scratch)
    T* red = su + (((size_t)RB * US + 3) & ~(size_t)3);     // RB x MC
    const int leaf = blockIdx.x;
    const int node = v.leaf_node[leaf];
    const int row0 = v.node_begin[node], ns = v.node_end[node] - row0;
    const int parent = v.node_parent[node];
    const bool pull = parent >= 0 && v.node_level[parent] >= pull_level;
    if (S == MC) {
        block_copy(sy, v.yhat + (long long)node * PD * S, PD * MC);
        if (pull) block_copy(b0, v.yhat + (long long)parent * PD * S, PD * MC);
    } else {
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            sy[e] = v.yhat[((long long)node * PD + e / MC) * S + c0 + e % MC];
        if (pull)
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
                b0[e] = v.yhat[((long long)parent * PD + e / MC) * S + c0 + e % MC];
    }
    if (pull) {
        for (int e = threadIdx.x; e < 2 * ps * ps; e += blockDim.x) sE[e] = v.E[e];
        const int halves = v.node_halves[node];
        T* in = b0;
        T* out = b1;
        int stride = 1;
        for (int k = 0; k < d; ++k) {
            __syncthreads();
            const bool last = (k == d - 1);
            mode_product<T, MC>(in, last ? sy : out, sE + ((halves >> k) & 1) * ps * ps, ps, PD, stride, false, last);
            T* t = in; in = out; out = t;
            stride *= ps;
        }
    }
    const int r = threadIdx.x % RB, part = threadIdx.x / RB;
    const int outer0 = part * (ps / 2), outer1 = part == 0 ? ps / 2 : ps;  // outermost index range
    const int mid = (d == 3) ? ps : 1;
    for (int p0 = 0; p0 < ns; p0 += RB) {
        const int nr = min(RB, ns - p0);
        __syncthreads();  // sy complete; su / red free
        for (int e = threadIdx.x; e < nr * d * ps; e += blockDim.x)
            su[(e / (d * ps)) * US + e % (d * ps)] = v.U[(long long)(row0 + p0) * d * ps + e];
        __syncthreads();
        T acc[MC];
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[c] = T(0);
        if (r < nr) {
            const T* u = su + r * US;
            for (int o = outer0; o < outer1; ++o) {
                const T wo = u[(d - 1) * ps + o];
                for (int i2 = 0; i2 < mid; ++i2) {
                    const T wm = (d == 3) ? wo * u[ps + i2] : wo;
                    const int Ib = ((d == 3) ? (o * ps + i2) : o) * ps;
                    for (int i1 = 0; i1 < ps; ++i1) {
                        const T w = wm * u[i1];
                        const T* yv = sy + (size_t)(Ib + i1) * MC;
#pragma unroll
                        for (int c = 0; c < MC; c += 4) {
                            T y4[4];
                            load_ct<T, 4>(yv + c, y4);
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[c + e] += w * y4[e];
                        }
                    }
                }
            }
        }
        if (part == 1) {
#pragma unroll
            for (int c = 0; c < MC; ++c) red[r * MC + c] = acc[c];
        }
        __syncthreads();
        if (part == 0 && r < nr) {
            const int i = p0 + r;
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[c] += red[r * MC + c];
            // the leaf's near item slots, then its mirror slots (D_st^T x_s)
            const int nq = v.items_by_leaf[leaf + 1] - v.items_by_leaf[leaf];
            const int nqm = v.mirror_by_leaf[leaf + 1] - v.mirror_by_leaf[leaf];
            for (int u = 0; u < nq + nqm; ++u) {
                const long long q = u < nq ? v.items_by_leaf[leaf] + u : v.n_items + v.mirror_by_leaf[leaf] + (u - nq);
                const T* pp = v.partials + (q * v.part_stride + i) * S + c0;
#pragma unroll
                for (int c = 0; c < MC; c += 4) {
                    T x[4];
                    load_ct<T, 4>(pp + c, x);
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[c + e] += x[e];
                }
            }
            const int orig = v.perm[row0 + i];
#pragma unroll
            for (int c = 0; c < MC; ++c)
                if (c0 + c < m) Y[orig + (long long)(c0 + c) * ldy] = acc[c];
        }
    }
}

int pick_mc(int m) {
    if (m <= 1) return 1;
    if (m <= 2) return 2;
    if (m <= 4) return 4;
    if (m <= 8) return 8;
    return 16;
}

// Explicit coupling, phase 2: yhat_s += sum_b L_k z_b (§4.5; L_k from the left cores, App. A.4),
// bulk-copy pipelined (one chunk of MC right-hand sides with S == MC,
// PD rows covered by one pass of 8-row x 4-column thread tiles).  CTA = (target s, part): as
// coupling_b_kernel, but a producer warp streams, for each far block b of the part, z_b (into one
// of NS small buffers) and L_k in chunks of whole columns (contiguous: [q PD + I]) by bulk copies
// into a ring of NS stages; the consumer warps take L_k from shared memory and release stages
// through per-warp mbarrier arrivals.  Every wait is bounded (timeouts counted in flags[1]).
namespace cb1 {
constexpr int NS = 4;
constexpr int STAGE = 16384;     // bytes of L_k per stage
constexpr int STB = STAGE + 32;  // plus the 16-byte rounding of a chunk's start and end
}  // namespace cb1

template <typename T>
__device__ __forceinline__ int coupling_chunk_cols(int PD) {
    const int Q = cb1::STAGE / (PD * (int)sizeof(T));
    return Q < 1 ? 1 : Q;
}

template <typename T, int MC>
__global__ void __launch_bounds__(kThreads + 32, 2) coupling_b_tma_kernel(DevView<T> v, int nsplit) {
    using namespace cb1;
    constexpr int CT = 4, CQ = MC / CT, RPT = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* stg = smem_raw;                                // NS x STB
    T* zbufs = reinterpret_cast<T*>(smem_raw + NS * STB);         // NS x zstride x MC
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int PD = v.PD, zst = v.zstride;
    const int ti = blockIdx.x / nsplit, part = blockIdx.x % nsplit;
    const int s = v.far_targets[ti];
    const int fb0 = v.far_by_target[ti], fb1 = v.far_by_target[ti + 1];
    const int per = (fb1 - fb0 + nsplit - 1) / nsplit;
    const int my0 = fb0 + part * per, my1 = min(fb1, my0 + per);
    if (my0 >= my1) return;
    const int Q = coupling_chunk_cols<T>(PD);
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kThreads / 32);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kThreads / 32) {
        if (lane == 0) {
            int t = 0;
            bool ok = true;
            for (int fb = my0; fb < my1 && ok; ++fb) {
                const int key = v.fb_key[fb];
                const int rd = v.key_ranks[(size_t)key * (v.Delta + 1) + v.d];
                const T* Lt = v.far_lr + v.key_lroff[key];
                for (int q0 = 0; q0 < rd; q0 += Q, ++t) {
                    const int st = t % NS;
                    if (t >= NS) ok = mbar_wait(&empty[st], (uint32_t)(((t / NS) - 1) & 1));
                    if (!ok || *(volatile int*)&abort_flag) {
                        ok = false;
                        break;
                    }
                    const int qn = min(Q, rd - q0);
                    const uintptr_t a0 = (uintptr_t)(Lt + (long long)q0 * PD);
                    const uintptr_t a1 = a0 + (uintptr_t)qn * PD * sizeof(T);
                    const uintptr_t s0 = a0 & ~(uintptr_t)15, e0 = (a1 + 15) & ~(uintptr_t)15;
                    const uint32_t bytes = (uint32_t)(e0 - s0);
                    const uint32_t zbytes = (q0 == 0) ? (uint32_t)(rd * MC * sizeof(T)) : 0u;
                    mbar_expect_tx(&full[st], bytes + zbytes);
                    bulk_g2s(stg + st * STB, (const void*)s0, bytes, &full[st]);
                    if (zbytes)
                        bulk_g2s(zbufs + (size_t)((fb - my0) % NS) * zst * MC, v.zbuf + (long long)fb * zst * MC, zbytes,
                                 &full[st]);
                }
            }
            if (!ok) {
                atomicAdd(v.flags + 1, 1);
                abort_flag = 1;
            }
            for (int u = max(0, t - NS); u < t; ++u) mbar_wait(&full[u % NS], (uint32_t)((u / NS) & 1));
        }
        return;
    }

    // consumer warps: thread = 8 consecutive rows I0.. of yhat_s x 4 right-hand sides
    const int cq = tid % CQ, rg = tid / CQ;
    const int I0 = rg * RPT;
    const bool active = I0 < PD;
    T acc[RPT][CT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[i][c] = T(0);
    bool ok = true;
    int t = 0;
    for (int fb = my0; fb < my1 && ok; ++fb) {
        const int key = v.fb_key[fb];
        const int rd = v.key_ranks[(size_t)key * (v.Delta + 1) + v.d];
        const T* Lt = v.far_lr + v.key_lroff[key];
        const T* zb = zbufs + (size_t)((fb - my0) % NS) * zst * MC;
        for (int q0 = 0; q0 < rd; q0 += Q, ++t) {
            const int st = t % NS;
            ok = mbar_wait(&full[st], (uint32_t)((t / NS) & 1)) && !*(volatile int*)&abort_flag;
            if (!ok) break;
            const int qn = min(Q, rd - q0);
            const uintptr_t a0 = (uintptr_t)(Lt + (long long)q0 * PD);
            const T* Ls = reinterpret_cast<const T*>(stg + st * STB + (a0 & 15)) + I0;
            if (active) {
                for (int qq = 0; qq < qn; qq += 8) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int q = qq + u;
                        if (q < qn) {
                            T l[RPT], x[CT];
                            if ((a0 & 15) == 0) {
                                load_ct<T, 4>(Ls + q * PD, *reinterpret_cast<T(*)[4]>(&l[0]));
                                load_ct<T, 4>(Ls + q * PD + 4, *reinterpret_cast<T(*)[4]>(&l[4]));
                            } else {
#pragma unroll
                                for (int i = 0; i < RPT; ++i) l[i] = Ls[q * PD + i];
                            }
                            load_ct<T, CT>(zb + (q0 + q) * MC + cq * CT, x);
#pragma unroll
                            for (int i = 0; i < RPT; i += 2)
#pragma unroll
                                for (int c = 0; c < CT; ++c) fma_pair(acc[i][c], acc[i + 1][c], l[i], l[i + 1], x[c], x[c]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[st])) : "memory");
        }
    }
    if (!ok) {
        if (lane == 0) atomicExch(&abort_flag, 1);
        return;
    }
    if (active) {
        T* dst = v.yhat + (long long)s * PD * MC;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            T* o = dst + (long long)(I0 + i) * MC + cq * CT;
            if (nsplit > 1) atomic_add_ct<T, CT>(o, acc[i]);
            else store_ct<T, CT>(o, acc[i]);
        }
    }
}

// Mirror products for the register-staged near field (mirror sharing, near_kernel): the block
// (t, s) of a stored block (s, t), s != t, is D_st^T, so its contribution (D_st^T x_s) goes to the
// block's mirror slot, which combine_kernel adds to leaf t.  One CTA per mirror slot; thread j
// owns column j of D_st: out[j][c] = sum_i (sum_k w_k G_{b,1}[(j r + k) n_s + i]) x_s[i][c],
// reading its column of every slab as one contiguous run.  (The bulk-copy near kernel forms these
// products from the same read of G_{b,1} as the forward ones.)
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) near_mirror_kernel(DevView<T> v, int S, int c0, int maxleaf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xsm = reinterpret_cast<T*>(smem_raw);  // n_s x MC
    T* sw = xsm + (size_t)maxleaf * MC;       // r
    const int q = blockIdx.x;
    const int b = v.mslot_block[q];
    const int snode = v.nb_s[b], tnode = v.nb_t[b];
    const int sb = v.node_begin[snode], ns = v.node_end[snode] - sb;
    const int nt = v.node_end[tnode] - v.node_begin[tnode];
    const int r = v.nb_rank[b];
    for (int e = threadIdx.x; e < ns * MC; e += blockDim.x) xsm[e] = v.Xc[(long long)(sb + e / MC) * S + c0 + e % MC];
    for (int k = threadIdx.x; k < r; k += blockDim.x) sw[k] = v.w[v.nb_woff[b] + k];
    __syncthreads();
    T* dst = v.partials + (long long)(v.n_items + q) * v.part_stride * S + c0;
    const T* G = v.near_cores + v.nb_off[b];
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        T acc[MC];
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[c] = T(0);
        const T* gj = G + (long long)j * r * ns;
        for (int i = 0; i < ns; ++i) {
            T dij = T(0);
            for (int k = 0; k < r; ++k) dij += sw[k] * __ldg(gj + (long long)k * ns + i);
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[c] += dij * xsm[i * MC + c];
        }
#pragma unroll
        for (int c = 0; c < MC; ++c) dst[(long long)j * S + c] = acc[c];
    }
}

// Adjoint near field: Xbar_t += D_b(theta)^T Ybar_s for every stored near block b = (s, t)
// (§4.3 blocks, transposed), accumulated into the first partial slot of the source leaf t (the
// other slots of t are zero), so that combine_kernel adds it like a forward near partial.  One CTA
// per block; thread j owns column j of D_b: out[j][c] = sum_i (sum_k w_k G_{b,1}[(j r + k) n_s + i])
// Ybar_s[i][c], reading its column of every slab as one contiguous run.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) near_adjoint_kernel(DevView<T> v, int S, int c0, int maxleaf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ys = reinterpret_cast<T*>(smem_raw);  // n_s x MC
    T* sw = ys + (size_t)maxleaf * MC;       // r
    const int b = blockIdx.x;
    const int snode = v.nb_s[b], tnode = v.nb_t[b];
    const int sb = v.node_begin[snode], ns = v.node_end[snode] - sb;
    const int tb = v.node_begin[tnode], nt = v.node_end[tnode] - tb;
    const int r = v.nb_rank[b];
    for (int e = threadIdx.x; e < ns * MC; e += blockDim.x) ys[e] = v.Xc[(long long)(sb + e / MC) * S + c0 + e % MC];
    for (int k = threadIdx.x; k < r; k += blockDim.x) sw[k] = v.w[v.nb_woff[b] + k];
    __syncthreads();
    const int tleaf = v.node_leaf[tnode];
    T* dst = v.partials + (long long)v.items_by_leaf[tleaf] * v.part_stride * S + c0;
    const T* G = v.near_cores + v.nb_off[b];
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        T acc[MC];
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[c] = T(0);
        const T* gj = G + (long long)j * r * ns;
        for (int i = 0; i < ns; ++i) {
            T dij = T(0);
            for (int k = 0; k < r; ++k) dij += sw[k] * __ldg(gj + (long long)k * ns + i);
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[c] += dij * ys[i * MC + c];
        }
        T* o = dst + (long long)j * S;
        constexpr int CT = MC < 4 ? MC : 4;
#pragma unroll
        for (int c = 0; c < MC; c += CT) atomic_add_ct<T, CT>(o + c, *reinterpret_cast<T(*)[CT]>(&acc[c]));
    }
}

// H_k^T of every class into HT at the offsets of H (for an adjoint set up after instantiation).
template <typename T>
__global__ void transpose_H_kernel(DevView<T> v, T* HT) {
    const int key = blockIdx.x;
    const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
    const int ra = rk[v.d], rb = rk[v.d + v.dtheta];
    const long long off = v.key_hoff[key];
    for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) HT[off + e / ra + (long long)rb * (e % ra)] = v.H[off + e];
}

template <typename T, int MC>
void set_smem(const void* fn, size_t bytes) {
    PH_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <typename T, int MC>
void run_matvec(ph_handle* h, DevView<T>& v, const T* X, long long ldx, int m, T* Y, long long ldy,
                cudaStream_t stream, int S, bool adj) {
    const Plan& plan = h->plan;
    const int nleaves = (int)plan.leaves.size();
    int maxleaf = 1;
    for (int l : plan.leaves) maxleaf = std::max(maxleaf, plan.nodes[l].size());
    const bool h2 = (h->opts.fmt == PH_FMT_H2);
    const int PD = v.PD;
    h->last_variants = 0;
    // fork: the far path runs on the side stream, concurrently with the near field
    cudaStream_t far = h->overlap ? h->side : stream;
    if (h->overlap) {
        PH_CUDA(cudaEventRecord(h->ev_fork, stream));
        PH_CUDA(cudaStreamWaitEvent(far, h->ev_fork, 0));
    }
    // bulk-copy pipelined near field when one chunk of right-hand sides covers X (rows of x_t
    // contiguous), rows are 16-byte multiples, leaves fit one CTA and a column of cores fits a stage
    const size_t sm_ntma = near_tma_smem<T>(maxleaf, MC, v.near_share != 0);
    const bool near_tma = h->use_bulk && S == MC && (MC * sizeof(T)) % 16 == 0 && maxleaf <= kThreads &&
                          (size_t)h->near_rank_max * maxleaf * sizeof(T) <= (size_t)nt1::STAGE &&
                          sm_ntma <= 110 * 1024 && v.n_items > 0;
    // with mirror sharing the stored near part is symmetric (each pair applied as D and D^T): the
    // adjoint's near field is the forward one
    const bool near_adj = adj && !v.near_share;
    if (near_adj && v.n_near > 0) {
        // adjoint near field: transposed blocks accumulated into zeroed partial slots
        PH_CUDA(cudaMemsetAsync(v.partials, 0, (size_t)std::max(1, v.n_items) * v.part_stride * S * sizeof(T), stream));
        const size_t smem = ((size_t)maxleaf * MC + kMaxNearRank) * sizeof(T);
        set_smem<T, MC>((const void*)near_adjoint_kernel<T, MC>, smem);
        for (int c0 = 0; c0 < S; c0 += MC) {
            ProfScope ps(h, 2, stream);
            near_adjoint_kernel<T, MC><<<v.n_near, kThreads, smem, stream>>>(v, S, c0, maxleaf);
            PH_LAUNCH("near_adjoint_kernel");
        }
    }
    for (int c0 = 0; c0 < S && !near_adj; c0 += MC) {
        ProfScope ps(h, 2, stream);
        if (near_tma) {
            h->last_variants |= 1;
            set_smem<T, MC>((const void*)near_tma_kernel<T, MC>, sm_ntma);
            near_tma_kernel<T, MC><<<v.n_items, kThreads + 32, sm_ntma, stream>>>(v, maxleaf);
            PH_LAUNCH("near_tma_kernel");
        } else {
            size_t smem = ((size_t)maxleaf * MC + (size_t)kThreads * MC + kMaxNearRank) * sizeof(T);
            set_smem<T, MC>((const void*)near_kernel<T, MC>, smem);
            near_kernel<T, MC><<<std::max(1, v.n_items), kThreads, smem, stream>>>(v, S, c0, maxleaf);
            PH_LAUNCH("near_kernel");
            if (v.n_mslots > 0) {
                const size_t sm_m = ((size_t)maxleaf * MC + kMaxNearRank) * sizeof(T);
                set_smem<T, MC>((const void*)near_mirror_kernel<T, MC>, sm_m);
                near_mirror_kernel<T, MC><<<v.n_mslots, kThreads, sm_m, stream>>>(v, S, c0, maxleaf);
                PH_LAUNCH("near_mirror_kernel");
            }
        }
    }
    if (v.n_far_targets > 0) {
        for (int c0 = 0; c0 < S; c0 += MC) {
            if (h2) {
                PH_CUDA(cudaMemsetAsync(v.xhat, 0, (size_t)v.n_nodes * PD * S * sizeof(T), far));
                // register-tiled leaf kernel when p_s is a multiple of 4 and p_s^d / 4 divides the CTA
                const int nt4 = PD / 4;
                const bool tiled = (v.p_s % 4 == 0) && nt4 >= 1 && nt4 <= kThreads && kThreads % nt4 == 0;
                const size_t sm_tiled = ((size_t)64 * v.d * v.p_s + 64 * MC + (size_t)(kThreads / std::max(1, nt4)) * PD * MC +
                                         (size_t)PD * MC + 2 * v.p_s * v.p_s) * sizeof(T);
                if (tiled && sm_tiled <= 200 * 1024) {
                    set_smem<T, MC>((const void*)upsweep_leaf_tiled_kernel<T, MC>, sm_tiled);
                    ProfScope ps(h, 3, far);
                    upsweep_leaf_tiled_kernel<T, MC><<<nleaves, kThreads, sm_tiled, far>>>(v, S, c0, h->min_far_level);
                } else {
                    size_t sm_leaf = ((size_t)32 * kMaxDim * kMaxPs + 32 * MC + ((2 * v.p_s * v.p_s + 3) & ~3) +
                                      2 * (size_t)PD * MC) * sizeof(T);
                    set_smem<T, MC>((const void*)upsweep_leaf_kernel<T, MC>, sm_leaf);
                    ProfScope ps(h, 3, far);
                    upsweep_leaf_kernel<T, MC><<<nleaves, kThreads, sm_leaf, far>>>(v, S, c0, h->min_far_level);
                }
                PH_LAUNCH("upsweep_leaf_kernel");
                size_t sm_tr = ((size_t)((2 * v.p_s * v.p_s + 3) & ~3) + 3 * (size_t)PD * MC) * sizeof(T);
                set_smem<T, MC>((const void*)transfer_kernel<T, MC>, sm_tr);
                for (int l = plan.depth - 1; l >= h->min_far_level; --l) {
                    if (!h->level_has_inner_child[l]) continue;
                    int cnt = h->level_nodes_off[l + 1] - h->level_nodes_off[l];
                    if (cnt == 0) continue;
                    ProfScope ps(h, 4, far);
                    transfer_kernel<T, MC><<<cnt, kThreads, sm_tr, far>>>(
                        v, h->d_level_nodes + h->level_nodes_off[l], S, c0, true, v.xhat, v.xhat);
                    PH_LAUNCH("transfer_kernel(up)");
                }
                if (h->opts.coupling == 0) {
                    {
                        ProfScope ps(h, 5, far);
                        const bool staged = (MC >= 4) && (PD % 32 == 0) && (h->rank_max_lr <= 64);
                        const bool tc = std::is_same<T, float>::value && MC == 16 && h->tc_elems > 0 &&
                                        (PD % 32 == 0) && (h->rank_max_lr <= 64) && h->use_tc && v.n_tcitems > 0;
                        bool launched = false;
                        if constexpr (std::is_same<T, float>::value && MC == 16) {
                            if (tc && S == 16) {
                                PH_CUDA(cudaFuncSetAttribute(coupling_a_umma_kernel,
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, tc2::SMEM));
                                const int grid = std::min(v.n_tcitems, h->num_sms);
                                coupling_a_umma_kernel<<<grid, tc2::THREADS, tc2::SMEM, far>>>(v);
                                h->last_variants |= 4;
                                launched = true;
                            }
                        }
                        if (launched) {
                        } else if (staged) {
                            if constexpr (MC >= 4) {  // staged needs MC >= 4; no instances below that
                                size_t sm_a = ((size_t)2 * 32 * 64 + 2 * 32 * 260) * sizeof(T);
                                set_smem<T, MC>((const void*)coupling_a_staged_kernel<T, MC>, sm_a);
                                coupling_a_staged_kernel<T, MC><<<std::max(1, v.n_citems), kThreads, sm_a, far>>>(
                                    v, S, c0);
                            }
                        } else {
                            size_t sm_a = ((size_t)64 * 33 + 32 * 68 + 64 * 68) * sizeof(T);
                            set_smem<T, MC>((const void*)coupling_a_kernel<T, MC>, sm_a);
                            coupling_a_kernel<T, MC><<<std::max(1, v.n_citems), kThreads, sm_a, far>>>(v, S, c0);
                        }
                        PH_LAUNCH("coupling_a_kernel");
                    }
                    {
                        ProfScope ps(h, 9, far);
                        constexpr int CQB = (MC < 4) ? 1 : MC / 4;
                        const int itemsb = ((PD + 7) / 8) * CQB;
                        const int nib = (itemsb + kThreads - 1) / kThreads;
                        const int nsplit = 4;
                        size_t sm_b = (size_t)8 * v.zstride * MC * sizeof(T);
                        const int nt = v.n_far_targets * nsplit;
                        const size_t sm_btma = (size_t)cb1::NS * cb1::STB + (size_t)cb1::NS * v.zstride * MC * sizeof(T);
                        const bool b_tma = h->use_bulk && S == MC && MC >= 4 && (MC * sizeof(T)) % 16 == 0 &&
                                           PD % 8 == 0 && itemsb <= kThreads &&
                                           (size_t)PD * sizeof(T) <= (size_t)cb1::STAGE && sm_btma <= 110 * 1024;
                        bool b_done = false;
                        if constexpr (MC >= 4) {  // b_tma needs MC >= 4; no instances below that
                            if (b_tma) {
                                const int nsp = 2;
                                set_smem<T, MC>((const void*)coupling_b_tma_kernel<T, MC>, sm_btma);
                                coupling_b_tma_kernel<T, MC><<<v.n_far_targets * nsp, kThreads + 32,
                                                               sm_btma, far>>>(v, nsp);
                                h->last_variants |= 2;
                                b_done = true;
                            }
                        }
                        if (b_done) {
                        } else if (nib <= 1) {
                            set_smem<T, MC>((const void*)coupling_b_kernel<T, MC, 1>, sm_b);
                            coupling_b_kernel<T, MC, 1><<<nt, kThreads, sm_b, far>>>(v, S, c0, nsplit);
                        } else if (nib <= 2) {
                            set_smem<T, MC>((const void*)coupling_b_kernel<T, MC, 2>, sm_b);
                            coupling_b_kernel<T, MC, 2><<<nt, kThreads, sm_b, far>>>(v, S, c0, nsplit);
                        } else if (nib <= 4) {
                            set_smem<T, MC>((const void*)coupling_b_kernel<T, MC, 4>, sm_b);
                            coupling_b_kernel<T, MC, 4><<<nt, kThreads, sm_b, far>>>(v, S, c0, nsplit);
                        } else {
                            throw Error(PH_ERR_UNSUPPORTED, "p_s^d too large for the coupling kernel");
                        }
                        PH_LAUNCH("coupling_b_kernel");
                    }
                } else {
                    const int zmax = h->coupling_zmax;
                    size_t sm_c = 2 * (size_t)zmax * ChainRow<MC>::value * sizeof(T);
                    const int CQ = MC < 4 ? 1 : MC / 4;
                    const int items_last = ((v.p_s + 3) / 4) * (PD / v.p_s) * CQ;
                    const int ni = (items_last + kThreads - 1) / kThreads;
                    const int nsplit = 4;
                    {
                        ProfScope ps(h, 5, far);
                        const int nt = v.n_far_targets * nsplit;
                        if (ni <= 1) {
                            set_smem<T, MC>((const void*)coupling_kernel<T, MC, 1>, sm_c);
                            coupling_kernel<T, MC, 1><<<nt, kThreads, sm_c, far>>>(v, S, c0, zmax, nsplit);
                        } else if (ni <= 2) {
                            set_smem<T, MC>((const void*)coupling_kernel<T, MC, 2>, sm_c);
                            coupling_kernel<T, MC, 2><<<nt, kThreads, sm_c, far>>>(v, S, c0, zmax, nsplit);
                        } else if (ni <= 4) {
                            set_smem<T, MC>((const void*)coupling_kernel<T, MC, 4>, sm_c);
                            coupling_kernel<T, MC, 4><<<nt, kThreads, sm_c, far>>>(v, S, c0, zmax, nsplit);
                        } else {
                            throw Error(PH_ERR_UNSUPPORTED, "p_s^d too large for the coupling kernel");
                        }
                    }
                    PH_LAUNCH("coupling_kernel");
                }
                for (int l = h->min_far_level; l < plan.depth; ++l) {
                    if (!h->level_has_inner_child[l]) continue;
                    int cnt = h->level_nodes_off[l + 1] - h->level_nodes_off[l];
                    if (cnt == 0) continue;
                    ProfScope ps(h, 6, far);
                    transfer_kernel<T, MC><<<cnt, kThreads, sm_tr, far>>>(
                        v, h->d_level_nodes + h->level_nodes_off[l], S, c0, false, v.yhat, v.yhat);
                    PH_LAUNCH("transfer_kernel(down)");
                }
            } else {
                int maxnode = v.far_max_target, rmax = 1;
                for (size_t key = 0; key < plan.key_rep.size(); ++key) {
                    const int* rk = &h->key_ranks[key * (h->Delta + 1)];
                    rmax = std::max(rmax, std::max(rk[v.d], rk[v.d + v.dtheta]));
                }
                size_t sm_h = ((size_t)maxnode * MC + 2 * (size_t)rmax * MC) * sizeof(T);
                set_smem<T, MC>((const void*)far_h_kernel<T, MC>, sm_h);
                ProfScope ps(h, 7, far);
                far_h_kernel<T, MC><<<v.n_far_targets, kThreads, sm_h, far>>>(v, S, c0, rmax);
                PH_LAUNCH("far_h_kernel");
            }
        }
    }
    if (h->overlap) {
        PH_CUDA(cudaEventRecord(h->ev_join, far));
        PH_CUDA(cudaStreamWaitEvent(stream, h->ev_join, 0));
    }
    for (int c0 = 0; c0 < S; c0 += MC) {
        const bool h2far = h2 && v.n_far_targets > 0;
        const int RB = kThreads / 2;
        const size_t sm_t = ((size_t)PD * MC + ((2 * v.p_s * v.p_s + 3) & ~3) +
                             std::max((size_t)2 * PD * MC, (((size_t)RB * (v.d * v.p_s + 1) + 3) & ~(size_t)3) +
                                                               (size_t)RB * MC)) * sizeof(T);
        ProfScope ps(h, 8, stream);
        if (h2far && MC >= 4 && (v.d == 2 || v.d == 3) && v.p_s % 2 == 0 && sm_t <= 200 * 1024) {
            if constexpr (MC >= 4) {
                set_smem<T, MC>((const void*)combine_tiled_kernel<T, MC>, sm_t);
                combine_tiled_kernel<T, MC><<<nleaves, kThreads, sm_t, stream>>>(v, Y, ldy, m, S, c0,
                                                                                 h->min_far_level);
            }
        } else {
            size_t sm = ((size_t)PD * MC + std::max((size_t)2 * PD * MC + ((2 * v.p_s * v.p_s + 3) & ~3),
                                                    (size_t)kThreads * v.d * v.p_s)) * sizeof(T);
            set_smem<T, MC>((const void*)combine_kernel<T, MC>, sm);
            combine_kernel<T, MC><<<nleaves, kThreads, sm, stream>>>(v, Y, ldy, m, S, c0, h2far ? 1 : 0,
                                                                     h->min_far_level);
        }
        PH_LAUNCH("combine_kernel");
    }
}

template <typename T>
ph_status matvec_typed(ph_handle* h, DevView<T>& v, const T* X, long long ldx, int m, T* Y, long long ldy,
                       cudaStream_t stream, bool adj = false) {
    const int MC = pick_mc(m);
    const int S = (int)ceil_div(m, MC) * MC;
    const bool h2 = (h->opts.fmt == PH_FMT_H2);
    const int check = h->opts.check_finite ? 1 : 0;
    if (check) PH_CUDA(cudaMemsetAsync(v.flags, 0, sizeof(int), stream));  // flags[1] counts on
    const long long total = (long long)v.n * S;
    int grid = (int)std::min<long long>(ceil_div(total, kThreads), 152 * 16);
    {
        ProfScope ps(h, 1, stream);
        gather_kernel<T><<<grid, kThreads, 0, stream>>>(v, X, ldx, m, S, check);
        PH_LAUNCH("gather_kernel");
    }
    if (h2 && v.n_far_targets > 0)
        PH_CUDA(cudaMemsetAsync(v.yhat, 0, (size_t)v.n_nodes * v.PD * S * sizeof(T), stream));
    if (!h2 && v.n_far_levels > 0)
        PH_CUDA(cudaMemsetAsync(v.yfar, 0, (size_t)v.n_far_levels * v.n * S * sizeof(T), stream));
    switch (MC) {
        case 1: run_matvec<T, 1>(h, v, X, ldx, m, Y, ldy, stream, S, adj); break;
        case 2: run_matvec<T, 2>(h, v, X, ldx, m, Y, ldy, stream, S, adj); break;
        case 4: run_matvec<T, 4>(h, v, X, ldx, m, Y, ldy, stream, S, adj); break;
        case 8: run_matvec<T, 8>(h, v, X, ldx, m, Y, ldy, stream, S, adj); break;
        default: run_matvec<T, 16>(h, v, X, ldx, m, Y, ldy, stream, S, adj); break;
    }
    post_timeout_flag(h, stream);
    if (check) {
        int bad[2] = {0, 0};
        PH_CUDA(cudaMemcpyAsync(bad, v.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
        PH_CUDA(cudaStreamSynchronize(stream));
        if (bad[0]) throw Error(PH_ERR_NONFINITE, "X has non-finite entries");
        if (bad[1] > h->seen_timeouts) {
            h->seen_timeouts = bad[1];
            throw Error(PH_ERR_TIMEOUT, "a bounded device-side wait ran out");
        }
    }
    return PH_OK;
}

template <typename T>
void instantiate_typed(ph_handle* h, DevView<T>& v, const double* theta, int deriv, cudaStream_t stream,
                       bool far = true) {
    const int near_ctas = (int)ceil_div(std::max(v.n_near, 1), kThreads);
    const int grid = near_ctas + (far ? v.n_keys : 0);
    double th[3] = {0, 0, 0};
    for (int k = 0; k < h->opts.dtheta; ++k) th[k] = theta[k];
    ProfScope ps(h, 0, stream);
    const size_t dsm = (h->opts.dtheta > 1 && v.n_keys > 0) ? (size_t)3 * 64 * 64 * sizeof(double) : 0;
    if (dsm) set_smem<T, 1>((const void*)instantiate_kernel<T>, dsm);
    instantiate_kernel<T><<<grid, kThreads, dsm, stream>>>(v, th[0], th[1], th[2], near_ctas, deriv);
    PH_LAUNCH("instantiate_kernel");
}

}  // namespace

static cudaEvent_t prof_event(ph_handle* h) {
    if (!h->prof_pool.empty()) {
        cudaEvent_t e = h->prof_pool.back();
        h->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    PH_CUDA(cudaEventCreate(&e));
    return e;
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

static const char* const kKindNames[PH_PROF_KINDS] = {"instantiate", "gather",        "near",  "upsweep_leaf",
                                                      "transfer_up", "coupling",      "transfer_down",
                                                      "far_h",       "combine",       "coupling_b"};

ProfScope::ProfScope(ph_handle* h_, int kind_, cudaStream_t s_) : h(h_), kind(kind_), s(s_) {
    nvtxRangePushA((kind >= 0 && kind < PH_PROF_KINDS) ? kKindNames[kind] : "libph");
    if (!h->prof) return;
    b = prof_event(h);
    PH_CUDA(cudaEventRecord(b, s));
}

ProfScope::~ProfScope() {
    if (b) {
        cudaEvent_t e = prof_event(h);
        cudaEventRecord(e, s);
        h->prof_recs.push_back({kind, b, e});
    }
    nvtxRangePop();
}

ph_status wait_bound_selftest(int device, double* waited) {
    int prev = 0;
    PH_CUDA(cudaGetDevice(&prev));
    PH_CUDA(cudaSetDevice(device));
    unsigned long long* d = nullptr;
    unsigned long long hres[2] = {1, 0};
    cudaError_t e = cudaMalloc(&d, sizeof(hres));
    if (e == cudaSuccess) {
        wait_bound_kernel<<<1, 32>>>(d);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(hres, d, sizeof(hres), cudaMemcpyDeviceToHost);
        cudaFree(d);
    }
    cudaSetDevice(prev);
    if (e != cudaSuccess) throw Error(PH_ERR_CUDA, std::string("wait_bound_kernel: ") + cudaGetErrorString(e));
    if (waited) *waited = (double)hres[1] * 1e-9;
    return hres[0] ? PH_OK : PH_ERR_TIMEOUT;
}

ph_status handle_timeout_selftest(ph_handle* h, cudaStream_t stream) {
    handle_timeout_kernel<<<1, 32, 0, stream>>>(h->d_flags);
    PH_LAUNCH("handle_timeout_kernel");
    post_timeout_flag(h, stream);
    return PH_OK;
}

ph_status online_instantiate(ph_handle* h, const double* theta, cudaStream_t stream, int deriv) {
    if (deriv < 0 && h->sur) {
        // the surrogate's cores when it is switched on (the derivative stays polynomial)
        online_instantiate_near(h, theta, stream);
        if (surrogate_instantiate_far(h, theta, stream)) return PH_OK;
    }
    if (h->opts.prec == PH_FP32) instantiate_typed<float>(h, h->vf, theta, deriv, stream);
    else instantiate_typed<double>(h, h->vd, theta, deriv, stream);
    return PH_OK;
}

void online_instantiate_near(ph_handle* h, const double* theta, cudaStream_t stream) {
    if (h->opts.prec == PH_FP32) instantiate_typed<float>(h, h->vf, theta, -1, stream, false);
    else instantiate_typed<double>(h, h->vd, theta, -1, stream, false);
}

ph_status online_matvec_view(ph_handle* h, DevView<float>& vf, DevView<double>& vd, const void* X, long ldx, int m,
                             void* Y, long ldy, cudaStream_t stream) {
    if (h->opts.prec == PH_FP32)
        return matvec_typed<float>(h, vf, (const float*)X, ldx, m, (float*)Y, ldy, stream);
    return matvec_typed<double>(h, vd, (const double*)X, ldx, m, (double*)Y, ldy, stream);
}

ph_status online_matvec_batched(ph_handle* h, const double* thetas, int n_theta, const void* X, long ldx, int m,
                                void* Y, long ldy, long stride_y, int deriv, cudaStream_t stream) {
    const int p = h->opts.degree[0] + 1;
    const size_t sc = h->scalar;
    // FP32 derivatives always take the direct route: the derivative weights alternate in sign and
    // grow like p^2 / (theta_hi - theta_lo), so combining FP32 node products would amplify their
    // rounding; the direct route cancels in FP64 inside the instantiation
    // (the node combination needs one theta grid for both fields)
    const bool one_grid = h->opts.near_degree[0] == 0 || h->opts.near_degree[0] == h->opts.degree[0];
    if (h->opts.dtheta != 1 || !one_grid || n_theta < p || (deriv >= 0 && h->opts.prec == PH_FP32)) {
        // one instantiation and product per theta
        for (int t = 0; t < n_theta; ++t) {
            online_instantiate(h, thetas + t, stream, deriv);
            online_matvec(h, X, ldx, m, (char*)Y + (size_t)t * stride_y * sc, ldy, stream);
        }
        return PH_OK;
    }
    const long n = h->plan.n;
    const size_t ybytes = (size_t)p * n * m * sc;
    if (ybytes > h->ynodes_bytes) {
        dev_free(h, h->d_ynodes);
        h->d_ynodes = dev_alloc(h, ybytes);
        h->ynodes_bytes = ybytes;
    }
    if ((size_t)n_theta > h->thetas_cap) {
        dev_free(h, h->d_thetas);
        h->d_thetas = (double*)dev_alloc(h, (size_t)n_theta * sizeof(double));
        h->thetas_cap = (size_t)n_theta;
    }
    for (int q = 0; q < p; ++q) {
        const double eta = h->theta_nodes[q];
        online_instantiate(h, &eta, stream, -1);
        online_matvec(h, X, ldx, m, (char*)h->d_ynodes + (size_t)q * n * m * sc, n, stream);
    }
    // pinned staging of the thetas: wait until the previous call's copy out of it has run, then
    // refill it and copy asynchronously
    if (h->ev_thetas) PH_CUDA(cudaEventSynchronize(h->ev_thetas));
    else PH_CUDA(cudaEventCreateWithFlags(&h->ev_thetas, cudaEventDisableTiming));
    if ((size_t)n_theta > h->host_thetas_cap) {
        if (h->host_thetas_pinned) PH_CUDA(cudaFreeHost(h->host_thetas_pinned));
        h->host_thetas_pinned = nullptr;
        h->host_thetas_cap = 0;
        PH_CUDA(cudaHostAlloc((void**)&h->host_thetas_pinned, (size_t)n_theta * sizeof(double), cudaHostAllocDefault));
        h->host_thetas_cap = (size_t)n_theta;
    }
    std::copy(thetas, thetas + n_theta, h->host_thetas_pinned);
    PH_CUDA(cudaMemcpyAsync(h->d_thetas, h->host_thetas_pinned, (size_t)n_theta * sizeof(double),
                            cudaMemcpyHostToDevice, stream));
    PH_CUDA(cudaEventRecord(h->ev_thetas, stream));
    const long long nel = (long long)n * m;
    dim3 grid((unsigned)std::max<long long>(1, std::min<long long>(ceil_div(nel, kThreads), (long long)h->num_sms * 4)),
              (unsigned)ceil_div(n_theta, 32));
    if (h->opts.prec == PH_FP32)
        node_combine_kernel<float><<<grid, kThreads, 0, stream>>>(h->vf, (const float*)h->d_ynodes, (int)n, m,
                                                                  h->d_thetas, n_theta, deriv, (float*)Y, ldy,
                                                                  stride_y);
    else
        node_combine_kernel<double><<<grid, kThreads, 0, stream>>>(h->vd, (const double*)h->d_ynodes, (int)n, m,
                                                                   h->d_thetas, n_theta, deriv, (double*)Y, ldy,
                                                                   stride_y);
    PH_LAUNCH("node_combine_kernel");
    return PH_OK;
}

void transpose_H(ph_handle* h, cudaStream_t stream) {
    const int nk = (int)h->plan.key_rep.size();
    if (nk == 0 || !h->d_HT) return;
    if (h->opts.prec == PH_FP32) transpose_H_kernel<float><<<nk, kThreads, 0, stream>>>(h->vf, (float*)h->d_HT);
    else transpose_H_kernel<double><<<nk, kThreads, 0, stream>>>(h->vd, (double*)h->d_HT);
    PH_LAUNCH("transpose_H_kernel");
}

ph_status online_matvec_transpose(ph_handle* h, const void* Y, long ldy, int m, void* X, long ldx,
                                  cudaStream_t stream) {
    build_adjoint(h, stream);
    ensure_workspace(h, m);
    if (h->opts.prec == PH_FP32)
        return matvec_typed<float>(h, h->vfT, (const float*)Y, ldy, m, (float*)X, ldx, stream, true);
    return matvec_typed<double>(h, h->vdT, (const double*)Y, ldy, m, (double*)X, ldx, stream, true);
}

ph_status online_matvec(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy, cudaStream_t stream) {
    ensure_workspace(h, m);
    if (h->opts.prec == PH_FP32)
        return matvec_typed<float>(h, h->vf, (const float*)X, ldx, m, (float*)Y, ldy, stream);
    return matvec_typed<double>(h, h->vd, (const double*)X, ldx, m, (double*)Y, ldy, stream);
}

}  // namespace ph
