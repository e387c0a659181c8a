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

#include "common.cuh"
#include "handle.h"

namespace ph {

namespace {

constexpr int kThreads = 256;

// ----------------------------------------------------------------------------- instantiate

// v_k(theta) = (w_k / (theta - eta_k)) / sum_j w_j / (theta - eta_j) with the
// barycentric weights w (Berrut & Trefethen, SIAM Review 2004, eq. 4.2); an
// exact node gives the exact unit vector.  One warp per parameter dimension.
__device__ void parametric_vectors(const double* nodes, const double* bw, const int* pt, int dt,
                                   const double* theta, double (*out)[kMaxPTheta]) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (warp < dt) {
        const int p = pt[warp];
        const double th = theta[warp];
        double num = 0.0;
        bool hit = false;
        if (lane < p) {
            double diff = th - nodes[warp * kMaxPTheta + lane];
            hit = (diff == 0.0);
            num = hit ? 0.0 : bw[warp * kMaxPTheta + lane] / diff;
        }
        unsigned any = __ballot_sync(0xffffffffu, hit);
        double den = num;
        for (int o = 16; o > 0; o >>= 1) den += __shfl_xor_sync(0xffffffffu, den, o);
        if (lane < p) out[warp][lane] = any ? (hit ? 1.0 : 0.0) : num / den;
    }
}

template <typename T>
__global__ void instantiate_kernel(DevView<T> v, double th0, double th1, double th2, int near_ctas) {
    __shared__ double sv[kMaxDim][kMaxPTheta];
    const double th[3] = {th0, th1, th2};
    parametric_vectors(v.theta_nodes, v.theta_bw, v.p_theta, v.dtheta, th, sv);
    __syncthreads();
    const int P = v.p_theta[0];
    if (blockIdx.x == 0 && threadIdx.x < P) v.v64[threadIdx.x] = sv[0][threadIdx.x];
    if ((int)blockIdx.x < near_ctas) {
        // near weights w_b[c] = sum_t G_{b,2}[c, t] v[t]  (d_theta = 1: G_{b,2} is r x P x 1)
        const int b = blockIdx.x * blockDim.x + threadIdx.x;
        if (b < v.n_near) {
            const int r = v.nb_rank[b];
            const double* G = v.near_theta + v.nb_toff[b];
            T* w = v.w + v.nb_woff[b];
            for (int c = 0; c < r; ++c) {
                double s = 0.0;
                for (int t = 0; t < P; ++t) s += G[c + r * t] * sv[0][t];
                w[c] = (T)s;
            }
        }
    } else {
        // far core matrix H_k = G_{k,d+1} x_2 v  (r_d x r_{d+1}, column-major)
        const int key = blockIdx.x - near_ctas;
        const int* rk = v.key_ranks + (size_t)key * (v.Delta + 1);
        const int ra = rk[v.d], rb = rk[v.d + 1];
        const double* G = v.far_theta + v.key_off[(size_t)key * v.Delta + v.d];
        T* H = v.H + v.key_hoff[key];
        for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) {
            const int a = e % ra, b = e / ra;
            double s = 0.0;
            for (int t = 0; t < P; ++t) s += G[a + ra * (t + P * b)] * sv[0][t];
            H[e] = (T)s;
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

// One CTA per target leaf s.  Thread (row i, group g) walks the columns j = g, g + G, ... of
// every near block (s, t): d_ij = sum_k w_k G_{b,1}[k][i + n_s j] (coalesced over i), then
// acc[c] += d_ij x_t[j][c] with x_t staged in shared memory.  The instantiated block is never
// written; the groups' partial sums are reduced in shared memory and Y_near written once.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) near_kernel(DevView<T> v, int S, int c0, int maxleaf) {
    extern __shared__ unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);              // maxleaf x MC
    T* red = xs + (size_t)maxleaf * MC;                   // kThreads x MC
    T* sw = red + (size_t)kThreads * MC;                  // kMaxNearRank
    const int leaf = blockIdx.x;
    const int snode = v.leaf_node[leaf];
    const int row0 = v.node_begin[snode];
    const int ns = v.node_end[snode] - row0;
    const int b0 = v.near_by_leaf[leaf], b1 = v.near_by_leaf[leaf + 1];
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
            if (active) {
                const long long slab = (long long)ns * nt;
                const T* Gp = v.near_cores + v.nb_off[b] + (rbase + i);
#pragma unroll 4
                for (int j = g; j < nt; j += G) {
                    const T* gj = Gp + (long long)j * ns;
                    T dij = T(0);
                    for (int k = 0; k < r; ++k) dij += sw[k] * __ldg(gj + k * slab);
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
            for (int c = 0; c < MC; ++c) v.Ynear[(long long)(row0 + rbase + i) * S + c0 + c] = acc[c];
        }
    }
}

// --------------------------------------------------------------------------------- H^2 sweeps

// xhat_s[I][c] = sum_{j in s} prod_k U_k[j][i_k] X[j][c]  (leaf stage of Alg. FastForward)
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) upsweep_leaf_kernel(DevView<T> v, int S, int c0) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int CH = 32;
    T* su = reinterpret_cast<T*>(smem_raw);               // CH x d x p_s
    T* sx = su + CH * kMaxDim * kMaxPs;                    // CH x MC
    const int leaf = blockIdx.x;
    const int node = v.leaf_node[leaf];
    const int row0 = v.node_begin[node], ns = v.node_end[node] - row0;
    const int ps = v.p_s, d = v.d, PD = v.PD;
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
}

// One mode-k product of the tensor z (p^d x MC, little-endian) with a p x p matrix in shared
// memory: out[.., a, ..] = sum_b A(a, b) z[.., b, ..], A(a, b) = E[b p + a] (transposed, up-sweep)
// or E[a p + b] (down-sweep).
template <typename T, int MC>
__device__ void mode_product(const T* z, T* out, const T* E, int p, int d, int k, bool transpose) {
    int stride = 1;
    for (int q = 0; q < k; ++q) stride *= p;
    int PD = 1;
    for (int q = 0; q < d; ++q) PD *= p;
    for (int e = threadIdx.x; e < PD * MC; e += blockDim.x) {
        const int I = e / MC, c = e % MC;
        const int a = (I / stride) % p;
        const int base = I - a * stride;
        T s = T(0);
        for (int b = 0; b < p; ++b) {
            const T m = transpose ? E[b * p + a] : E[a * p + b];
            s += m * z[(base + b * stride) * MC + c];
        }
        out[e] = s;
    }
}

// Up-sweep (transpose = true): xhat_s = sum over children s' of (E_{s',d} (x) .. (x) E_{s',1})^T xhat_s'.
// Down-sweep (transpose = false): yhat_s' += (E_{s',d} (x) .. (x) E_{s',1}) yhat_s for each child s'.
// FastKron (§3.6.3) applies the Kronecker factors one mode at a time.  One CTA per node of `level`.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) transfer_kernel(DevView<T> v, const int* nodes, int S, int c0,
                                                            bool up, T* src_all, T* dst_all) {
    extern __shared__ unsigned char smem_raw[];
    const int PD = v.PD, p = v.p_s, d = v.d;
    T* sE = reinterpret_cast<T*>(smem_raw);  // 2 p^2
    T* b0 = sE + 2 * p * p;
    T* b1 = b0 + (size_t)PD * MC;
    T* sacc = b1 + (size_t)PD * MC;
    for (int e = threadIdx.x; e < 2 * p * p; e += blockDim.x) sE[e] = v.E[e];
    const int node = nodes[blockIdx.x];
    const int cb = v.node_child_off[node], ce = v.node_child_off[node + 1];
    if (up) {
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x) sacc[e] = T(0);
        for (int q = cb; q < ce; ++q) {
            const int ch = v.node_children[q];
            const int halves = v.node_halves[ch];
            __syncthreads();
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
                b0[e] = src_all[((long long)ch * PD + e / MC) * S + c0 + e % MC];
            T* in = b0;
            T* out = b1;
            for (int k = 0; k < d; ++k) {
                __syncthreads();
                mode_product<T, MC>(in, out, sE + ((halves >> k) & 1) * p * p, p, d, k, true);
                T* t = in; in = out; out = t;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x) sacc[e] += in[e];
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
            const int halves = v.node_halves[ch];
            T* in = sacc;
            T* out = b0;
            for (int k = 0; k < d; ++k) {
                __syncthreads();
                mode_product<T, MC>(in, out, sE + ((halves >> k) & 1) * p * p, p, d, k, false);
                in = out;
                out = (out == b0) ? b1 : b0;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
                dst_all[((long long)ch * PD + e / MC) * S + c0 + e % MC] += in[e];
        }
    }
}

// Multiplication stage of Alg. "Modified H^2-Matrix MVM": for every far block (s, t) with
// compressed class k, z = xhat_t; d right-core steps z <- reshape(z, [p^{d-i-1}, p r]) G^{1}^T;
// z <- H_k z; d left-core steps z <- G^{2} reshape(z, [r, p^i]); yhat_s += z.  One CTA per target.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) coupling_kernel(DevView<T> v, int S, int c0) {
    extern __shared__ unsigned char smem_raw[];
    const int PD = v.PD, p = v.p_s, d = v.d, Delta = v.Delta;
    T* yacc = reinterpret_cast<T*>(smem_raw);
    T* z0 = yacc + (size_t)PD * MC;
    T* z1 = z0 + (size_t)PD * MC;
    const int ti = blockIdx.x;
    const int s = v.far_targets[ti];
    for (int e = threadIdx.x; e < PD * MC; e += blockDim.x) yacc[e] = T(0);
    for (int fb = v.far_by_target[ti]; fb < v.far_by_target[ti + 1]; ++fb) {
        const int t = v.fb_t[fb], key = v.fb_key[fb];
        const int* rk = v.key_ranks + (size_t)key * (Delta + 1);
        const long long* off = v.key_off + (size_t)key * Delta;
        __syncthreads();
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            z0[e] = v.xhat[((long long)t * PD + e / MC) * S + c0 + e % MC];
        T* in = z0;
        T* out = z1;
        // right cores G_{Delta}, ..., G_{Delta-d+1}: out[A + a s'] = sum_K in[A + a K] G[s' + r' K]
        int a = PD / p;
        for (int i = 0; i < d; ++i) {
            const int core = Delta - 1 - i;  // 0-based
            const int rin = rk[core + 1], rout = rk[core];
            const int K = p * rin;
            const T* G = v.far_cores + off[core];
            __syncthreads();
            for (int e = threadIdx.x; e < a * rout * MC; e += blockDim.x) {
                const int c = e % MC, q = e / MC;
                const int A = q % a, so = q / a;
                T acc = T(0);
                for (int kk = 0; kk < K; ++kk) acc += in[(A + a * kk) * MC + c] * G[so + rout * kk];
                out[e] = acc;
            }
            T* tmp = in; in = out; out = tmp;
            a /= p;
        }
        // H step: out[x] = sum_y H[x + r_d y] in[y]
        {
            const int ra = rk[d], rb = rk[d + 1];
            const T* H = v.H + v.key_hoff[key];
            __syncthreads();
            for (int e = threadIdx.x; e < ra * MC; e += blockDim.x) {
                const int c = e % MC, x = e / MC;
                T acc = T(0);
                for (int y = 0; y < rb; ++y) acc += H[x + ra * y] * in[y * MC + c];
                out[e] = acc;
            }
            T* tmp = in; in = out; out = tmp;
        }
        // left cores G_d, ..., G_1: out[(s' + r' I) + r' p B] = sum_S G[s' + r' I + r' p S] in[S + r B]
        int bsz = 1;
        for (int i = 0; i < d; ++i) {
            const int core = d - 1 - i;
            const int rin = rk[core + 1], rout = rk[core];
            const T* G = v.far_cores + off[core];
            const int rows = rout * p;
            __syncthreads();
            for (int e = threadIdx.x; e < rows * bsz * MC; e += blockDim.x) {
                const int c = e % MC, q = e / MC;
                const int row = q % rows, B = q / rows;
                T acc = T(0);
                for (int ss = 0; ss < rin; ++ss) acc += G[row + rows * ss] * in[(ss + rin * B) * MC + c];
                out[e] = acc;
            }
            T* tmp = in; in = out; out = tmp;
            bsz *= p;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x) yacc[e] += in[e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
        v.yhat[((long long)s * PD + e / MC) * S + c0 + e % MC] = yacc[e];
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
        const int ra = rk[v.d], rb = rk[v.d + 1];
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

// Y[perm[i] + c ldy] = Y_near[i][c] + (U_s yhat_s)[i][c] (H^2, leaf stage of FastBackward)
//                    or Y_near[i][c] + sum over levels of y_far (H).  One CTA per leaf.
template <typename T, int MC>
__global__ void __launch_bounds__(kThreads) combine_kernel(DevView<T> v, T* __restrict__ Y, long long ldy,
                                                           int m, int S, int c0, int h2) {
    extern __shared__ unsigned char smem_raw[];
    T* sy = reinterpret_cast<T*>(smem_raw);  // PD x MC
    const int leaf = blockIdx.x;
    const int node = v.leaf_node[leaf];
    const int row0 = v.node_begin[node], ns = v.node_end[node] - row0;
    const int ps = v.p_s, d = v.d, PD = v.PD;
    if (h2) {
        for (int e = threadIdx.x; e < PD * MC; e += blockDim.x)
            sy[e] = v.yhat[((long long)node * PD + e / MC) * S + c0 + e % MC];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const long long row = row0 + i;
        T acc[MC];
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[c] = v.Ynear[row * S + c0 + c];
        if (h2) {
            const T* u = v.U + row * d * ps;
            for (int I = 0; I < PD; ++I) {
                int r = I;
                T w = u[r % ps];
                if (d > 1) { r /= ps; w *= u[ps + r % ps]; }
                if (d > 2) { r /= ps; w *= u[2 * ps + r % ps]; }
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[c] += w * sy[I * MC + c];
            }
        } else {
            for (int sl = 0; sl < v.n_far_levels; ++sl)
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[c] += v.yfar[((long long)sl * v.n + row) * S + c0 + c];
        }
        const int orig = v.perm[row];
#pragma unroll
        for (int c = 0; c < MC; ++c)
            if (c0 + c < m) Y[orig + (long long)(c0 + c) * ldy] = acc[c];
    }
}

int pick_mc(int m) {
    if (m <= 1) return 1;
    if (m <= 2) return 2;
    if (m <= 4) return 4;
    if (m <= 8) return 8;
    return 16;
}

template <typename T, int MC>
void set_smem(const void* fn, size_t bytes) {
    PH_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <typename T, int MC>
void run_matvec(ph_handle* h, DevView<T>& v, const T* X, long long ldx, int m, T* Y, long long ldy,
                cudaStream_t stream, int S) {
    const Plan& plan = h->plan;
    const int nleaves = (int)plan.leaves.size();
    int maxleaf = 1;
    for (int l : plan.leaves) maxleaf = std::max(maxleaf, plan.nodes[l].size());
    const bool h2 = (h->opts.fmt == PH_FMT_H2);
    const int PD = v.PD;
    // fork: the far path runs on the side stream, concurrently with the near field
    PH_CUDA(cudaEventRecord(h->ev_fork, stream));
    PH_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    for (int c0 = 0; c0 < S; c0 += MC) {
        size_t smem = ((size_t)maxleaf * MC + (size_t)kThreads * MC + kMaxNearRank) * sizeof(T);
        set_smem<T, MC>((const void*)near_kernel<T, MC>, smem);
        ProfScope ps(h, 2, stream);
        near_kernel<T, MC><<<nleaves, kThreads, smem, stream>>>(v, S, c0, maxleaf);
        PH_LAUNCH("near_kernel");
    }
    if (!plan.far_targets.empty()) {
        for (int c0 = 0; c0 < S; c0 += MC) {
            if (h2) {
                size_t sm_leaf = ((size_t)32 * kMaxDim * kMaxPs + 32 * MC) * sizeof(T);
                {
                    ProfScope ps(h, 3, h->side);
                    upsweep_leaf_kernel<T, MC><<<nleaves, kThreads, sm_leaf, h->side>>>(v, S, c0);
                }
                PH_LAUNCH("upsweep_leaf_kernel");
                size_t sm_tr = ((size_t)2 * v.p_s * v.p_s + 3 * (size_t)PD * MC) * sizeof(T);
                set_smem<T, MC>((const void*)transfer_kernel<T, MC>, sm_tr);
                for (int l = plan.depth - 1; l >= h->min_far_level; --l) {
                    int cnt = h->level_nodes_off[l + 1] - h->level_nodes_off[l];
                    if (cnt == 0) continue;
                    ProfScope ps(h, 4, h->side);
                    transfer_kernel<T, MC><<<cnt, kThreads, sm_tr, h->side>>>(
                        v, h->d_level_nodes + h->level_nodes_off[l], S, c0, true, v.xhat, v.xhat);
                    PH_LAUNCH("transfer_kernel(up)");
                }
                size_t sm_c = 3 * (size_t)PD * MC * sizeof(T);
                set_smem<T, MC>((const void*)coupling_kernel<T, MC>, sm_c);
                {
                    ProfScope ps(h, 5, h->side);
                    coupling_kernel<T, MC><<<(int)plan.far_targets.size(), kThreads, sm_c, h->side>>>(v, S, c0);
                }
                PH_LAUNCH("coupling_kernel");
                for (int l = h->min_far_level; l < plan.depth; ++l) {
                    int cnt = h->level_nodes_off[l + 1] - h->level_nodes_off[l];
                    if (cnt == 0) continue;
                    ProfScope ps(h, 6, h->side);
                    transfer_kernel<T, MC><<<cnt, kThreads, sm_tr, h->side>>>(
                        v, h->d_level_nodes + h->level_nodes_off[l], S, c0, false, v.yhat, v.yhat);
                    PH_LAUNCH("transfer_kernel(down)");
                }
            } else {
                int maxnode = 1, rmax = 1;
                for (int s : plan.far_targets) maxnode = std::max(maxnode, plan.nodes[s].size());
                for (size_t key = 0; key < plan.key_rep.size(); ++key) {
                    const int* rk = &h->key_ranks[key * (h->Delta + 1)];
                    rmax = std::max(rmax, std::max(rk[v.d], rk[v.d + 1]));
                }
                size_t sm_h = ((size_t)maxnode * MC + 2 * (size_t)rmax * MC) * sizeof(T);
                set_smem<T, MC>((const void*)far_h_kernel<T, MC>, sm_h);
                ProfScope ps(h, 7, h->side);
                far_h_kernel<T, MC><<<(int)plan.far_targets.size(), kThreads, sm_h, h->side>>>(v, S, c0, rmax);
                PH_LAUNCH("far_h_kernel");
            }
        }
    }
    PH_CUDA(cudaEventRecord(h->ev_join, h->side));
    PH_CUDA(cudaStreamWaitEvent(stream, h->ev_join, 0));
    for (int c0 = 0; c0 < S; c0 += MC) {
        size_t sm = (size_t)PD * MC * sizeof(T);
        set_smem<T, MC>((const void*)combine_kernel<T, MC>, sm);
        ProfScope ps(h, 8, stream);
        combine_kernel<T, MC><<<nleaves, kThreads, sm, stream>>>(v, Y, ldy, m, S, c0,
                                                                 (h2 && !plan.far_targets.empty()) ? 1 : 0);
        PH_LAUNCH("combine_kernel");
    }
}

template <typename T>
ph_status matvec_typed(ph_handle* h, DevView<T>& v, const T* X, long long ldx, int m, T* Y, long long ldy,
                       cudaStream_t stream) {
    const int MC = pick_mc(m);
    const int S = (int)ceil_div(m, MC) * MC;
    const bool h2 = (h->opts.fmt == PH_FMT_H2);
    const int check = h->opts.check_finite ? 1 : 0;
    if (check) PH_CUDA(cudaMemsetAsync(v.flags, 0, sizeof(int), stream));
    const long long total = (long long)v.n * S;
    int grid = (int)std::min<long long>(ceil_div(total, kThreads), 152 * 16);
    {
        ProfScope ps(h, 1, stream);
        gather_kernel<T><<<grid, kThreads, 0, stream>>>(v, X, ldx, m, S, check);
        PH_LAUNCH("gather_kernel");
    }
    if (h2 && !h->plan.far_targets.empty())
        PH_CUDA(cudaMemsetAsync(v.yhat, 0, (size_t)v.n_nodes * v.PD * S * sizeof(T), stream));
    if (!h2 && v.n_far_levels > 0)
        PH_CUDA(cudaMemsetAsync(v.yfar, 0, (size_t)v.n_far_levels * v.n * S * sizeof(T), stream));
    switch (MC) {
        case 1: run_matvec<T, 1>(h, v, X, ldx, m, Y, ldy, stream, S); break;
        case 2: run_matvec<T, 2>(h, v, X, ldx, m, Y, ldy, stream, S); break;
        case 4: run_matvec<T, 4>(h, v, X, ldx, m, Y, ldy, stream, S); break;
        case 8: run_matvec<T, 8>(h, v, X, ldx, m, Y, ldy, stream, S); break;
        default: run_matvec<T, 16>(h, v, X, ldx, m, Y, ldy, stream, S); break;
    }
    if (check) {
        int bad = 0;
        PH_CUDA(cudaMemcpyAsync(&bad, v.flags, sizeof(int), cudaMemcpyDeviceToHost, stream));
        PH_CUDA(cudaStreamSynchronize(stream));
        if (bad) throw Error(PH_ERR_NONFINITE, "X has non-finite entries");
    }
    return PH_OK;
}

template <typename T>
void instantiate_typed(ph_handle* h, DevView<T>& v, const double* theta, cudaStream_t stream) {
    const int near_ctas = (int)ceil_div(std::max(v.n_near, 1), kThreads);
    const int grid = near_ctas + v.n_keys;
    double th[3] = {0, 0, 0};
    for (int k = 0; k < h->opts.dtheta; ++k) th[k] = theta[k];
    ProfScope ps(h, 0, stream);
    instantiate_kernel<T><<<grid, kThreads, 0, stream>>>(v, th[0], th[1], th[2], near_ctas);
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

ProfScope::ProfScope(ph_handle* h_, int kind_, cudaStream_t s_) : h(h_), kind(kind_), s(s_) {
    if (!h->prof) return;
    b = prof_event(h);
    PH_CUDA(cudaEventRecord(b, s));
}

ProfScope::~ProfScope() {
    if (!b) return;
    cudaEvent_t e = prof_event(h);
    cudaEventRecord(e, s);
    h->prof_recs.push_back({kind, b, e});
}

ph_status online_instantiate(ph_handle* h, const double* theta, cudaStream_t stream) {
    if (h->opts.prec == PH_FP32) instantiate_typed<float>(h, h->vf, theta, stream);
    else instantiate_typed<double>(h, h->vd, theta, stream);
    return PH_OK;
}

ph_status online_matvec(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy, cudaStream_t stream) {
    ensure_workspace(h, m);
    if (h->opts.prec == PH_FP32)
        return matvec_typed<float>(h, h->vf, (const float*)X, ldx, m, (float*)Y, ldy, stream);
    return matvec_typed<double>(h, h->vd, (const double*)X, ldx, m, (double*)Y, ldy, stream);
}

}  // namespace ph
