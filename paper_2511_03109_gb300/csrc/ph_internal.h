// Internal declarations of libph (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "ph.h"

namespace ph {

constexpr int kMaxDim = 3;
constexpr int kMaxPs = 16;
constexpr int kMaxPTheta = 32;
constexpr int kMaxNearRank = 128;  // near ranks r_{b,1}: never binds for <= 128 theta-grid points
constexpr int kMaxThetaGrid = 1024;  // product of the p_theta_i

// One node sigma of the cluster tree (§3.2).  Points of a node are the
// contiguous range [begin, end) of the cluster order; inside a node the order
// of the original index set I is kept (§3.1).
struct Node {
    int level = 0;
    int parent = -1;
    int halves = 0;  // bit k set: high half of the parent box in dimension k
    int begin = 0, end = 0;
    int leaf = -1;   // position in the leaf list, -1 for inner nodes
    std::vector<int> children;
    double lo[kMaxDim] = {0, 0, 0}, hi[kMaxDim] = {0, 0, 0};
    int size() const { return end - begin; }
};

// Cluster tree, block cluster tree and the translation classes of far blocks.
struct Plan {
    int d = 0;
    long n = 0;
    int depth = 0;
    std::vector<Node> nodes;           // depth-first pre-order
    std::vector<int> perm;             // cluster position -> original point index
    std::vector<int> leaves;           // node ids of the leaves, in cluster order
    std::vector<int> near_s, near_t;   // near blocks (node ids), grouped by target leaf
    std::vector<int> inner_near_s, inner_near_t;  // adaptive trees: near blocks with an inner cluster
    std::vector<int> far_s, far_t;     // far blocks (node ids), grouped by target node
    std::vector<int> far_key;          // far block -> compressed-tensor class
    std::vector<int> key_rep;          // class -> representative far block
    std::vector<int> near_by_leaf;     // CSR offsets: near blocks of leaf l are [near_by_leaf[l], near_by_leaf[l+1])
    std::vector<int> far_targets;      // nodes that own far blocks, in order
    std::vector<int> far_by_target;    // CSR offsets over far_targets
};

// Builds the uniform cluster tree of depth l_max over [0,1]^d and the block
// cluster tree with admissibility eta.  Throws std::invalid_argument for
// points outside the root box.
// leaf_size > 0 builds the adaptive tree instead: a node is split while it holds more than
// leaf_size points and its level is below 20 (l_max is then ignored); near blocks between a leaf
// and an inner cluster go to inner_near_s / inner_near_t.
void build_plan(const double* points, long n, int d, int l_max, double eta, bool dedup, Plan& plan,
                int leaf_size = 0);

bool kernel_translation_invariant(ph_kernel k);

// Chebyshev nodes of the first kind on [a, b], ascending (§2.2), and their
// barycentric weights w_k = 1 / prod_{j != k} (eta_k - eta_j), scaled to max |w| = 1.
void cheb_nodes(double a, double b, int p, double* out);
void bary_weights(const double* nodes, int p, double* w);
// Lagrange values ell_k(x), k < p, by the barycentric formula (exact unit row at a node).
void lagrange_bary(const double* nodes, const double* w, int p, double x, double* out);

}  // namespace ph
