// Cluster tree and block partition of the cluster method (cluster.cpp).  Internal.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"

namespace fl {

struct ClusterPlan {
    int dim = 0, leaf = 0, nodes = 0, depth = 0;
    double eta = 0.0;
    int64_t n = 0;
    std::vector<int> perm;         // n: DOFs in tree order
    std::vector<int> lo, hi;       // per node: range of perm
    std::vector<int> son;          // 2 per node (-1: leaf)
    std::vector<int> level;        // per node
    std::vector<double> center;    // dim per node: centre of the cluster cube
    std::vector<double> side;      // per node: side of the cube
    std::vector<int> far, near;    // pairs of node ids (admissible; inadmissible leaf pairs)
};

// Builds the tree over P's DOFs and the partition for admissibility parameter eta and
// leaves of at most `leaf` DOFs.  FL_EINVAL for leaf < 1 or eta < 0.
int build_cluster_plan(const Plan& P, double eta, int leaf, ClusterPlan& C);

// The near field assembled directly (hnear.cpp): the tiles of element blocks its entries need
// and, per internal cell K with DOFs, the facets of the boundary of N(K) (K, its touching
// cells and the cells at vertex-graph distance 1) with their classes.
struct HNearPlan {
    std::vector<int> tiles;        // 2 per tile (I <= J), ordered by (I, J)
    std::vector<int64_t> toff;     // tiles + 1: offsets of the tiles' partial blocks
    std::vector<int> trow_ptr;     // nblk + 1: the tiles of block row I are trow_ptr[I] .. trow_ptr[I + 1] - 1
    std::vector<uint32_t> rowmask; // per tile: bit kk set when row cell 32 I + kk pairs with a cell of block J
                                   // in some near-field entry (the far kernel skips the other rows)
    std::vector<int> F;            // facet table, dim vertex ids per facet: the boundary facets of
    std::vector<double> FN, FLEN;  // Omega (ids < nf) then (nf + nvpc M + e): facet e of internal
                                   // cell M, normal pointing into M
    std::vector<int> ef_ptr, ef_fac, ef_cls;  // internal cell -> facets of the boundary of N(K):
                                              // class 2 / 3 shares two / one vertex with K, 1 at
                                              // vertex-graph distance 1, 0 the rest
};
int plan_hnear(const Plan& P, const ClusterPlan& C, HNearPlan& Q, std::string& err);

// Device copies of an HNearPlan and its tiles' partial blocks (the contribution slots, row sums
// and cell blocks are the mesh handle's, shared with its other assemblies).
struct HNearDev {
    int64_t ntiles = 0;
    int* tiles = nullptr;
    int64_t* toff = nullptr;
    int* trow_ptr = nullptr;
    uint32_t* rowmask = nullptr;
    int* F = nullptr;
    double *FN = nullptr, *FLEN = nullptr;
    int *ef_ptr = nullptr, *ef_fac = nullptr, *ef_cls = nullptr;
    double* P = nullptr;  // partial blocks of the tiles
};

}  // namespace fl
