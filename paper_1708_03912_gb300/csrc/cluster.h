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

// The strong form by the cluster method (adaptive.cu): the cell-rule points grouped by the leaf
// of the DOF of their cell closest to them (ties: the lower DOF; cells without a DOF vertex form
// one group of their own, with every DOF near and no far part), per group the near leaves as a
// bitset and the facets where the near part's normal derivative can jump (the facets of the cells
// touching a near DOF), and the far kernel's blocks.
struct HsfPlan {
    int kc = 0;
    int64_t npts = 0;
    int groups = 0, words = 0;            // groups; 32-bit words per near-leaf bitset
    std::vector<int> gnode;               // per group: its leaf node, or -1 (the cells without DOFs)
    std::vector<int> gp_ptr, gp_idx;      // per group: its points (internal cell k, point a: k q + a)
    std::vector<int> pgroup, plocal;      // per point: its group and its position in the group's list
    std::vector<int64_t> gf_ptr;          // per group: its facets (strong-form facet ids, ascending)
    std::vector<int> gf_fac;
    std::vector<uint32_t> gbits;          // groups x words
    std::vector<int> dof_leaf;            // per DOF: its leaf's index (leaves in node order)
    std::vector<int> gch;                 // per group: facet chunks of the far kernel
    std::vector<int64_t> gpo;             // per group: offset of its partial sums (points x chunks)
    std::vector<int> blk_g, blk_p0, blk_ch;  // far-kernel blocks: group, first point, facet chunk
    int64_t nparts = 0, maxf = 0;         // partial sums; the longest facet list
};
int plan_hsf(const Plan& P, const ClusterPlan& C, const std::vector<int>& c2f, int64_t nfac, int kc, HsfPlan& Q,
             std::string& err);

struct HsfDev {
    int groups = 0, words = 0, md = 0, m = 0;
    int64_t nparts = 0, nblocks = 0, maxf = 0;
    int *gnode = nullptr, *gp_ptr = nullptr, *gp_idx = nullptr, *pgroup = nullptr, *plocal = nullptr, *gf_fac = nullptr;
    int64_t *gf_ptr = nullptr, *gpo = nullptr;
    uint32_t* gbits = nullptr;
    int *dof_leaf = nullptr, *gch = nullptr, *blk_g = nullptr, *blk_p0 = nullptr, *blk_ch = nullptr;
    double* cj = nullptr;     // per group facet: the near part's jump times 1/(2sm)
    double* part = nullptr;   // far-kernel partial sums
    // the H-matrix's far field: per node yh [md], cube centre [d] and side
    const double *yh = nullptr, *center = nullptr, *side = nullptr;
};

}  // namespace fl
