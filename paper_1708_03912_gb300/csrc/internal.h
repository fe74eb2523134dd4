// Internal declarations shared by the host planner (planner.cpp) and the CUDA
// kernels (assemble.cu, linalg.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fraclap.h"

namespace fl {

constexpr int TILE = 32;        // elements per block: one warp lane per element
constexpr int MAXK_FAR = 6;     // collapsed rule orders compiled for the far-field kernel
constexpr int MAXQ_NEAR = 144;  // k_near <= 12 in 2D

// Quadrature rule on the reference cell: points (barycentric-style coordinates),
// weights, and P1 shape values at the points.
struct Rule {
    int k = 0, q = 0;
    std::vector<double> lam;   // q * dim   (1D: t; 2D: lambda1, lambda2)
    std::vector<double> w;     // q         (reference weights; 1D sums to 1, 2D to 1/2)
    std::vector<double> phi;   // q * (dim+1)
};

void gauss01(int k, std::vector<double>& x, std::vector<double>& w);
Rule make_rule(int dim, int k);

// Host-side plan of one mesh and one degree-of-freedom set.
struct Plan {
    int dim = 0, nvpc = 0;           // nvpc = vertices per cell = dim + 1
    int64_t nv = 0, nc = 0, nf = 0;
    std::vector<double> V;           // nv * dim
    std::vector<int> C;              // nc * nvpc, oriented, original cell order
    std::vector<double> jac;         // nc: reference-to-physical measure factor (2|K| or h)
    std::vector<int> F;              // nf * dim facet vertices (2D: sorted pair)
    std::vector<double> FN;          // nf * dim inward unit normal
    std::vector<double> FLEN;        // nf facet length (1 in 1D)
    std::vector<char> onb;           // nv on-boundary flag
    std::vector<int> v2c_ptr, v2c;   // vertex -> cells (original ids)
    std::vector<int> nbr_ptr, nbr;   // vertex -> neighbour vertices through mesh edges
    std::vector<int> v2f_ptr, v2f;   // vertex -> facets
    // internal (spatial) cell order
    std::vector<int> perm;           // internal -> original
    std::vector<int> iperm;          // original -> internal

    // ----- degree-of-freedom dependent part -----
    int paper_all = 0;               // 1: all vertices are DOFs
    int64_t n = 0;
    std::vector<int> vod, dov;       // dof -> vertex, vertex -> dof (-1)
    int64_t nblk = 0;
    std::vector<int> cdof;           // nc * nvpc (internal order): dof or -1
    std::vector<char> hasdof;        // nc (internal)
    std::vector<int> L_ptr, L_dof;   // per block: sorted dofs touched
    std::vector<int> loc;            // nc * nvpc (internal): index into the block's L list or -1
    std::vector<int> inc_ptr, inc_ent;  // per global L position: lane*nvpc+slot entries
    int maxL = 0;
    std::vector<int> tiles;          // ntiles * 2 (I <= J); empty until ensure_plan_tiles (the
                                     // symmetry reduction's subset is built by plan_symmetry)
    std::vector<int64_t> toff;       // ntiles + 1 offsets into the partial-tile storage
    std::vector<int> occ_ptr, occ_blk, occ_loc;  // dof -> (block, local index) occurrences
    std::vector<int> ex_ptr, ex_idx; // internal cell -> sorted internal partners handled elsewhere
    // near separated pairs (vertex-graph distance 1), internal indices, unordered
    std::vector<int> np_a, np_b;
    std::vector<int> enp_ptr, enp_ent;  // internal cell -> (pair*2 + role)
    // touching pairs (2D: common edge = 0, common vertex = 1; 1D: common vertex = 2)
    std::vector<int> tp_type, tp_vert;  // tp_vert: 5 vertex ids per pair (canonical order)
    std::vector<int> tp_cell;        // 2 original cell ids per pair (lower first)
    // element/facet pairs handled by the element kernel: internal cell -> (facet, class)
    // class 1 = near (distance 1), 2 = facet is an edge of the cell / 1D touching,
    // 3 = facet and cell share one vertex
    std::vector<int> ef_ptr, ef_fac, ef_cls;
    // contributions to the sparse near-field part
    int64_t nslots = 0;
    std::vector<int64_t> tp_slot;    // per touching pair, base slot (block of nloc^2)
    int64_t np_slot0 = 0;            // near pair p: np_slot0 + p * nvpc^2
    int64_t el_slot0 = 0;            // internal cell k: el_slot0 + k * nvpc^2
    std::vector<int> csr_ptr;        // n + 1
    std::vector<int> csr_col;
    std::vector<int64_t> g_ptr;      // nnz + 1
    std::vector<int64_t> g_slot;
    // ----- symmetry reduction (fl_create_sector; symmetry.cpp) -----
    int sym_K = 0;                   // > 0: the mesh is K rotated copies of a sector
    int64_t n_red = 0;               // orbits of the DOFs (the reduced problem's size)
    std::vector<int> red_rep;        // n_red: the whole DOF whose row represents orbit r
    std::vector<int> red_ptr, red_mem;  // orbit -> its whole DOFs, ascending
    std::vector<int> red_row;        // whole DOF -> r if it represents orbit r, else -1
    std::vector<int> red_vertex;     // n_red: the sector vertex of orbit r
    std::vector<int64_t> tri_list;   // upper-triangle tile index -> position in tiles, or -1
};

// Builds the mesh part (orientation, facets, adjacency, spatial order: Morton order of the cell
// centroids, with the cells flagged in `first`, if given, ahead of the rest).
int plan_mesh(Plan& P, int dim, int64_t nv, const double* V, int64_t nc, const int32_t* C, std::string& err,
              const std::vector<char>* first = nullptr);
// Builds the DOF-dependent part (all but the dense assembly's tile list).
int plan_dofs(Plan& P, int paper_all, std::string& err);
// The dense assembly's tile list: every block pair I <= J, ordered by (I, J), with the offsets of
// their partial blocks.  Built on first use (the cluster method and the strong form never need
// it: nblk^2 / 2 tiles, 40 M at 287 k cells); no-op once built or under the symmetry reduction.
// May throw std::bad_alloc.
void ensure_plan_tiles(Plan& P);
// Number of tiles of the dense assembly, built or not.
int64_t plan_tile_count(const Plan& P);
// Symmetry reduction (symmetry.cpp).  replicate_sector: the K copies of a sector mesh rotated by
// 2 pi l / K about the origin, vertices closer than 1e-10 in both coordinates merged (the
// earliest one kept), cells copy by copy; vmap[l * nv + v] = whole vertex of copy l of v.
void replicate_sector(int64_t nv, const double* V, int64_t nc, const int32_t* C, int K, std::vector<double>& W,
                      std::vector<int32_t>& CW, std::vector<int>& vmap);
// The orbits of P's DOFs (needs plan_dofs first) and the tiles restricted to the blocks
// holding a cell of a representative's support; vmap as from replicate_sector.
int plan_symmetry(Plan& P, int K, int64_t nvs, const std::vector<int>& vmap, std::string& err);

}  // namespace fl
