// Handle (fl_ctx) layout and device-table bookkeeping.  Internal.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

namespace fl {

// Identity of a captured batch of CG iterations (pointers and sizes baked into the graph).
struct CgGraphKey {
    int64_t n;
    int dtype;
    const void* M;
    int64_t ldm;
    const double* dinv;
    double* d;
    double* r;
    float* pf;
    bool operator==(const CgGraphKey& o) const {
        return n == o.n && dtype == o.dtype && M == o.M && ldm == o.ldm && dinv == o.dinv && d == o.d && r == o.r &&
               pf == o.pf;
    }
};
struct CgGraph {
    CgGraphKey key;
    cudaGraphExec_t exec;
};

// Offsets of the per-s quadrature tables in one float64 buffer (built by build_rules).
struct RuleOffsets {
    int qf, qn, kf, kn, kt, kb;
    int64_t far_lam, far_w, far_phi;
    int64_t near_lam, near_w, near_phi;
    int64_t glf_t, glf_w, gln_t, gln_w;   // Gauss points on facets
    int64_t t_edge, t_vert, t_1d, t_ident, b_own, b_vert;
    int n_edge, n_vert, n_1d, n_ident, n_own, n_bvert;
};

// Compact record of a boundary facet (2D): the edge from e0 to e0 + (ex, ey) with its
// inward unit normal and length.
struct FacetRec {
    double e0x, e0y;   // start point
    double ex, ey;     // edge vector E1 - E0
    double nx, ny;     // inward unit normal
    double len, pad;
};

// One device allocation owned by a handle.
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Device copies of one Plan (one DOF set).
struct DevTables {
    bool ready = false;
    bool dense_ready = false;  // the dense assembly's tiles and far-field workspace (ensure_dense)
    // mesh
    double* V = nullptr;        // nv*dim
    double* jac_orig = nullptr; // nc (original order)
    int* F = nullptr;
    double* FN = nullptr;
    double* FLEN = nullptr;
    // internal cells
    double* cvx = nullptr;  // nc*nvpc*dim
    double* cen = nullptr;  // nc*dim
    double* jac = nullptr;  // nc
    char* hasdof = nullptr;
    int* loc = nullptr;
    int* cdof = nullptr;
    int *L_ptr = nullptr, *inc_ptr = nullptr, *inc_ent = nullptr;
    int* tiles = nullptr;
    int64_t* toff = nullptr;
    const uint32_t* tile_rowmask = nullptr;  // per tile, the row cells to compute (null: all; the double-word far kernel)
    int *occ_ptr = nullptr, *occ_blk = nullptr, *occ_loc = nullptr;
    int *ex_ptr = nullptr, *ex_idx = nullptr;
    int *np_a = nullptr, *np_b = nullptr, *enp_ptr = nullptr, *enp_ent = nullptr;
    int *tp_type = nullptr, *tp_vert = nullptr, *tp_cell = nullptr;
    int64_t* tp_slot = nullptr;
    int *ef_ptr = nullptr, *ef_fac = nullptr, *ef_cls = nullptr;
    int *csr_ptr = nullptr, *csr_col = nullptr, *csr_row = nullptr;
    int64_t *g_ptr = nullptr, *g_slot = nullptr;
    int64_t *v2c_ptr = nullptr;
    int* v2c = nullptr;
    int* vod = nullptr;
    int* dov = nullptr;     // nv: vertex -> dof or -1
    int* corig = nullptr;   // nc*nvpc vertex ids of the internal-order cells
    int* cells = nullptr;   // nc*nvpc oriented cells in original order
    // workspace (sized for float64)
    void* P = nullptr;      // partial far-field tiles
    void* Pd = nullptr;     // nblk * nc * Qf partial row sums
    void* pts = nullptr;    // nc * Qf * dim offsets from centroids
    void* pts_dw = nullptr; // nc * 16 double-word offsets (2D, float64 mode, k_far = 4)
    void* pts_near_dw = nullptr;  // nc * 36 double-word offsets of the near rule (2D, k_near = 6)
    double* Dn = nullptr;   // nnear * 2 * Qn
    double* Bf = nullptr;   // nc * Qf boundary sums (far facets)
    double* Bfp = nullptr;  // facet-chunk partials of Bf (double-word boundary kernel)
    double* eblk = nullptr; // nc * 6 far-independent part of each cell's diagonal block
    double* contrib = nullptr;
    double* csr_val = nullptr;
    void* facet_rec = nullptr;  // compact boundary-facet records (2D)
    double* rule = nullptr; // per-s rule tables (see assemble.cu)
    size_t rule_len = 0;
    float* rule32 = nullptr;  // their float32 copy (mixed-mode touching pairs)
    size_t rule32_len = 0;
    void* rule_dw = nullptr;  // their double-word copy (float pairs; float64-mode touching pairs)
    size_t rule_dw_len = 0;
    double rule_s = -1.0;        // the s the device tables hold (NaN while being rebuilt)
    bool rule32_ready = false;   // the float32 copy matches them
    std::vector<double> rule_host;
    RuleOffsets rule_ro{};
    // symmetry reduction (Plan::sym_K > 0)
    int *red_rep = nullptr, *red_ptr = nullptr, *red_mem = nullptr, *red_row = nullptr;
    int64_t* tri_list = nullptr;
    int* sector_of = nullptr;  // whole vertex -> the sector vertex it copies
    // strong form of the adaptive loop (adaptive.cu), built on first use
    bool sf_ready = false;
    int64_t sf_nfac = 0, sf_nint = 0;  // facets; the first sf_nint are interior
    int* sf_fac = nullptr;     // nfac*4: vertices a, b (1D: a twice), cell K+, cell K- (-1 on the boundary)
    double* sf_fn = nullptr;   // nfac*(dim+1): unit normal outward of K+, length (1D: 1)
    int* sf_c2f = nullptr;     // nc*nvpc: facets of every cell (original order)
    std::vector<int> sf_c2f_host;  // its host copy (the cluster strong form's planner)
    int* sf_perm = nullptr;    // nc: internal -> original cell
    int *sf_v2e_ptr = nullptr, *sf_v2e = nullptr;  // vertex -> facets through it (2D)
    double* sf_rule = nullptr; // cell rule, edge rule, near-edge rule of the last call
    size_t sf_rule_cap = 0;
    int sf_rule_key[3] = {0, 0, 0};
};

}  // namespace fl

struct fl_ctx {
    int dim = 0;
    int dof_mode = FL_DOF_INTERIOR;
    fl_options opt{};
    int device = 0;
    std::string err;
    fl::Plan plan[2];       // [0]: interior vertices, [1]: all vertices
    bool planned[2] = {false, false};
    fl::DevTables dev[2];
    std::vector<fl::DBuf> bufs;
    int profiling = 0;
    int no_persistent = 0;  // 1: run CG as captured kernel batches instead of one cooperative launch
    unsigned long long wait_ns = 2000000000ull;  // bound of a grid-barrier wait in the current solve
    int far_f64_pipe = 0;   // 1: float64-mode separated pairs on the float64 pipe (double-word otherwise)
    int far_variant = 0;    // launch variant of the double-word far kernel (0: tuning table, else 3)
    cudaEvent_t ev[2 * FL_NSTAGES] = {};
    bool ev_made = false;
    bool ev_recorded = false;
    int64_t h2d_bytes = 0;
    int64_t ws_bytes = 0;
    std::vector<fl::CgGraph> cg_graphs;   // captured CG batches, keyed by their pointers
    cudaStream_t cap_stream = nullptr;    // stream used only for graph capture
    // second stream of fl_assemble: the near, touching and boundary stages run on it while the
    // far-field stage runs on the caller's stream (fork/join by the two events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr;
    void* solve_ws = nullptr;     // solver workspace (device), grown on demand
    void* solve_host = nullptr;   // pinned scalars read back by the solver
    size_t solve_ws_bytes = 0;
    void* batch_ws = nullptr;     // batched-solver workspace (device), grown on demand
    size_t batch_ws_bytes = 0;
    void* batch_host = nullptr;   // pinned scalars of the batched solver
    void* sf_ws = nullptr;        // strong-form workspace (device), grown on demand
    size_t sf_ws_bytes = 0;
    // symmetry reduction (fl_create_sector): the mesh is sym_K rotated copies of a sector
    int sym_K = 0;
    int64_t sym_nvs = 0;            // sector vertices
    std::vector<int> sym_vmap;      // sym_K * sym_nvs: whole vertex of copy l of sector vertex v
    int* sym_sector_of = nullptr;   // device, whole vertex -> a sector vertex it copies
    void* sym_ws = nullptr;         // reduced-assembly workspace (representatives' rows), grown on demand
    size_t sym_ws_bytes = 0;
};

namespace fl {
// every kernel launch site bumps this counter (fl_launch_count)
void count_launch(int n = 1);
// returns plan index for order s (building it on demand); -1 on error (h->err set)
int plan_for(fl_ctx* h, double s);
// FL_ENOTIMPL with a message for calls that do not take a symmetry-reduced handle
int sym_unsupported(fl_ctx* h, const char* what);
// device copies of plan pi's tables (uploaded once per handle and plan)
int ensure_device_tables(fl_ctx* h, int pi, cudaStream_t st);
// caching allocator (pool.cpp): device and pinned host blocks reused across handles
cudaError_t pool_dev_alloc(void** out, size_t bytes);
void pool_dev_free(void* p);
cudaError_t pool_host_alloc(void** out, size_t bytes);
void pool_host_free(void* p);
int set_err(fl_ctx* h, int code, const std::string& msg);
// y = A x for a dense matrix of type dtype (linalg.cu); x, y float64 with strides; xf: n floats of
// scratch for the float32 copy of x (unused for FL_F64)
cudaError_t gemv(int dtype, const void* A, int64_t lda, int64_t n, const double* x, int64_t incx, double* y,
                 int64_t incy, float* xf, cudaStream_t st, bool xf_ready = false);
// z = V(r), float64 vectors on the finest level of a multigrid hierarchy (mg.cu)
int mg_precondition(fl_mg_handle m, const double* r, double* z, cudaStream_t st);
// tuning table (tune.cpp)
std::string device_name();
void tune_record(const std::string& device, const std::string& kernel, int64_t n, int nrhs, int nslices, int p0,
                 int p1, double ms);
bool tune_lookup(const std::string& device, const std::string& kernel, int64_t n, int nrhs, int nslices, int* p0,
                 int* p1);
unsigned tune_generation();  // changes whenever the table changes
// float64-mode separated pairs in double-word arithmetic (far_dw.cu): whether they apply
// (2D, k_far = 4, s in {1/4, 1/2, 3/4}), the double-word point offsets, the tile kernel,
// the launch variant it takes and the autotuner's record of one
bool far_dw_applies(const fl_ctx* h, const Plan& P, int pw);
int prep_far_dw(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, cudaStream_t st);
// (ntiles < 0: all of P.tiles; else the first ntiles of the tile list in t)
int launch_far_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                  cudaStream_t st, int64_t ntiles = -1);
int far_dw_variant(const fl_ctx* h, const Plan& P, int pw);
int bnd_dw_chunks(int64_t nc);
int launch_bnd_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                  cudaStream_t st);
void far_dw_record(const Plan& P, int pw, int variant, double ms);
// float64-mode near pairs (vertex-graph distance 1) in double-word arithmetic (far_dw.cu):
// 2D, k_near = 6, s in {1/4, 1/2, 3/4}, unless the float64 pipe is requested
bool near_dw_applies(const fl_ctx* h, const Plan& P, int pw);
// float64-mode touching pairs (2D) in double-word arithmetic, s in {1/4, 1/2, 3/4}
bool touch_dw_applies(const fl_ctx* h, const Plan& P, int pw);
int launch_touch_dw(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, double s, double C, int pw,
                    cudaStream_t st);
int launch_near_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                   double C, cudaStream_t st);
// the cluster method's near field from local computations (assemble.cu): nnz entries (row, col
// DOF ids) into nz_val; uses the handle's contribution slots and row-sum buffers
struct HNearDev;
int assemble_hnear(fl_ctx* h, int pi, double s, int precision, const HNearDev& q, int64_t nnz, const int* nz_row,
                   const int* nz_col, double* nz_val, cudaStream_t st);
// adaptive loop (adaptive.cu, refine.cpp)
int strong_form(fl_ctx* h, double s, const double* u, int k_cell, int k_edge, int k_near, double* S, cudaStream_t st);
int br_indicators(fl_ctx* h, double s, const double* u, const double* f, int k_cell, int k_edge, int k_near,
                  double* eta, double* S, cudaStream_t st);
int mark_max(fl_ctx* h, double s, const double* eta, double theta, uint8_t* dof_marks, uint8_t* cell_marks,
             cudaStream_t st);
// the strong form by the cluster method (adaptive.cu): the facet topology's host data for the
// planner, and the evaluation with the plan's device copies (far field: H's yh after the far chain)
struct HsfDev;
int sf_topology(fl_ctx* h, int pi, cudaStream_t st, const std::vector<int>** c2f, int64_t* nfac);
// the same facets on the host alone: cell -> facets, and the two vertices of every facet
int sf_facets_host(const Plan& P, std::vector<int>& c2f, std::vector<int>& fac_vert, int64_t* nfac);
int strong_form_cluster(fl_ctx* h, double s, const double* u, int kc, int ke, int kn, const HsfDev& g, double* S,
                        cudaStream_t st);
int br_from_strong_form(fl_ctx* h, double s, const double* f, int kc, const double* S, double* eta, cudaStream_t st);
// Y = alpha M X + beta B, M the P1 mass matrix on the DOFs (assemble.cu; Y may be B)
int mass_apply(fl_ctx* h, double s, int nrhs, double alpha, const double* X, int64_t ldx, double beta, const double* B,
               int64_t ldb, double* Y, int64_t ldy, cudaStream_t st);
int refine_mesh(int dim, int64_t nv, const double* V, int64_t nc, const int32_t* C, const uint8_t* marks,
                int64_t cap_v, int64_t cap_c, double* V_out, int32_t* C_out, int64_t* nv_out, int64_t* nc_out,
                std::string& err);
}  // namespace fl
