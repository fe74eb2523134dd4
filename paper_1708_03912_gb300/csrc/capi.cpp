// C ABI entry points that manage handles, DOF sets and dispatch to the device code.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>

#include "context.h"

namespace fl {
int assemble(fl_ctx* h, double s, int precision, double* A, int64_t lda, cudaStream_t st);
int tune_assemble(fl_ctx* h, double s, double* A, int64_t lda, int reps, int* best_variant, double* best_ms,
                  cudaStream_t st);
int assemble_nearfield_csr(fl_ctx* h, double s, int precision, int64_t* nnz, int32_t* rowptr, int32_t* col,
                           double* val, cudaStream_t st);
int load_vector(fl_ctx* h, double s, const double* f, int nrhs, double* b, int64_t ldb, cudaStream_t st);
int heat_matrix(fl_ctx* h, double s, double dt, const double* A, int64_t lda, double* H, int64_t ldh, cudaStream_t st);
int mass_apply(fl_ctx* h, double s, int nrhs, double alpha, const double* X, int64_t ldx, double beta, const double* B,
               int64_t ldb, double* Y, int64_t ldy, cudaStream_t st);

int plan_for(fl_ctx* h, double s) {
    if (!(s > 0.0 && s < 1.0)) {
        set_err(h, FL_EINVAL, "s must lie in (0, 1)");
        return -1;
    }
    const int idx = (h->dof_mode == FL_DOF_PAPER && s < 0.5) ? 1 : 0;
    if (!h->planned[idx]) {
        // the mesh part always lives in plan[0]
        h->plan[idx] = h->plan[0];
        std::string err;
        int r = plan_dofs(h->plan[idx], idx, err);
        if (r == FL_OK && h->sym_K) r = plan_symmetry(h->plan[idx], h->sym_K, h->sym_nvs, h->sym_vmap, err);
        if (r != FL_OK) {
            set_err(h, r, err);
            return -1;
        }
        h->planned[idx] = true;
    }
    return idx;
}

int sym_unsupported(fl_ctx* h, const char* what) {
    return set_err(h, FL_ENOTIMPL, std::string(what) + " is not available on a symmetry-reduced (sector) handle");
}
}  // namespace fl

#include <atomic>

static thread_local std::string g_create_err;
static std::atomic<uint64_t> g_launches{0};

namespace fl {
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace fl

extern "C" {

void fl_default_options(fl_options* o) {
    if (!o) return;
    o->k_far = 4;
    o->k_near = 6;
    o->k_touch = 8;
    o->k_bnd = 8;
    o->regional = 0;
    o->k_vertex = 6;
    o->far_f64_pipe = 0;
}

// sector: the symmetry reduction's K and copy map (vertices and cells are then the whole mesh)
struct SectorArgs {
    int K;
    int64_t nvs;
    std::vector<int> vmap;
};

static int create_impl(fl_handle* out, int dim, int64_t n_vertices, const double* vertices_host, int64_t n_cells,
                       const int32_t* cells_host, int dof_mode, const fl_options* opt, SectorArgs* sec) {
    g_create_err.clear();
    if (!out) {
        g_create_err = "handle pointer is NULL";
        return FL_EINVAL;
    }
    *out = nullptr;
    fl_options o;
    fl_default_options(&o);
    if (opt) o = *opt;
    if (dof_mode != FL_DOF_INTERIOR && dof_mode != FL_DOF_PAPER) {
        g_create_err = "unknown dof_mode";
        return FL_EINVAL;
    }
    if (o.k_far < 1 || o.k_far > 32 || o.k_near < 1 || o.k_near > 32 || o.k_touch < 1 || o.k_touch > 32 ||
        o.k_bnd < 1 || o.k_bnd > 32 || o.k_vertex < 1 || o.k_vertex > 32) {
        g_create_err = "quadrature orders must lie in [1, 32]";
        return FL_EINVAL;
    }
    fl_ctx* h = new (std::nothrow) fl_ctx;
    if (!h) {
        g_create_err = "out of host memory";
        return FL_ENOMEM;
    }
    h->dim = dim;
    h->dof_mode = dof_mode;
    h->opt = o;
    h->far_f64_pipe = o.far_f64_pipe ? 1 : 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        dev = 0;
        cudaGetLastError();
    }
    h->device = dev;
    std::string err;
    int r;
    try {
        // symmetry reduction: the cells at a copy-0 vertex (every representative's support lies
        // among them) first, so that they fill few blocks of the tile scheme
        std::vector<char> first;
        if (sec) {
            std::vector<char> c0(n_vertices, 0);
            for (int64_t v = 0; v < sec->nvs; ++v) c0[sec->vmap[v]] = 1;
            first.assign(n_cells, 0);
            for (int64_t k = 0; k < n_cells; ++k)
                for (int a = 0; a < 3; ++a) first[k] |= c0[cells_host[3 * k + a]];
        }
        r = fl::plan_mesh(h->plan[0], dim, n_vertices, vertices_host, n_cells, cells_host, err, sec ? &first : nullptr);
        if (r == FL_OK) {
            r = fl::plan_dofs(h->plan[0], 0, err);
            if (r == FL_OK && sec) {
                h->sym_K = sec->K;
                h->sym_nvs = sec->nvs;
                h->sym_vmap = sec->vmap;
                r = fl::plan_symmetry(h->plan[0], sec->K, sec->nvs, h->sym_vmap, err);
            }
            if (r == FL_OK) h->planned[0] = true;
        }
    } catch (const std::bad_alloc&) {
        r = FL_ENOMEM;
        err = "out of host memory in the planner";
    }
    if (r != FL_OK) {
        g_create_err = err;
        delete h;
        return r;
    }
    *out = h;
    return FL_OK;
}

int fl_create(fl_handle* out, int dim, int64_t n_vertices, const double* vertices_host, int64_t n_cells,
              const int32_t* cells_host, int dof_mode, const fl_options* opt) {
    return create_impl(out, dim, n_vertices, vertices_host, n_cells, cells_host, dof_mode, opt, nullptr);
}

int fl_create_sector(fl_handle* out, int64_t n_vertices, const double* vertices_host, int64_t n_cells,
                     const int32_t* cells_host, int K, const fl_options* opt) {
    g_create_err.clear();
    if (!out || !vertices_host || !cells_host || n_vertices < 3 || n_cells < 1) {
        g_create_err = "NULL pointer or empty sector mesh";
        return FL_EINVAL;
    }
    if (K < 2 || K > 64) {
        g_create_err = "K must lie in [2, 64]";
        return FL_EINVAL;
    }
    for (int64_t i = 0; i < 3 * n_cells; ++i)
        if (cells_host[i] < 0 || cells_host[i] >= n_vertices) {
            g_create_err = "cell vertex index out of range";
            return FL_EINVAL;
        }
    SectorArgs sec;
    sec.K = K;
    sec.nvs = n_vertices;
    std::vector<double> W;
    std::vector<int32_t> CW;
    try {
        fl::replicate_sector(n_vertices, vertices_host, n_cells, cells_host, K, W, CW, sec.vmap);
    } catch (const std::bad_alloc&) {
        g_create_err = "out of host memory";
        return FL_ENOMEM;
    }
    // the sector must be the wedge 0 <= phi <= 2 pi / K, and each vertex on its second ray must
    // meet the rotated image of one on its first ray
    {
        const double wedge = 2.0 * M_PI / K;
        std::vector<char> hit(W.size() / 2, 0);
        for (int64_t u = 0; u < n_vertices; ++u) hit[sec.vmap[(size_t)n_vertices + u]] = 1;  // copy 1
        int64_t n_first = 0, n_second = 0;
        for (int64_t v = 0; v < n_vertices; ++v) {
            const double x = vertices_host[2 * v], y = vertices_host[2 * v + 1];
            const double r = std::hypot(x, y);
            if (r < 1e-12) continue;
            n_first += std::fabs(std::atan2(y, x)) < 1e-9;
            n_second += std::fabs(std::atan2(y, x) - wedge) < 1e-9;
            const double phi = std::atan2(y, x);
            if (phi < -1e-9 || phi > wedge + 1e-9) {
                g_create_err = "a vertex outside the wedge 0 <= phi <= 2 pi / K";
                return FL_EINVAL;
            }
            if (std::fabs(phi - wedge) < 1e-9 && !hit[sec.vmap[v]]) {
                g_create_err = "a vertex on the ray phi = 2 pi / K without the rotated image of one on phi = 0";
                return FL_EINVAL;
            }
        }
        if (n_first == 0 || n_first != n_second) {
            g_create_err = "the sector's two rays carry different numbers of vertices (not a wedge of angle 2 pi / K?)";
            return FL_EINVAL;
        }
    }
    return create_impl(out, 2, (int64_t)W.size() / 2, W.data(), (int64_t)CW.size() / 3, CW.data(), FL_DOF_INTERIOR,
                       opt, &sec);
}

void fl_destroy(fl_handle h) {
    if (!h) return;
    if (!h->bufs.empty() || h->solve_ws || h->batch_ws || h->batch_host || h->sf_ws || h->sym_ws) {
        cudaSetDevice(h->device);
        cudaDeviceSynchronize();
        for (auto& b : h->bufs) fl::pool_dev_free(b.p);  // back to the cache (the device is idle)
        if (h->ev_made)
            for (int k = 0; k < 2 * FL_NSTAGES; ++k) cudaEventDestroy(h->ev[k]);
        if (h->solve_ws) fl::pool_dev_free(h->solve_ws);
        if (h->solve_host) fl::pool_host_free(h->solve_host);
        if (h->batch_ws) fl::pool_dev_free(h->batch_ws);
        if (h->batch_host) fl::pool_host_free(h->batch_host);
        if (h->sf_ws) fl::pool_dev_free(h->sf_ws);
        if (h->sym_ws) fl::pool_dev_free(h->sym_ws);
    }
    for (auto& g : h->cg_graphs) cudaGraphExecDestroy(g.exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->side) {
        cudaSetDevice(h->device);
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_far) cudaEventDestroy(h->ev_far);
    delete h;
}

const char* fl_last_error(fl_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int fl_num_dofs(fl_handle h, double s, int64_t* n) {
    if (!h || !n) return FL_EINVAL;
    int pi = fl::plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    *n = h->plan[pi].sym_K ? h->plan[pi].n_red : h->plan[pi].n;
    return FL_OK;
}

int fl_dof_vertices(fl_handle h, double s, int32_t* vod) {
    if (!h || !vod) return FL_EINVAL;
    int pi = fl::plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const auto& P = h->plan[pi];
    if (P.sym_K) {
        for (int64_t r = 0; r < P.n_red; ++r) vod[r] = P.red_vertex[r];
        return FL_OK;
    }
    for (int64_t i = 0; i < P.n; ++i) vod[i] = P.vod[i];
    return FL_OK;
}

int fl_assemble(fl_handle h, double s, int precision, double* A_dev, int64_t lda, void* stream) {
    if (!h) return FL_EINVAL;
    h->err.clear();
    try {
        return fl::assemble(h, s, precision, A_dev, lda, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_tune_assemble(fl_handle h, double s, double* A_dev, int64_t lda, int reps, int* best_variant, double* best_ms,
                     void* stream) {
    if (!h) return FL_EINVAL;
    h->err.clear();
    try {
        return fl::tune_assemble(h, s, A_dev, lda, reps, best_variant, best_ms, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_set_far_variant(fl_handle h, int variant) {
    if (!h) return FL_EINVAL;
    if (variant < 0 || variant > 4) return fl::set_err(h, FL_EINVAL, "variant must lie in 0..4");
    h->far_variant = variant;
    return FL_OK;
}

int fl_assemble_nearfield_csr(fl_handle h, double s, int precision, int64_t* nnz, int32_t* rowptr_dev,
                              int32_t* col_dev, double* val_dev, void* stream) {
    if (!h) return FL_EINVAL;
    if (h->sym_K) return fl::sym_unsupported(h, "fl_assemble_nearfield_csr");
    h->err.clear();
    try {
        return fl::assemble_nearfield_csr(h, s, precision, nnz, rowptr_dev, col_dev, val_dev, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_heat_matrix(fl_handle h, double s, double dt, const double* A_dev, int64_t lda, double* H_dev, int64_t ldh,
                   void* stream) {
    if (!h) return FL_EINVAL;
    if (h->sym_K) return fl::sym_unsupported(h, "fl_heat_matrix");
    h->err.clear();
    try {
        return fl::heat_matrix(h, s, dt, A_dev, lda, H_dev, ldh, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_mass_apply(fl_handle h, double s, int nrhs, double alpha, const double* X_dev, int64_t ldx, double beta,
                  const double* B_dev, int64_t ldb, double* Y_dev, int64_t ldy, void* stream) {
    if (!h) return FL_EINVAL;
    if (h->sym_K) return fl::sym_unsupported(h, "fl_mass_apply");
    h->err.clear();
    try {
        return fl::mass_apply(h, s, nrhs, alpha, X_dev, ldx, beta, B_dev, ldb, Y_dev, ldy, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_strong_form(fl_handle h, double s, const double* u_dev, int k_cell, int k_edge, int k_near, double* S_dev,
                   void* stream) {
    if (!h) return FL_EINVAL;
    if (h->sym_K) return fl::sym_unsupported(h, "fl_strong_form");
    h->err.clear();
    try {
        return fl::strong_form(h, s, u_dev, k_cell, k_edge, k_near, S_dev, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_br_indicators(fl_handle h, double s, const double* u_dev, const double* f_nodal_dev, int k_cell, int k_edge,
                     int k_near, double* eta_dev, double* S_dev, void* stream) {
    if (!h) return FL_EINVAL;
    if (h->sym_K) return fl::sym_unsupported(h, "fl_br_indicators");
    h->err.clear();
    try {
        return fl::br_indicators(h, s, u_dev, f_nodal_dev, k_cell, k_edge, k_near, eta_dev, S_dev,
                                 (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fl::set_err(h, FL_ENOMEM, "out of host memory");
    }
}

int fl_mark_max(fl_handle h, double s, const double* eta_dev, double theta, uint8_t* dof_marks_dev,
                uint8_t* cell_marks_dev, void* stream) {
    if (!h) return FL_EINVAL;
    if (h->sym_K) return fl::sym_unsupported(h, "fl_mark_max");
    h->err.clear();
    return fl::mark_max(h, s, eta_dev, theta, dof_marks_dev, cell_marks_dev, (cudaStream_t)stream);
}

int fl_refine(int dim, int64_t n_vertices, const double* vertices, int64_t n_cells, const int32_t* cells,
              const uint8_t* cell_marks, int64_t cap_vertices, int64_t cap_cells, double* vertices_out,
              int32_t* cells_out, int64_t* n_vertices_out, int64_t* n_cells_out) {
    std::string err;
    int r;
    try {
        r = fl::refine_mesh(dim, n_vertices, vertices, n_cells, cells, cell_marks, cap_vertices, cap_cells,
                            vertices_out, cells_out, n_vertices_out, n_cells_out, err);
    } catch (const std::bad_alloc&) {
        r = FL_ENOMEM;
        err = "out of host memory in fl_refine";
    }
    if (r != FL_OK) g_create_err = err;
    return r;
}

int fl_load_vector(fl_handle h, double s, const double* f_nodal_dev, int nrhs, double* b_dev, int64_t ldb,
                   void* stream) {
    if (!h) return FL_EINVAL;
    h->err.clear();
    return fl::load_vector(h, s, f_nodal_dev, nrhs, b_dev, ldb, (cudaStream_t)stream);
}

int fl_get_stats(fl_handle h, double s, fl_stats* st) {
    if (!h || !st) return FL_EINVAL;
    int pi = fl::plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const fl::Plan& P = h->plan[pi];
    fl_stats o{};
    o.n_cells = P.nc;
    o.n_vertices = P.nv;
    o.n_facets = P.nf;
    o.n_dofs = P.sym_K ? P.n_red : P.n;
    o.n_tiles = fl::plan_tile_count(P);
    o.n_touch_pairs = (int64_t)P.tp_type.size();
    o.n_near_pairs = (int64_t)P.np_a.size();
    int64_t nd = 0;
    for (char c : P.hasdof) nd += c ? 1 : 0;
    o.n_cells_with_dof = nd;
    const int64_t nodof = P.nc - nd;
    const int64_t all = P.nc * (P.nc - 1) / 2 - nodof * (nodof - 1) / 2;
    o.n_far_pairs = all - o.n_touch_pairs - o.n_near_pairs;
    o.nnz_nearfield = (int64_t)P.csr_col.size();
    o.h2d_bytes = h->h2d_bytes;
    o.workspace_bytes = h->ws_bytes + (int64_t)h->solve_ws_bytes + (int64_t)h->batch_ws_bytes;
    *st = o;
    return FL_OK;
}

int fl_set_profiling(fl_handle h, int enable) {
    if (!h) return FL_EINVAL;
    if (enable < 0 || enable > 2) return fl::set_err(h, FL_EINVAL, "enable must be 0, 1 or 2");
    h->profiling = enable;
    h->ev_recorded = false;
    return FL_OK;
}

int fl_stage_ms(fl_handle h, double* ms) {
    if (!h || !ms) return FL_EINVAL;
    if (!h->ev_recorded) return fl::set_err(h, FL_EINVAL, "no profiled fl_assemble yet");
    const int last = h->profiling == 2 ? FL_STAGE_FAR : FL_NSTAGES - 1;
    if (cudaEventSynchronize(h->ev[2 * last + 1]) != cudaSuccess)
        return fl::set_err(h, FL_ECUDA, "cudaEventSynchronize");
    for (int i = 0; i < FL_NSTAGES; ++i) {
        float t = 0.f;
        if (h->profiling == 2 && i != FL_STAGE_FAR) {
            ms[i] = 0.0;
            continue;
        }
        if (cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            t = 0.f;
        }
        ms[i] = (double)t;
    }
    return FL_OK;
}

uint64_t fl_launch_count(void) { return g_launches.load(); }

}  // extern "C"
