// Galerkin multigrid on nested P1 spaces.  Section 5 proposes multigrid for the
// dense systems without an algorithm; this is the textbook V-cycle:
//   * prolongation P_ij = phi_j^coarse(x_i) (coarse hat functions at the fine DOF
//     vertices, located in the coarse mesh by a bucket grid; exact for nested spaces),
//   * coarse operators A_c = P^T A P, formed on the device in float64,
//   * damped Jacobi smoothing x += w D^-1 (r - A x), w = 4 / (3 lambda), lambda from ten
//     power-iteration steps on D^-1 A started at (1, ..., 1),
//   * an explicit inverse of the coarsest operator (Gauss-Jordan on the device),
//   * the cycle itself in float32 on float32 copies of the level operators.
// fl_mg_solve runs float64 conjugate gradients preconditioned by one V-cycle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "device.h"

namespace fl {
namespace mg {

struct Level {
    int64_t n = 0;
    const double* A64 = nullptr;  // level operator (level 0: the caller's matrix)
    int64_t lda = 0;
    double* A64_own = nullptr;    // owned storage of the coarse operators
    float* A32 = nullptr;         // float32 copy, row pitch ld32 (a multiple of 4)
    int64_t ld32 = 0;
    float* dinv = nullptr;        // w / a_ii
    float omega = 0.f;
    // prolongation from the next coarser level into this one (rows: this level's DOFs)
    int64_t nc = 0;
    int *p_ptr = nullptr, *p_col = nullptr;
    float* p_val = nullptr;
    int *pt_ptr = nullptr, *pt_col = nullptr;  // its transpose (rows: coarse DOFs)
    float* pt_val = nullptr;
    double* pt_val64 = nullptr;
    float *x = nullptr, *r = nullptr, *t = nullptr;  // cycle vectors
};

}  // namespace mg
}  // namespace fl

struct fl_mg {
    int device = 0;
    std::vector<fl::mg::Level> lv;
    std::vector<void*> owned;     // every device allocation of the hierarchy
    float* cinv = nullptr;        // inverse of the coarsest operator (float32, nc x nc)
    int nu = 2;
    bool ready = false;
    std::string err;
    double* sw = nullptr;         // solver workspace (float64 vectors and partial sums)
    size_t sw_n = 0;
    double* hsc = nullptr;        // pinned scalars
};

namespace fl {
namespace mg {

constexpr int RB = 256;  // reduction blocks

static int fail(fl_mg* m, int code, const std::string& msg) {
    m->err = msg;
    return code;
}

template <typename T>
static T* dalloc(fl_mg* m, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    m->owned.push_back(p);
    return (T*)p;
}

// ---------------------------------------------------------------- kernels --
// AP[i][j] = sum_{(k, w) in P^T row j} A[i][k] w; block per fine row i
__global__ void ap_kernel(int64_t nf, int64_t nc, const double* __restrict__ A, int64_t lda,
                          const int* __restrict__ pt_ptr, const int* __restrict__ pt_col,
                          const double* __restrict__ pt_val, double* __restrict__ AP) {
    for (int64_t i = blockIdx.x; i < nf; i += gridDim.x) {
        const double* Ai = A + i * lda;
        for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
            double acc = 0.0;
            for (int e = pt_ptr[j]; e < pt_ptr[j + 1]; ++e) acc = fma(__ldg(Ai + pt_col[e]), pt_val[e], acc);
            AP[i * nc + j] = acc;
        }
    }
}

// Ac[j][l] = sum_{(k, w) in P^T row j} w AP[k][l]; block per coarse row j
__global__ void ptap_kernel(int64_t nc, const double* __restrict__ AP, const int* __restrict__ pt_ptr,
                            const int* __restrict__ pt_col, const double* __restrict__ pt_val,
                            double* __restrict__ Ac) {
    for (int64_t j = blockIdx.x; j < nc; j += gridDim.x) {
        for (int64_t l = threadIdx.x; l < nc; l += blockDim.x) {
            double acc = 0.0;
            for (int e = pt_ptr[j]; e < pt_ptr[j + 1]; ++e) acc = fma(pt_val[e], AP[(int64_t)pt_col[e] * nc + l], acc);
            Ac[j * nc + l] = acc;
        }
    }
}

__global__ void f32_copy_kernel(int64_t n, const double* A, int64_t lda, float* B, int64_t ldb) {
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ldb; j += (int64_t)gridDim.x * blockDim.x)
            B[i * ldb + j] = (j < n) ? (float)A[i * lda + j] : 0.f;
}

__global__ void diag_kernel(int64_t n, const double* A, int64_t lda, double* d) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = A[i * lda + i];
}

// deterministic partial sums of x.y (grid-stride, fixed block count), then one block adds them
__global__ void dot_part_kernel(int64_t n, const double* a, const double* b, double* part) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}
__global__ void dot_sum_kernel(const double* part, int nb, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nb; ++i) t += part[i];
        *out = t;
    }
}

// x = y / sqrt(*nrm2)
__global__ void scale_kernel(int64_t n, const double* y, const double* nrm2, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = y[i] / sqrt(*nrm2);
}

// ---- preconditioned CG (float64) ----
// x += a p; r -= a q with a = rz / pq read on the device
__global__ void cg_xr_kernel(int64_t n, const double* sc, double* x, double* r, const double* p, const double* q) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = sc[0] / sc[1];
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
}
// p = z + (rz_new / rz) p
__global__ void cg_p_kernel(int64_t n, const double* sc, const double* z, double* p) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = fma(sc[2] / sc[0], p[i], z[i]);
}

// x := y / d (element-wise)
__global__ void div_kernel(int64_t n, const double* y, const double* d, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = y[i] / d[i];
}

__global__ void fill_kernel(int64_t n, double v, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void dinv_kernel(int64_t n, const double* d, float omega, float* dinv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = (float)(omega / d[i]);
}

// Gauss-Jordan inversion step k (no pivoting; the operators are SPD): save row and column k
__global__ void gj_save_kernel(int64_t n, const double* M, int64_t k, double* colk, double* rowk) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        colk[i] = M[i * n + k];
        rowk[i] = M[k * n + i];
    }
}
__global__ void gj_update_kernel(int64_t n, double* M, int64_t k, const double* colk, const double* rowk) {
    const double piv = rowk[k];
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
            double v;
            if (i == k && j == k) v = 1.0 / piv;
            else if (i == k) v = rowk[j] / piv;
            else if (j == k) v = -colk[i] / piv;
            else v = M[i * n + j] - colk[i] * rowk[j] / piv;
            M[i * n + j] = v;
        }
    }
}

// ---- V-cycle (float32) ----
// y = A x, warp per row, 16-byte loads (ld a multiple of 4, rows 16-byte aligned)
__global__ void gemv32_kernel(int64_t n, const float* __restrict__ A, int64_t ld, const float* __restrict__ x,
                              float* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float4* a = reinterpret_cast<const float4*>(A + row * ld);
    const float4* xv = reinterpret_cast<const float4*>(x);
    float s = 0.f;
    const int64_t nv = ld >> 2;
    for (int64_t k = lane; k < nv; k += 32) {
        const float4 av = __ldcs(a + k);
        const float4 b = __ldg(xv + k);
        s = fmaf(av.x, b.x, fmaf(av.y, b.y, fmaf(av.z, b.z, fmaf(av.w, b.w, s))));
    }
    s = warp_sum(s);
    if (lane == 0) y[row] = s;
}

// x = dinv .* r (first smoothing step from x = 0)
__global__ void smooth0_kernel(int64_t n, const float* dinv, const float* r, float* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = dinv[i] * r[i];
}
// x += dinv .* (r - y)
__global__ void smooth_kernel(int64_t n, const float* dinv, const float* r, const float* y, float* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = fmaf(dinv[i], r[i] - y[i], x[i]);
}
// rc[j] = sum_{(k, w) in P^T row j} w (r[k] - y[k])
__global__ void restrict_kernel(int64_t nc, const int* pt_ptr, const int* pt_col, const float* pt_val, const float* r,
                                const float* y, float* rc) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nc) return;
    float acc = 0.f;
    for (int e = pt_ptr[j]; e < pt_ptr[j + 1]; ++e) {
        const int k = pt_col[e];
        acc = fmaf(pt_val[e], r[k] - y[k], acc);
    }
    rc[j] = acc;
}
// x[i] += sum_{(j, w) in P row i} w xc[j]
__global__ void prolong_kernel(int64_t n, const int* p_ptr, const int* p_col, const float* p_val, const float* xc,
                               float* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = x[i];
    for (int e = p_ptr[i]; e < p_ptr[i + 1]; ++e) acc = fmaf(p_val[e], xc[p_col[e]], acc);
    x[i] = acc;
}
__global__ void d2f_kernel(int64_t n, const double* a, float* b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void f2d_kernel(int64_t n, const float* a, double* b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

static unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static void gemv32(const Level& L, const float* A, int64_t ld, int64_t n, const float* x, float* y,
                   cudaStream_t st) {
    (void)L;
    gemv32_kernel<<<nb(n * 32), 256, 0, st>>>(n, A, ld, x, y);
    fl::count_launch();
}

// One V-cycle on level l: lv[l].x = V(lv[l].r)
static void vcycle(fl_mg* m, size_t l, cudaStream_t st) {
    Level& L = m->lv[l];
    if (l + 1 == m->lv.size()) {
        gemv32(L, m->cinv, L.ld32, L.n, L.r, L.x, st);
        return;
    }
    Level& C = m->lv[l + 1];
    const unsigned g = nb(L.n);
    for (int k = 0; k < m->nu; ++k) {
        if (k == 0) {
            smooth0_kernel<<<g, 256, 0, st>>>(L.n, L.dinv, L.r, L.x);
        } else {
            gemv32(L, L.A32, L.ld32, L.n, L.x, L.t, st);
            smooth_kernel<<<g, 256, 0, st>>>(L.n, L.dinv, L.r, L.t, L.x);
        }
        fl::count_launch();
    }
    if (m->nu == 0) cudaMemsetAsync(L.x, 0, L.n * sizeof(float), st);
    gemv32(L, L.A32, L.ld32, L.n, L.x, L.t, st);
    restrict_kernel<<<nb(C.n), 256, 0, st>>>(C.n, L.pt_ptr, L.pt_col, L.pt_val, L.r, L.t, C.r);
    fl::count_launch();
    vcycle(m, l + 1, st);
    prolong_kernel<<<g, 256, 0, st>>>(L.n, L.p_ptr, L.p_col, L.p_val, C.x, L.x);
    fl::count_launch();
    for (int k = 0; k < m->nu; ++k) {
        gemv32(L, L.A32, L.ld32, L.n, L.x, L.t, st);
        smooth_kernel<<<g, 256, 0, st>>>(L.n, L.dinv, L.r, L.t, L.x);
        fl::count_launch();
    }
}

// ---------------------------------------------------- point location (host) --
struct Locator {
    int dim;
    const Plan* pc;
    double x0 = 0, y0 = 0, hx = 1, hy = 1;
    int G = 1;
    std::vector<int> b_ptr, b_cell;
    explicit Locator(const Plan& P) : dim(P.dim), pc(&P) {
        const int64_t nc = P.nc;
        if (dim == 1) return;
        double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
        for (int64_t v = 0; v < P.nv; ++v) {
            xmin = std::min(xmin, P.V[2 * v]);
            xmax = std::max(xmax, P.V[2 * v]);
            ymin = std::min(ymin, P.V[2 * v + 1]);
            ymax = std::max(ymax, P.V[2 * v + 1]);
        }
        G = std::max(1, (int)std::sqrt((double)nc));
        x0 = xmin;
        y0 = ymin;
        hx = std::max((xmax - xmin) / G, 1e-300);
        hy = std::max((ymax - ymin) / G, 1e-300);
        std::vector<int> cnt((size_t)G * G + 1, 0);
        auto range = [&](int64_t c, int& i0, int& i1, int& j0, int& j1) {
            double a0 = 1e300, a1 = -1e300, b0 = 1e300, b1 = -1e300;
            for (int k = 0; k < 3; ++k) {
                const int v = P.C[3 * c + k];
                a0 = std::min(a0, P.V[2 * v]);
                a1 = std::max(a1, P.V[2 * v]);
                b0 = std::min(b0, P.V[2 * v + 1]);
                b1 = std::max(b1, P.V[2 * v + 1]);
            }
            i0 = std::clamp((int)std::floor((a0 - x0) / hx) - 1, 0, G - 1);
            i1 = std::clamp((int)std::floor((a1 - x0) / hx) + 1, 0, G - 1);
            j0 = std::clamp((int)std::floor((b0 - y0) / hy) - 1, 0, G - 1);
            j1 = std::clamp((int)std::floor((b1 - y0) / hy) + 1, 0, G - 1);
        };
        for (int64_t c = 0; c < nc; ++c) {
            int i0, i1, j0, j1;
            range(c, i0, i1, j0, j1);
            for (int i = i0; i <= i1; ++i)
                for (int j = j0; j <= j1; ++j) ++cnt[(size_t)i * G + j + 1];
        }
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        b_ptr = cnt;
        b_cell.resize(cnt.back());
        std::vector<int> fillp(cnt.begin(), cnt.end() - 1);
        for (int64_t c = 0; c < nc; ++c) {
            int i0, i1, j0, j1;
            range(c, i0, i1, j0, j1);
            for (int i = i0; i <= i1; ++i)
                for (int j = j0; j <= j1; ++j) b_cell[fillp[(size_t)i * G + j]++] = (int)c;
        }
    }
    // coarse cell containing point x and its barycentric weights (vertex order of the cell)
    bool locate(const double* x, int& cell, double lam[3]) const {
        const Plan& P = *pc;
        if (dim == 1) {
            for (int64_t c = 0; c < P.nc; ++c) {
                const double a = P.V[P.C[2 * c]], b = P.V[P.C[2 * c + 1]];
                const double t = (x[0] - a) / (b - a);
                if (t >= -1e-12 && t <= 1 + 1e-12) {
                    cell = (int)c;
                    lam[0] = 1 - t;
                    lam[1] = t;
                    return true;
                }
            }
            return false;
        }
        const int i = std::clamp((int)std::floor((x[0] - x0) / hx), 0, G - 1);
        const int j = std::clamp((int)std::floor((x[1] - y0) / hy), 0, G - 1);
        const size_t bk = (size_t)i * G + j;
        for (int e = b_ptr[bk]; e < b_ptr[bk + 1]; ++e) {
            const int c = b_cell[e];
            const double* a = &P.V[2 * P.C[3 * c]];
            const double* b = &P.V[2 * P.C[3 * c + 1]];
            const double* d = &P.V[2 * P.C[3 * c + 2]];
            const double m00 = b[0] - a[0], m01 = d[0] - a[0], m10 = b[1] - a[1], m11 = d[1] - a[1];
            const double det = m00 * m11 - m01 * m10;
            const double rx = x[0] - a[0], ry = x[1] - a[1];
            const double l1 = (m11 * rx - m01 * ry) / det, l2 = (-m10 * rx + m00 * ry) / det;
            const double l0 = 1 - l1 - l2;
            if (l0 >= -1e-12 && l1 >= -1e-12 && l2 >= -1e-12) {
                cell = c;
                lam[0] = l0;
                lam[1] = l1;
                lam[2] = l2;
                return true;
            }
        }
        return false;
    }
};

}  // namespace mg
}  // namespace fl

namespace fl {
// z = V(r) for float64 vectors on the finest level (used by the flexible CG)
int mg_precondition(fl_mg_handle m, const double* r, double* z, cudaStream_t st) {
    if (!m || !m->ready) return FL_EINVAL;
    mg::Level& L = m->lv[0];
    const unsigned g = mg::nb(L.n);
    mg::d2f_kernel<<<g, 256, 0, st>>>(L.n, r, L.r);
    mg::vcycle(m, 0, st);
    mg::f2d_kernel<<<g, 256, 0, st>>>(L.n, L.x, z);
    fl::count_launch(2);
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}
}  // namespace fl

using namespace fl;
using namespace fl::mg;

extern "C" {

int fl_prolongation(fl_handle fine, fl_handle coarse, double s, int64_t* nnz, int32_t* rowptr, int32_t* col,
                    double* val) {
    if (!fine || !coarse || !nnz) return FL_EINVAL;
    if (fine->sym_K || coarse->sym_K) return sym_unsupported(fine->sym_K ? fine : coarse, "fl_prolongation");
    if (fine->dim != coarse->dim) return set_err(fine, FL_EINVAL, "meshes of different dimension");
    const int pf = plan_for(fine, s), pc = plan_for(coarse, s);
    if (pf < 0) return FL_EINVAL;
    if (pc < 0) return set_err(fine, FL_EINVAL, "coarse mesh: " + coarse->err);
    const Plan& F = fine->plan[pf];
    const Plan& C = coarse->plan[pc];
    const int nvpc = C.dim + 1;
    Locator loc(C);
    std::vector<int32_t> ptr(F.n + 1, 0), cols;
    std::vector<double> vals;
    for (int64_t i = 0; i < F.n; ++i) {
        const double* x = &F.V[(size_t)F.vod[i] * F.dim];
        int cell;
        double lam[3] = {0, 0, 0};
        if (!loc.locate(x, cell, lam))
            return set_err(fine, FL_EINVAL, "fine vertex " + std::to_string(F.vod[i]) + " lies in no coarse cell");
        for (int k = 0; k < nvpc; ++k) {
            const int j = C.dov[C.C[(size_t)cell * nvpc + k]];
            if (j >= 0 && std::fabs(lam[k]) > 1e-15) {
                cols.push_back(j);
                vals.push_back(lam[k]);
            }
        }
        ptr[i + 1] = (int32_t)cols.size();
    }
    *nnz = (int64_t)cols.size();
    if (rowptr) std::memcpy(rowptr, ptr.data(), ptr.size() * sizeof(int32_t));
    if (col) std::memcpy(col, cols.data(), cols.size() * sizeof(int32_t));
    if (val) std::memcpy(val, vals.data(), vals.size() * sizeof(double));
    return FL_OK;
}

int fl_mg_create(fl_mg_handle* out, const double* A_dev, int64_t lda, int64_t n) {
    if (!out || !A_dev || n < 1 || lda < n) return FL_EINVAL;
    fl_mg* m = new (std::nothrow) fl_mg;
    if (!m) return FL_ENOMEM;
    cudaGetDevice(&m->device);
    Level L;
    L.n = n;
    L.A64 = A_dev;
    L.lda = lda;
    m->lv.push_back(L);
    *out = m;
    return FL_OK;
}

const char* fl_mg_last_error(fl_mg_handle m) { return m ? m->err.c_str() : ""; }

int fl_mg_add_level(fl_mg_handle m, int64_t nc, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                    const double* val, void* stream) {
    if (!m || nc < 1 || nnz < 0 || !rowptr || !col || !val) return FL_EINVAL;
    if (m->ready) return fail(m, FL_EINVAL, "hierarchy already set up");
    cudaStream_t st = (cudaStream_t)stream;
    Level& F = m->lv.back();
    const int64_t nf = F.n;
    if (rowptr[0] != 0 || rowptr[nf] != nnz) return fail(m, FL_EINVAL, "prolongation rows do not match the level");
    std::vector<int> pt_cnt(nc + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) {
        if (col[e] < 0 || col[e] >= nc) return fail(m, FL_EINVAL, "prolongation column out of range");
        ++pt_cnt[col[e] + 1];
    }
    for (int64_t j = 0; j < nc; ++j) pt_cnt[j + 1] += pt_cnt[j];
    std::vector<int> pt_col(nnz);
    std::vector<double> pt_val(nnz);
    std::vector<float> pval(nnz), ptval(nnz);
    std::vector<int> fillp(pt_cnt.begin(), pt_cnt.end() - 1);
    for (int64_t i = 0; i < nf; ++i)
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int q = fillp[col[e]]++;
            pt_col[q] = (int)i;
            pt_val[q] = val[e];
            ptval[q] = (float)val[e];
        }
    for (int64_t e = 0; e < nnz; ++e) pval[e] = (float)val[e];
    F.nc = nc;
    F.p_ptr = dalloc<int>(m, nf + 1);
    F.p_col = dalloc<int>(m, std::max<int64_t>(nnz, 1));
    F.p_val = dalloc<float>(m, std::max<int64_t>(nnz, 1));
    F.pt_ptr = dalloc<int>(m, nc + 1);
    F.pt_col = dalloc<int>(m, std::max<int64_t>(nnz, 1));
    F.pt_val = dalloc<float>(m, std::max<int64_t>(nnz, 1));
    F.pt_val64 = dalloc<double>(m, std::max<int64_t>(nnz, 1));
    double* Ac = dalloc<double>(m, (size_t)nc * nc);
    double* AP = nullptr;
    if (cudaMalloc((void**)&AP, (size_t)nf * nc * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        AP = nullptr;
    }
    if (!F.p_ptr || !F.p_col || !F.p_val || !F.pt_ptr || !F.pt_col || !F.pt_val || !F.pt_val64 || !Ac || !AP) {
        if (AP) cudaFree(AP);
        return fail(m, FL_ENOMEM, "multigrid level");
    }
    cudaMemcpyAsync(F.p_ptr, rowptr, (nf + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.p_col, col, nnz * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.p_val, pval.data(), nnz * sizeof(float), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.pt_ptr, pt_cnt.data(), (nc + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.pt_col, pt_col.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.pt_val, ptval.data(), nnz * sizeof(float), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.pt_val64, pt_val.data(), nnz * sizeof(double), cudaMemcpyHostToDevice, st);
    ap_kernel<<<(unsigned)std::min<int64_t>(nf, 65535), 256, 0, st>>>(nf, nc, F.A64, F.lda, F.pt_ptr, F.pt_col,
                                                                       F.pt_val64, AP);
    ptap_kernel<<<(unsigned)std::min<int64_t>(nc, 65535), 256, 0, st>>>(nc, AP, F.pt_ptr, F.pt_col, F.pt_val64, Ac);
    fl::count_launch(2);
    const cudaError_t e1 = cudaStreamSynchronize(st);  // host vectors above must outlive the copies
    cudaFree(AP);
    if (e1 != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(m, FL_ECUDA, "Galerkin product");
    Level C;
    C.n = nc;
    C.A64 = Ac;
    C.A64_own = Ac;
    C.lda = nc;
    m->lv.push_back(C);
    return FL_OK;
}

int fl_mg_setup(fl_mg_handle m, int nu, void* stream) {
    if (!m || nu < 0 || nu > 8) return FL_EINVAL;
    if (m->ready) return FL_OK;
    if (m->lv.size() < 2) return fail(m, FL_EINVAL, "add at least one coarse level");
    cudaStream_t st = (cudaStream_t)stream;
    m->nu = nu;
    int64_t nmax = 0;
    for (Level& L : m->lv) nmax = std::max(nmax, L.n);
    double* d = dalloc<double>(m, nmax);
    double* x = dalloc<double>(m, nmax);
    double* y = dalloc<double>(m, nmax);
    double* part = dalloc<double>(m, RB + 1);
    double* h = nullptr;
    if (!d || !x || !y || !part || cudaMallocHost((void**)&h, sizeof(double)) != cudaSuccess)
        return fail(m, FL_ENOMEM, "multigrid setup");
    for (size_t l = 0; l < m->lv.size(); ++l) {
        Level& L = m->lv[l];
        const int64_t n = L.n;
        L.ld32 = (n + 3) / 4 * 4;
        L.x = dalloc<float>(m, L.ld32);
        L.r = dalloc<float>(m, L.ld32);
        L.t = dalloc<float>(m, L.ld32);
        if (!L.x || !L.r || !L.t) {
            cudaFreeHost(h);
            return fail(m, FL_ENOMEM, "multigrid vectors");
        }
        cudaMemsetAsync(L.x, 0, L.ld32 * sizeof(float), st);
        cudaMemsetAsync(L.r, 0, L.ld32 * sizeof(float), st);
        cudaMemsetAsync(L.t, 0, L.ld32 * sizeof(float), st);
        const bool coarsest = (l + 1 == m->lv.size());
        if (!coarsest) {
            L.A32 = dalloc<float>(m, (size_t)n * L.ld32);
            L.dinv = dalloc<float>(m, n);
            if (!L.A32 || !L.dinv) {
                cudaFreeHost(h);
                return fail(m, FL_ENOMEM, "multigrid level copy");
            }
            f32_copy_kernel<<<dim3(nb(L.ld32), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, st>>>(
                n, L.A64, L.lda, L.A32, L.ld32);
            diag_kernel<<<nb(n), 256, 0, st>>>(n, L.A64, L.lda, d);
            fill_kernel<<<nb(n), 256, 0, st>>>(n, 1.0, x);
            fl::count_launch(3);
            // ten steps of x <- D^-1 A x / ||D^-1 A x||, then lambda = ||D^-1 A x|| / ||x||
            for (int k = 0; k <= 10; ++k) {
                if (fl::gemv(FL_F64, L.A64, L.lda, n, x, 1, y, 1, nullptr, st) != cudaSuccess) {
                    cudaFreeHost(h);
                    return fail(m, FL_ECUDA, "power iteration");
                }
                div_kernel<<<nb(n), 256, 0, st>>>(n, y, d, y);
                dot_part_kernel<<<RB, 256, 0, st>>>(n, y, y, part);
                dot_sum_kernel<<<1, 32, 0, st>>>(part, RB, part + RB);
                fl::count_launch(3);
                if (k == 10) {
                    double yy = 0, xx = 0;
                    cudaMemcpyAsync(&yy, part + RB, sizeof(double), cudaMemcpyDeviceToHost, st);
                    dot_part_kernel<<<RB, 256, 0, st>>>(n, x, x, part);
                    dot_sum_kernel<<<1, 32, 0, st>>>(part, RB, part + RB);
                    fl::count_launch(2);
                    cudaMemcpyAsync(h, part + RB, sizeof(double), cudaMemcpyDeviceToHost, st);
                    if (cudaStreamSynchronize(st) != cudaSuccess) {
                        cudaFreeHost(h);
                        return fail(m, FL_ECUDA, "power iteration");
                    }
                    xx = *h;
                    L.omega = (float)(4.0 / (3.0 * std::sqrt(yy / xx)));
                } else {
                    scale_kernel<<<nb(n), 256, 0, st>>>(n, y, part + RB, x);
                    fl::count_launch();
                }
            }
            dinv_kernel<<<nb(n), 256, 0, st>>>(n, d, L.omega, L.dinv);
            fl::count_launch();
        } else {
            // explicit inverse of the coarsest operator
            double* M = dalloc<double>(m, (size_t)n * n);
            m->cinv = dalloc<float>(m, (size_t)n * L.ld32);
            if (!M || !m->cinv) {
                cudaFreeHost(h);
                return fail(m, FL_ENOMEM, "coarse inverse");
            }
            cudaMemcpy2DAsync(M, n * sizeof(double), L.A64, L.lda * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, st);
            const dim3 gg(nb(n), (unsigned)std::min<int64_t>(n, 1024));
            for (int64_t k = 0; k < n; ++k) {
                gj_save_kernel<<<nb(n), 256, 0, st>>>(n, M, k, x, y);
                gj_update_kernel<<<gg, 256, 0, st>>>(n, M, k, x, y);
            }
            fl::count_launch((int)(2 * n));
            f32_copy_kernel<<<dim3(nb(L.ld32), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, st>>>(
                n, M, n, m->cinv, L.ld32);
            fl::count_launch();
        }
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaFreeHost(h);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(m, FL_ECUDA, "multigrid setup");
    m->ready = true;
    return FL_OK;
}

int fl_mg_level(fl_mg_handle m, int level, int64_t* n, const double** A_dev, int64_t* lda) {
    if (!m || level < 0 || level >= (int)m->lv.size()) return FL_EINVAL;
    if (n) *n = m->lv[level].n;
    if (A_dev) *A_dev = m->lv[level].A64;
    if (lda) *lda = m->lv[level].lda;
    return FL_OK;
}

int fl_mg_level_copy(fl_mg_handle m, int level, double* dst_dev, int64_t ldd, void* stream) {
    if (!m || !dst_dev || level < 0 || level >= (int)m->lv.size() || ldd < m->lv[level].n) return FL_EINVAL;
    const Level& L = m->lv[level];
    return cudaMemcpy2DAsync(dst_dev, ldd * sizeof(double), L.A64, L.lda * sizeof(double), L.n * sizeof(double), L.n,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream) == cudaSuccess
               ? FL_OK
               : fail(m, FL_ECUDA, "copy");
}

int fl_mg_omega(fl_mg_handle m, int level, float* omega) {
    if (!m || !omega || level < 0 || level >= (int)m->lv.size()) return FL_EINVAL;
    *omega = m->lv[level].omega;
    return FL_OK;
}

int fl_mg_vcycle(fl_mg_handle m, const float* r_dev, float* z_dev, void* stream) {
    if (!m || !r_dev || !z_dev) return FL_EINVAL;
    if (!m->ready) return fail(m, FL_EINVAL, "fl_mg_setup first");
    cudaStream_t st = (cudaStream_t)stream;
    Level& L = m->lv[0];
    cudaMemcpyAsync(L.r, r_dev, L.n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    vcycle(m, 0, st);
    cudaMemcpyAsync(z_dev, L.x, L.n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError() == cudaSuccess ? FL_OK : fail(m, FL_ECUDA, "V-cycle");
}

int fl_mg_solve(fl_mg_handle m, const double* b_dev, double* u_dev, double tol, int maxit, fl_solve_info* info,
                void* stream) {
    if (!m || !b_dev || !u_dev || !(tol > 0) || maxit < 1) return FL_EINVAL;
    if (!m->ready) return fail(m, FL_EINVAL, "fl_mg_setup first");
    cudaStream_t st = (cudaStream_t)stream;
    Level& L = m->lv[0];
    const int64_t n = L.n;
    // workspace: r, z, p, q (float64), partial sums, 4 scalars [rz, pq, rz_new, rr]
    const size_t need = 4 * (size_t)n + RB + 8;
    if (m->sw_n < need) {
        if (m->sw) cudaFree(m->sw);
        m->sw = nullptr;
        m->sw_n = 0;
        if (cudaMalloc((void**)&m->sw, need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(m, FL_ENOMEM, "solver workspace");
        }
        m->sw_n = need;
    }
    if (!m->hsc && cudaMallocHost((void**)&m->hsc, 8 * sizeof(double)) != cudaSuccess)
        return fail(m, FL_ENOMEM, "pinned scalars");
    double *r = m->sw, *z = r + n, *p = z + n, *q = p + n, *part = q + n, *sc = part + RB;
    const unsigned g = nb(n);
    auto dot = [&](const double* a, const double* b, double* out) {
        dot_part_kernel<<<RB, 256, 0, st>>>(n, a, b, part);
        dot_sum_kernel<<<1, 32, 0, st>>>(part, RB, out);
        fl::count_launch(2);
    };
    auto precond = [&](const double* rin, double* zout) {
        d2f_kernel<<<g, 256, 0, st>>>(n, rin, L.r);
        fl::count_launch();
        vcycle(m, 0, st);
        f2d_kernel<<<g, 256, 0, st>>>(n, L.x, zout);
        fl::count_launch();
    };
    cudaMemsetAsync(u_dev, 0, n * sizeof(double), st);
    cudaMemcpyAsync(r, b_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    dot(r, r, sc + 3);
    cudaMemcpyAsync(m->hsc + 3, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st);
    precond(r, z);
    cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    dot(r, z, sc + 0);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(m, FL_ECUDA, "solve start");
    const double bb = m->hsc[3];
    double rr = bb;
    int it = 0, status = FL_ENOTCONV;
    if (bb == 0.0) status = FL_OK;
    while (status == FL_ENOTCONV && it < maxit) {
        if (fl::gemv(FL_F64, L.A64, L.lda, n, p, 1, q, 1, nullptr, st) != cudaSuccess)
            return fail(m, FL_ECUDA, "matvec");
        dot(p, q, sc + 1);
        cg_xr_kernel<<<g, 256, 0, st>>>(n, sc, u_dev, r, p, q);
        fl::count_launch();
        dot(r, r, sc + 3);
        precond(r, z);
        dot(r, z, sc + 2);
        cg_p_kernel<<<g, 256, 0, st>>>(n, sc, z, p);
        fl::count_launch();
        cudaMemcpyAsync(m->hsc, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(sc, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, st);  // rz <- rz_new
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(m, FL_ECUDA, "solve step");
        ++it;
        if (!(m->hsc[1] > 0.0)) {
            status = FL_ENOTSPD;
            break;
        }
        rr = m->hsc[3];
        if (rr <= tol * tol * bb) status = FL_OK;
    }
    if (info) {
        info->iterations = it;
        info->outer_iterations = 1;
        info->rel_residual = bb > 0 ? std::sqrt(rr / bb) : 0.0;
        info->status = status;
    }
    return status;
}

void fl_mg_destroy(fl_mg_handle m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    for (void* p : m->owned) cudaFree(p);
    if (m->sw) cudaFree(m->sw);
    if (m->hsc) cudaFreeHost(m->hsc);
    delete m;
}

}  // extern "C"
