// Cluster-method (H-matrix) approximation of the stiffness matrix and its product
// (Section 6 of arXiv:1708.03912).
//
// On an admissible pair of clusters (sigma, tau) the supports are disjoint and
// a(phi_i, phi_j) = -C(d,s) int int k(x,y) phi_i(x) phi_j(y); the kernel
// k = |x-y|^{-d-2s} is replaced by its tensor Chebyshev interpolant of order m on the two
// cluster cubes, sum_{alpha,beta} k(xi_alpha^sigma, xi_beta^tau) L_alpha^sigma(x) L_beta^tau(y).
// The product y = A x then splits into
//   near field   y_i += sum_j A_ij x_j over the inadmissible leaf pairs (exact entries, CSR);
//   upward pass  xh_c = sum_{i in c} (int phi_i L_alpha^c) x_i on the leaves (the basis
//                far-field coefficients, Gauss order m+1 per cell), and
//                xh_f = sum_sons S_son^T xh_son with the shift coefficients
//                S_son[beta][alpha] = L_alpha^f(xi_beta^son);
//   couplings    yh_sigma = sum over its admissible partners tau of K_{sigma tau} xh_tau;
//   downward     yh_son += S_son yh_f, and y_i += -C sum_alpha (int phi_i L_alpha) yh_leaf.
// Cluster tree and partition: cluster.cpp (host).  Every sum runs in a fixed order, so the
// product is bitwise reproducible; all arithmetic is float64.
// Schedule: the near-field product runs on a second stream beside the far-field chain; the
// passes take one launch per direction below a split level (one block per subtree walks all
// of its levels) and one above it (one block walks the top levels); the couplings are pair
// products followed by per-node sums; the whole product is captured once per (x, y) as a
// CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "cluster.h"
#include "context.h"
#include "device.h"

struct fl_hm {
    fl_ctx* mesh = nullptr;
    int device = 0, pi = 0, d = 0, m = 0, md = 0;
    double s = 0.0, C = 0.0;
    fl::ClusterPlan plan;
    std::vector<int> nz_ptr_h;  // near CSR row pointer (host copy, for sizes)
    int64_t nnz = 0, bytes = 0;
    std::vector<void*> bufs;
    // device arrays
    int *perm = nullptr, *leaf_of = nullptr, *parent = nullptr;
    int *lo_d = nullptr, *hi_d = nullptr, *son_d = nullptr;
    double *center = nullptr, *side = nullptr;
    double *coef = nullptr, *shift = nullptr, *shiftT = nullptr, *kmat = nullptr;
    int *far_ptr = nullptr, *far_tau = nullptr;
    int* leaves = nullptr;
    // the passes in four launches: the tree splits at level `split`; below it one block per
    // subtree walks all its levels, above it one block walks the top levels
    int split = 0, nsub = 0, sub_levels = 0, ntop_up = 0, ntop_down = 0;
    int *sub_off = nullptr, *sub_nodes = nullptr;           // per subtree and level: its nodes
    int *top_up_off = nullptr, *top_up = nullptr;           // internal nodes above the split, deepest level first
    int *top_down_off = nullptr, *top_down = nullptr;       // nodes of levels 1..split
    int nleaves = 0, nsig = 0;
    int* sig_nodes = nullptr;  // nodes with admissible partners, in node order
    int *nz_ptr = nullptr, *nz_row = nullptr, *nz_col = nullptr;
    double* nz_val = nullptr;
    bool near_ready = false;
    // the near field from local computations (fl_hmatrix_assemble_near), planned on first use
    bool hn_planned = false;
    fl::HNearDev hn;
    int64_t hn_entries = 0, hn_bytes = 0;  // tile partial entries; bytes of the plan and workspace
    // the strong form by the cluster method (fl_hmatrix_strong_form), planned per cell rule
    int hsf_kc = 0;
    fl::HsfDev hsf;
    double *xh = nullptr, *yh = nullptr;
    double* Pb = nullptr;  // per admissible pair: K_b xh[tau]
    // Jacobi-PCG with the product (fl_hmatrix_solve), allocated on first use
    double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_dinv = nullptr;
    bool dinv_ready = false;            // cg_dinv matches the near field and (dinv_alpha, dinv_beta)
    double dinv_alpha = 0.0, dinv_beta = 1.0;
    double *cg_part = nullptr, *cg_scal = nullptr, *cg_host = nullptr;
    // products captured as CUDA graphs, keyed by (x, y): the near-field product runs on a second
    // stream beside the chain of small far-field launches, and the graph launches them at once
    struct Graph {
        const double* x;
        double* y;
        cudaGraphExec_t exec;
        int launches;  // kernels the graph holds
    };
    std::vector<Graph> graphs;
    cudaStream_t cap = nullptr, side_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
};

namespace fl {
namespace {

int hm_fail(fl_hm* H, int code, const std::string& msg) {
    if (H) H->err = msg;
    return code;
}

int hm_enqueue(fl_hm* H, const double* x_dev, double* y_dev, cudaStream_t st, cudaStream_t side, bool far_only);

template <typename T>
int hm_upload(fl_hm* H, T** dst, const std::vector<T>& src, cudaStream_t st) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
    if (pool_dev_alloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return hm_fail(H, FL_ENOMEM, "cluster tables");
    }
    H->bufs.push_back(p);
    H->bytes += (int64_t)bytes;
    *dst = (T*)p;
    if (!src.empty() && cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return hm_fail(H, FL_ECUDA, "cluster table upload");
    return FL_OK;
}

int hm_alloc(fl_hm* H, double** dst, size_t count) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(double), 16);
    if (pool_dev_alloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return hm_fail(H, FL_ENOMEM, "cluster workspace");
    }
    H->bufs.push_back(p);
    H->bytes += (int64_t)bytes;
    *dst = (double*)p;
    return FL_OK;
}

// 1D Lagrange basis value l_k(t) of the m Chebyshev points of [c - L/2, c + L/2]
__device__ double cheb_node(double c, double L, int m, int k) {
    return c + 0.5 * L * cos((2.0 * (k + 1) - 1.0) * M_PI / (2.0 * m));
}
__device__ double lagrange1(double c, double L, int m, int k, double t) {
    const double xk = cheb_node(c, L, m, k);
    double v = 1.0;
    for (int l = 0; l < m; ++l)
        if (l != k) v *= (t - cheb_node(c, L, m, l)) / (xk - cheb_node(c, L, m, l));
    return v;
}
// tensor Lagrange polynomial alpha of cluster (c, L) at x
__device__ double lagrange_d(const double* c, double L, int m, int d, int alpha, const double* x) {
    if (d == 1) return lagrange1(c[0], L, m, alpha, x[0]);
    return lagrange1(c[0], L, m, alpha / m, x[0]) * lagrange1(c[1], L, m, alpha % m, x[1]);
}
__device__ void cheb_point_d(const double* c, double L, int m, int d, int alpha, double* x) {
    if (d == 1) {
        x[0] = cheb_node(c[0], L, m, alpha);
    } else {
        x[0] = cheb_node(c[0], L, m, alpha / m);
        x[1] = cheb_node(c[1], L, m, alpha % m);
    }
}

// the same 1D Lagrange value from the cluster's nodes computed once (x[l] = cheb_node(.., l)):
// the same operations in the same order as lagrange1
__device__ double lagrange1_nodes(const double* x, int m, int k, double t) {
    double v = 1.0;
    for (int l = 0; l < m; ++l)
        if (l != k) v *= (t - x[l]) / (x[k] - x[l]);
    return v;
}

// leaf coefficients int phi_i L_alpha^leaf, one thread per (tree position, alpha); the rule
// (lam [q][d], w [q], on the reference cell) integrates the degree 2m-1 integrand exactly
__global__ void leaf_coef_kernel(int64_t n, int d, int m, int md, const int* perm, const int* leaf_of,
                                 const double* center, const double* side, const int* vod, const int64_t* v2c_ptr,
                                 const int* v2c, const int* cells, const double* V, const double* jac, int q,
                                 const double* lam, const double* w, double* coef) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * md) return;
    const int64_t p = t / md;
    const int alpha = (int)(t - p * md);
    const int c = leaf_of[p];
    const int v = vod[perm[p]];
    const int nv = d + 1;
    // the leaf's Chebyshev nodes per axis (m <= 12), computed once per thread
    double xn[2][12];
    for (int k = 0; k < d; ++k)
        for (int l = 0; l < m; ++l) xn[k][l] = cheb_node(center[(int64_t)c * d + k], side[c], m, l);
    const int a0 = d == 1 ? alpha : alpha / m, a1 = d == 1 ? 0 : alpha % m;
    double acc = 0.0;
    for (int64_t e = v2c_ptr[v]; e < v2c_ptr[v + 1]; ++e) {
        const int K = v2c[e];
        const int* cell = cells + (int64_t)K * nv;
        int a = 0;
        while (cell[a] != v) ++a;
        for (int r = 0; r < q; ++r) {
            double x[2];
            double phi;
            if (d == 1) {
                const double tt = lam[r];
                x[0] = V[cell[0]] + tt * (V[cell[1]] - V[cell[0]]);
                phi = a == 0 ? 1.0 - tt : tt;
            } else {
                const double l1 = lam[2 * r], l2 = lam[2 * r + 1];
                for (int k = 0; k < 2; ++k)
                    x[k] = V[2 * cell[0] + k] + l1 * (V[2 * cell[1] + k] - V[2 * cell[0] + k]) +
                           l2 * (V[2 * cell[2] + k] - V[2 * cell[0] + k]);
                phi = a == 0 ? 1.0 - l1 - l2 : (a == 1 ? l1 : l2);
            }
            const double Lv = d == 1 ? lagrange1_nodes(xn[0], m, a0, x[0])
                                     : lagrange1_nodes(xn[0], m, a0, x[0]) * lagrange1_nodes(xn[1], m, a1, x[1]);
            acc += w[r] * jac[K] * phi * Lv;
        }
    }
    coef[p * md + alpha] = acc;
}

// shift coefficients S_son[beta][alpha] = L_alpha^father(xi_beta^son), one thread per entry, and
// their transpose ST_son[alpha][beta] (the downward pass reads them along beta)
__global__ void shift_kernel(int nodes, int d, int m, int md, const int* parent, const double* center,
                             const double* side, double* S, double* ST) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nodes * md * md) return;
    const int c = (int)(t / ((int64_t)md * md));
    const int r = (int)(t - (int64_t)c * md * md);
    const int beta = r / md, alpha = r - beta * md;
    const int f = parent[c];
    double v = 0.0;
    if (f >= 0) {
        double x[2];
        cheb_point_d(center + (int64_t)c * d, side[c], m, d, beta, x);
        v = lagrange_d(center + (int64_t)f * d, side[f], m, d, alpha, x);
    }
    S[t] = v;
    ST[(int64_t)c * md * md + (int64_t)alpha * md + beta] = v;
}

// kernel matrices of the admissible pairs, in sigma-major order: K[b][alpha][beta]
__global__ void kmat_kernel(int nfar, int d, int m, int md, const int* far_sig, const int* far_tau,
                            const double* center, const double* side, double expo, double* K) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nfar * md * md) return;
    const int b = (int)(t / ((int64_t)md * md));
    const int r = (int)(t - (int64_t)b * md * md);
    const int alpha = r / md, beta = r - alpha * md;
    const int a = far_sig[b], c = far_tau[b];
    double xa[2], xb[2];
    cheb_point_d(center + (int64_t)a * d, side[a], m, d, alpha, xa);
    cheb_point_d(center + (int64_t)c * d, side[c], m, d, beta, xb);
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) r2 += (xa[k] - xb[k]) * (xa[k] - xb[k]);
    K[t] = pow(r2, expo);
}

__global__ void near_gather_kernel(int64_t nnz, const int* row, const int* col, const double* A, int64_t lda,
                                   double* val) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) val[e] = A[(int64_t)row[e] * lda + col[e]];
}

// y = N x, one warp per row (columns ascending)
__global__ void near_spmv_kernel(int64_t n, const int* ptr, const int* col, const double* val, const double* x,
                                 double* y) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    // four entries per lane in flight, four accumulators
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    const int e1 = ptr[row + 1];
    int e = ptr[row] + lane;
    for (; e + 96 < e1; e += 128) {
        const double v0 = __ldcs(val + e), v1 = __ldcs(val + e + 32), v2 = __ldcs(val + e + 64), v3 = __ldcs(val + e + 96);
        const int c0 = __ldcs(col + e), c1 = __ldcs(col + e + 32), c2 = __ldcs(col + e + 64), c3 = __ldcs(col + e + 96);
        a0 = fma(v0, x[c0], a0);
        a1 = fma(v1, x[c1], a1);
        a2 = fma(v2, x[c2], a2);
        a3 = fma(v3, x[c3], a3);
    }
    for (; e < e1; e += 32) a0 = fma(val[e], x[col[e]], a0);
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) y[row] = acc;
}

// upward pass on the leaves: xh[c][alpha] = sum_{p in c} coef[p][alpha] x[perm[p]]
__global__ void up_leaf_kernel(int nleaves, int md, const int* leaves, const int* lo, const int* hi, const int* perm,
                               const double* coef, const double* x, double* xh) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nleaves * md) return;
    const int c = leaves[t / md];
    const int alpha = (int)(t % md);
    double acc = 0.0;
    for (int p = lo[c]; p < hi[c]; ++p) acc = fma(coef[(int64_t)p * md + alpha], x[perm[p]], acc);
    xh[(int64_t)c * md + alpha] = acc;
}

// Products with the md x md matrices of the passes: MD > 0 fixes md at compile time (the loops
// unroll, four accumulators keep loads in flight), MD = 0 takes md.  Threads of one node are
// consecutive in alpha (beta), and every matrix is laid out so that they read consecutive
// addresses.
template <int MD>
__device__ __forceinline__ double dot_strided(const double* __restrict__ Mx, int64_t stride, const double* __restrict__ v,
                                              int md) {
    const int n = MD ? MD : md;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = 0;
#pragma unroll
    for (; k + 4 <= n; k += 4) {
        a0 = fma(Mx[(int64_t)k * stride], v[k], a0);
        a1 = fma(Mx[(int64_t)(k + 1) * stride], v[k + 1], a1);
        a2 = fma(Mx[(int64_t)(k + 2) * stride], v[k + 2], a2);
        a3 = fma(Mx[(int64_t)(k + 3) * stride], v[k + 3], a3);
    }
    for (; k < n; ++k) a0 = fma(Mx[(int64_t)k * stride], v[k], a0);
    return (a0 + a1) + (a2 + a3);
}

// couplings, in two fully parallel steps: per admissible pair b = (sigma, tau) and alpha,
// Pb[b][alpha] = sum_beta K_b[alpha][beta] xh[tau][beta]; then per (sigma, alpha)
// yh[sigma][alpha] = sum over sigma's pairs, in pair order, of Pb[b][alpha]
template <int MD>
__global__ void pair_product_kernel(int nfar, int md_rt, const int* far_tau, const double* K, const double* xh,
                                    double* Pb) {
    const int md = MD ? MD : md_rt;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nfar * md) return;
    const int64_t b = t / md;
    const int alpha = (int)(t - b * md);
    Pb[t] = dot_strided<MD>(K + b * md * md + (int64_t)alpha * md, 1, xh + (int64_t)far_tau[b] * md, md);
}

__global__ void couple_sum_kernel(int nsig, int md, const int* sig_nodes, const int* far_ptr, const double* Pb,
                                  double* yh) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nsig * md) return;
    const int sgm = sig_nodes[t / md];
    const int alpha = (int)(t % md);
    double acc = 0.0;
    for (int b = far_ptr[sgm]; b < far_ptr[sgm + 1]; ++b) acc += Pb[(int64_t)b * md + alpha];
    yh[(int64_t)sgm * md + alpha] = acc;
}

// the upward pass of a list of levels (in order) in one block: xh[f] for the internal nodes
template <int MD>
__device__ __forceinline__ void up_levels(int nlev, const int* off, const int* nodes, int md, const int* son,
                                          const double* S, double* xh) {
    for (int j = 0; j < nlev; ++j) {
        const int lo = off[j], cnt = off[j + 1] - lo;
        for (int t = threadIdx.x; t < cnt * md; t += blockDim.x) {
            const int f = nodes[lo + t / md];
            if (son[2 * f] < 0) continue;
            const int alpha = t % md;
            double acc = 0.0;
            for (int q = 0; q < 2; ++q) {
                const int c = son[2 * f + q];
                acc += dot_strided<MD>(S + (int64_t)c * md * md + alpha, md, xh + (int64_t)c * md, md);
            }
            xh[(int64_t)f * md + alpha] = acc;
        }
        __syncthreads();
    }
}

// the downward pass of a list of levels (in order) in one block: yh[c] += ST_c yh[parent]
template <int MD>
__device__ __forceinline__ void down_levels(int nlev, const int* off, const int* nodes, int md, const int* parent,
                                            const double* ST, double* yh) {
    for (int j = 0; j < nlev; ++j) {
        const int lo = off[j], cnt = off[j + 1] - lo;
        for (int t = threadIdx.x; t < cnt * md; t += blockDim.x) {
            const int c = nodes[lo + t / md];
            const int beta = t % md;
            yh[(int64_t)c * md + beta] +=
                dot_strided<MD>(ST + (int64_t)c * md * md + beta, md, yh + (int64_t)parent[c] * md, md);
        }
        __syncthreads();
    }
}

// subtree k (one block): its levels from the deepest up to its root
template <int MD>
__global__ void up_sub_kernel(int nlev, int md_rt, const int* sub_off, const int* sub_nodes, const int* son,
                              const double* S, double* xh) {
    const int md = MD ? MD : md_rt;
    const int* off = sub_off + (int64_t)blockIdx.x * (nlev + 1);
    // levels stored root first: walk them backwards through a reversed offset view
    for (int j = nlev - 1; j >= 0; --j) up_levels<MD>(1, off + j, sub_nodes, md, son, S, xh);
}

template <int MD>
__global__ void up_top_kernel(int nlev, int md_rt, const int* off, const int* nodes, const int* son, const double* S,
                              double* xh) {
    up_levels<MD>(nlev, off, nodes, MD ? MD : md_rt, son, S, xh);
}

template <int MD>
__global__ void down_top_kernel(int nlev, int md_rt, const int* off, const int* nodes, const int* parent,
                                const double* ST, double* yh) {
    down_levels<MD>(nlev, off, nodes, MD ? MD : md_rt, parent, ST, yh);
}

// subtree k (one block): its levels below its root, top down
template <int MD>
__global__ void down_sub_kernel(int nlev, int md_rt, const int* sub_off, const int* sub_nodes, const int* parent,
                                const double* ST, double* yh) {
    const int* off = sub_off + (int64_t)blockIdx.x * (nlev + 1);
    down_levels<MD>(nlev - 1, off + 1, sub_nodes, MD ? MD : md_rt, parent, ST, yh);
}

// leaves to DOFs: y[perm[p]] += mC sum_alpha coef[p][alpha] yh[leaf][alpha]
__global__ void down_leaf_kernel(int64_t n, int md, const int* perm, const int* leaf_of, const double* coef,
                                 const double* yh, double mC, double* y) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double* cp = coef + p * md;
    const double* yl = yh + (int64_t)leaf_of[p] * md;
    double acc = 0.0;
    for (int alpha = 0; alpha < md; ++alpha) acc = fma(cp[alpha], yl[alpha], acc);
    y[perm[p]] += mC * acc;
}

// ------------------------------------------------------------ Jacobi-PCG --
constexpr int HCG_BLOCKS = 256, HCG_THREADS = 256;

// dinv[i] = 1 / (alpha M_ii + beta A_ii), A_ii from the near field (the diagonal lies in every leaf's
// own block), M_ii = sum over the cells K around DOF i's vertex of 2 |K| / ((d+1)(d+2)) (P1 mass)
__global__ void hcg_diag_kernel(int64_t n, const int* ptr, const int* col, const double* val, double alpha,
                                double beta, int dim, const int* vod, const int64_t* v2c_ptr, const int* v2c,
                                const double* jac_orig, double* dinv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e)
        if (col[e] == i) d = val[e];
    d *= beta;
    if (alpha != 0.0) {
        const double scale = dim == 2 ? 0.5 : 1.0;  // |K| = jac / 2 (2D), jac (1D)
        const double den = 2.0 / ((dim + 1.0) * (dim + 2.0));
        double m = 0.0;
        const int v = vod[i];
        for (int64_t q = v2c_ptr[v]; q < v2c_ptr[v + 1]; ++q) m += scale * jac_orig[v2c[q]] * den;
        d += alpha * m;
    }
    dinv[i] = d > 0.0 ? 1.0 / d : 0.0;
}

// per block: the partial sums of a.b and c.d (fixed grid, fixed order)
__global__ void hcg_dots_kernel(int64_t n, const double* a, const double* b, const double* c, const double* d,
                                double* part) {
    __shared__ double sh[2][HCG_THREADS / 32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        s0 = fma(a[i], b[i], s0);
        if (c) s1 = fma(c[i], d[i], s1);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < HCG_THREADS / 32; ++w) {
            t0 += sh[0][w];
            t1 += sh[1][w];
        }
        part[2 * blockIdx.x] = t0;
        part[2 * blockIdx.x + 1] = t1;
    }
}

// out[k] = sum over blocks of part[2 b + k], k = 0, 1 (one thread each, block order)
__global__ void hcg_sum_kernel(const double* part, double* out) {
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int b = 0; b < HCG_BLOCKS; ++b) t += part[2 * b + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// u += alpha p, r -= alpha q, z = D^-1 r (alpha = scal[0] / scal[2])
__global__ void hcg_update_kernel(int64_t n, const double* scal, const double* p, const double* q,
                                  const double* dinv, double* u, double* r, double* z) {
    const double alpha = scal[0] / scal[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = fma(alpha, p[i], u[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        z[i] = dinv[i] * ri;
    }
}

// p = z + beta p (beta = scal[1] / scal[0], the new and old r.z); the new r.z becomes the old
__global__ void hcg_direction_kernel(int64_t n, double* scal, const double* z, double* p) {
    const double beta = scal[1] / scal[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

__global__ void hcg_start_kernel(int64_t n, const double* b, const double* dinv, double* u, double* r, double* z,
                                 double* p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = 0.0;
        r[i] = b[i];
        z[i] = dinv[i] * b[i];
        p[i] = z[i];
    }
}

unsigned blocks_for(int64_t work, int threads) { return (unsigned)std::max<int64_t>(1, (work + threads - 1) / threads); }

}  // namespace
}  // namespace fl

using namespace fl;

static double frac_constant_h(int d, double s) {
    return std::pow(2.0, 2 * s) * s * std::tgamma(s + d / 2.0) / (std::pow(M_PI, d / 2.0) * std::tgamma(1.0 - s));
}

extern "C" {

int fl_cluster_plan(fl_handle h, double s, double eta, int leaf, int64_t* sizes, int32_t* perm, int32_t* node,
                    int32_t* far, int32_t* near) {
    if (!h || !sizes) return FL_EINVAL;
    h->err.clear();
    if (h->sym_K) return sym_unsupported(h, "fl_cluster_plan");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    ClusterPlan C;
    if (build_cluster_plan(h->plan[pi], eta, leaf, C) != FL_OK) return set_err(h, FL_EINVAL, "leaf < 1 or eta < 0");
    sizes[0] = C.nodes;
    sizes[1] = (int64_t)C.far.size() / 2;
    sizes[2] = (int64_t)C.near.size() / 2;
    if (perm) std::copy(C.perm.begin(), C.perm.end(), perm);
    if (node)
        for (int c = 0; c < C.nodes; ++c) {
            node[4 * c] = C.lo[c];
            node[4 * c + 1] = C.hi[c];
            node[4 * c + 2] = C.son[2 * c];
            node[4 * c + 3] = C.son[2 * c + 1];
        }
    if (far) std::copy(C.far.begin(), C.far.end(), far);
    if (near) std::copy(C.near.begin(), C.near.end(), near);
    return FL_OK;
}

int fl_near_region_plan(fl_handle h, double s, double eta, int leaf, int64_t* sizes, int32_t* cell_perm,
                        int32_t* ef_ptr, int32_t* ef_fac, int32_t* ef_cls, int32_t* fac_vert, double* fac_normal) {
    if (!h || !sizes) return FL_EINVAL;
    h->err.clear();
    if (h->sym_K) return sym_unsupported(h, "fl_near_region_plan");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    try {
        ClusterPlan C;
        if (build_cluster_plan(P, eta, leaf, C) != FL_OK) return set_err(h, FL_EINVAL, "leaf < 1 or eta < 0");
        HNearPlan Q;
        std::string err;
        const int rc = plan_hnear(P, C, Q, err);
        if (rc != FL_OK) return set_err(h, rc, err);
        sizes[0] = (int64_t)Q.tiles.size() / 2;
        sizes[1] = (int64_t)Q.ef_fac.size();
        sizes[2] = (int64_t)Q.FLEN.size();
        sizes[3] = P.nc;
        if (cell_perm) std::copy(P.perm.begin(), P.perm.end(), cell_perm);
        if (ef_ptr) std::copy(Q.ef_ptr.begin(), Q.ef_ptr.end(), ef_ptr);
        if (ef_fac) std::copy(Q.ef_fac.begin(), Q.ef_fac.end(), ef_fac);
        if (ef_cls) std::copy(Q.ef_cls.begin(), Q.ef_cls.end(), ef_cls);
        if (fac_vert) std::copy(Q.F.begin(), Q.F.end(), fac_vert);
        if (fac_normal) std::copy(Q.FN.begin(), Q.FN.end(), fac_normal);
    } catch (const std::bad_alloc&) {
        return set_err(h, FL_ENOMEM, "out of host memory");
    }
    return FL_OK;
}

int fl_near_region_tiles(fl_handle h, double s, double eta, int leaf, int64_t* ntiles, int32_t* tiles,
                         uint32_t* rowmask) {
    if (!h || !ntiles) return FL_EINVAL;
    h->err.clear();
    if (h->sym_K) return sym_unsupported(h, "fl_near_region_tiles");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    try {
        ClusterPlan C;
        if (build_cluster_plan(P, eta, leaf, C) != FL_OK) return set_err(h, FL_EINVAL, "leaf < 1 or eta < 0");
        HNearPlan Q;
        std::string err;
        const int rc = plan_hnear(P, C, Q, err);
        if (rc != FL_OK) return set_err(h, rc, err);
        *ntiles = (int64_t)Q.tiles.size() / 2;
        if (tiles) std::copy(Q.tiles.begin(), Q.tiles.end(), tiles);
        if (rowmask) std::copy(Q.rowmask.begin(), Q.rowmask.end(), rowmask);
    } catch (const std::bad_alloc&) {
        return set_err(h, FL_ENOMEM, "out of host memory");
    }
    return FL_OK;
}

int fl_strong_form_cluster_plan(fl_handle h, double s, double eta, int leaf, int k_cell, int64_t* sizes,
                                int32_t* pgroup, int32_t* gnode, int64_t* gf_ptr, int32_t* gf_fac,
                                int32_t* fac_vert) {
    if (!h || !sizes) return FL_EINVAL;
    h->err.clear();
    if (h->sym_K) return sym_unsupported(h, "fl_strong_form_cluster_plan");
    if (k_cell < 1 || k_cell > 16) return set_err(h, FL_EINVAL, "k_cell in [1, 16]");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (P.dim != 2) return set_err(h, FL_ENOTIMPL, "the cluster strong form is 2D");
    try {
        ClusterPlan C;
        if (build_cluster_plan(P, eta, leaf, C) != FL_OK) return set_err(h, FL_EINVAL, "leaf < 1 or eta < 0");
        std::vector<int> c2f, fv;
        int64_t nfac = 0;
        if (sf_facets_host(P, c2f, fv, &nfac) != FL_OK) return set_err(h, FL_EINVAL, "non-conforming mesh");
        HsfPlan Q;
        std::string err;
        const int rc = plan_hsf(P, C, c2f, nfac, k_cell, Q, err);
        if (rc != FL_OK) return set_err(h, rc, err);
        sizes[0] = Q.npts;
        sizes[1] = Q.groups;
        sizes[2] = (int64_t)Q.gf_fac.size();
        sizes[3] = nfac;
        if (pgroup) std::copy(Q.pgroup.begin(), Q.pgroup.end(), pgroup);
        if (gnode) std::copy(Q.gnode.begin(), Q.gnode.end(), gnode);
        if (gf_ptr) std::copy(Q.gf_ptr.begin(), Q.gf_ptr.end(), gf_ptr);
        if (gf_fac) std::copy(Q.gf_fac.begin(), Q.gf_fac.end(), gf_fac);
        if (fac_vert) std::copy(fv.begin(), fv.end(), fac_vert);
    } catch (const std::bad_alloc&) {
        return set_err(h, FL_ENOMEM, "out of host memory");
    }
    return FL_OK;
}

void fl_hmatrix_destroy(fl_hmatrix H) {
    if (!H) return;
    if (!H->bufs.empty() || !H->graphs.empty()) {
        cudaSetDevice(H->device);
        cudaDeviceSynchronize();
        for (void* p : H->bufs) pool_dev_free(p);
    }
    for (auto& g : H->graphs) cudaGraphExecDestroy(g.exec);
    if (H->cg_host) pool_host_free(H->cg_host);
    if (H->cap) cudaStreamDestroy(H->cap);
    if (H->side_st) cudaStreamDestroy(H->side_st);
    if (H->ev_fork) cudaEventDestroy(H->ev_fork);
    if (H->ev_join) cudaEventDestroy(H->ev_join);
    delete H;
}

int fl_hmatrix_create(fl_handle h, double s, int m, double eta, int leaf, fl_hmatrix* out, void* stream) {
    if (!h || !out) return FL_EINVAL;
    h->err.clear();
    *out = nullptr;
    if (h->sym_K) return sym_unsupported(h, "fl_hmatrix_create");
    if (m < 1 || m > 12) return set_err(h, FL_EINVAL, "Chebyshev order m must lie in [1, 12]");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    fl_hm* H = new (std::nothrow) fl_hm;
    if (!H) return set_err(h, FL_ENOMEM, "out of host memory");
    H->mesh = h;
    H->device = h->device;
    H->pi = pi;
    H->d = P.dim;
    H->m = m;
    H->md = P.dim == 1 ? m : m * m;
    H->s = s;
    H->C = frac_constant_h(P.dim, s);
    cudaStream_t st = (cudaStream_t)stream;
    auto fail = [&](int code, const std::string& msg) {
        set_err(h, code, msg + (H->err.empty() ? "" : ": " + H->err));
        fl_hmatrix_destroy(H);
        return code;
    };
    try {
        if (build_cluster_plan(P, eta, leaf, H->plan) != FL_OK) return fail(FL_EINVAL, "leaf < 1 or eta < 0");
        if (cudaSetDevice(h->device) != cudaSuccess) return fail(FL_ECUDA, "cudaSetDevice");
        // the mesh tables (vertices, cells, vertex -> cells) come from the handle
        if (ensure_device_tables(h, pi, st) != FL_OK) return fail(FL_ECUDA, "mesh tables");
        const ClusterPlan& C = H->plan;
        const int nn = C.nodes, md = H->md, d = H->d;
        const int64_t n = C.n;
        std::vector<int> parent(nn, -1), leaf_of(n, -1), leaves;
        for (int c = 0; c < nn; ++c) {
            for (int q = 0; q < 2; ++q)
                if (C.son[2 * c + q] >= 0) parent[C.son[2 * c + q]] = c;
            if (C.son[2 * c] < 0) {
                leaves.push_back(c);
                for (int p = C.lo[c]; p < C.hi[c]; ++p) leaf_of[p] = c;
            }
        }
        // level lists: fathers for the upward pass (deepest first), non-root nodes for the
        // downward pass (shallowest first)
        // split level: the first holding at least 64 nodes (the deepest if none does)
        std::vector<int> per_level(C.depth + 1, 0);
        for (int c = 0; c < nn; ++c) ++per_level[C.level[c]];
        int Ls = C.depth;
        for (int L = 0; L <= C.depth; ++L)
            if (per_level[L] >= 64) {
                Ls = L;
                break;
            }
        H->split = Ls;
        std::vector<int> top_up, top_up_off(1, 0), top_down, top_down_off(1, 0);
        for (int L = Ls - 1; L >= 0; --L) {
            for (int c = 0; c < nn; ++c)
                if (C.level[c] == L && C.son[2 * c] >= 0) top_up.push_back(c);
            top_up_off.push_back((int)top_up.size());
        }
        for (int L = 1; L <= Ls; ++L) {
            for (int c = 0; c < nn; ++c)
                if (C.level[c] == L) top_down.push_back(c);
            top_down_off.push_back((int)top_down.size());
        }
        H->ntop_up = Ls;
        H->ntop_down = Ls;
        // subtrees rooted at the split level, their nodes level by level (root first)
        const int NL = C.depth - Ls + 1;
        std::vector<int> sub_nodes, sub_off;
        for (int r = 0; r < nn; ++r) {
            if (C.level[r] != Ls) continue;
            std::vector<int> cur(1, r), nxt;
            for (int j = 0; j < NL; ++j) {
                sub_off.push_back((int)sub_nodes.size());
                sub_nodes.insert(sub_nodes.end(), cur.begin(), cur.end());
                nxt.clear();
                for (int c : cur)
                    if (C.son[2 * c] >= 0) {
                        nxt.push_back(C.son[2 * c]);
                        nxt.push_back(C.son[2 * c + 1]);
                    }
                cur.swap(nxt);
            }
            sub_off.push_back((int)sub_nodes.size());
            ++H->nsub;
        }
        H->sub_levels = NL;
        // admissible pairs grouped by sigma (in node order; within sigma in partition order)
        const int nfar = (int)C.far.size() / 2;
        std::vector<int> far_ptr(nn + 1, 0), far_sig(nfar), far_tau(nfar), sig_nodes;
        for (int b = 0; b < nfar; ++b) ++far_ptr[C.far[2 * b] + 1];
        for (int c = 0; c < nn; ++c) far_ptr[c + 1] += far_ptr[c];
        {
            std::vector<int> fill(far_ptr.begin(), far_ptr.end() - 1);
            for (int b = 0; b < nfar; ++b) {
                const int k = fill[C.far[2 * b]]++;
                far_sig[k] = C.far[2 * b];
                far_tau[k] = C.far[2 * b + 1];
            }
        }
        for (int c = 0; c < nn; ++c)
            if (far_ptr[c + 1] > far_ptr[c]) sig_nodes.push_back(c);
        // near field CSR over the original DOF numbering, columns ascending.  Every row of a leaf
        // has the same columns (the DOFs of the leaf's near partners), so each leaf's column list
        // is sorted once and copied into its rows.
        std::vector<std::vector<int>> lcols(nn);
        for (size_t b = 0; b + 1 < C.near.size(); b += 2) {
            const int a = C.near[b], c = C.near[b + 1];
            for (int q = C.lo[c]; q < C.hi[c]; ++q) lcols[a].push_back(C.perm[q]);
        }
        for (int c : leaves) std::sort(lcols[c].begin(), lcols[c].end());
        std::vector<int> rowleaf(n, -1);
        for (int c : leaves)
            for (int p = C.lo[c]; p < C.hi[c]; ++p) rowleaf[C.perm[p]] = c;
        std::vector<int> nz_ptr(n + 1, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t next = (int64_t)nz_ptr[i] + (int64_t)lcols[rowleaf[i]].size();
            if (next > INT32_MAX) return fail(FL_ENOMEM, "near field larger than 2^31 entries");
            nz_ptr[i + 1] = (int)next;
        }
        std::vector<int> nz_row(nz_ptr[n]), nz_col(nz_ptr[n]);
        for (int64_t i = 0; i < n; ++i) {
            const std::vector<int>& L = lcols[rowleaf[i]];
            std::copy(L.begin(), L.end(), nz_col.begin() + nz_ptr[i]);
            std::fill(nz_row.begin() + nz_ptr[i], nz_row.begin() + nz_ptr[i + 1], (int)i);
        }
        H->nnz = nz_ptr[n];
        H->nleaves = (int)leaves.size();
        H->nsig = (int)sig_nodes.size();
        // quadrature of the leaf coefficients: Gauss order m + 1 (collapsed on triangles)
        const Rule R = make_rule(d, m + 1);
        std::vector<int> lo(C.lo), hi(C.hi), son(C.son);
        int *d_lo = nullptr, *d_hi = nullptr, *d_son = nullptr, *d_far_sig = nullptr;
        double *d_lam = nullptr, *d_w = nullptr;
        int rc = FL_OK;
        if ((rc = hm_upload(H, &H->perm, C.perm, st)) || (rc = hm_upload(H, &H->leaf_of, leaf_of, st)) ||
            (rc = hm_upload(H, &H->parent, parent, st)) || (rc = hm_upload(H, &H->center, C.center, st)) ||
            (rc = hm_upload(H, &H->side, C.side, st)) || (rc = hm_upload(H, &d_lo, lo, st)) ||
            (rc = hm_upload(H, &d_hi, hi, st)) || (rc = hm_upload(H, &d_son, son, st)) ||
            (rc = hm_upload(H, &H->far_ptr, far_ptr, st)) || (rc = hm_upload(H, &H->far_tau, far_tau, st)) ||
            (rc = hm_upload(H, &d_far_sig, far_sig, st)) || (rc = hm_upload(H, &H->sig_nodes, sig_nodes, st)) ||
            (rc = hm_upload(H, &H->sub_off, sub_off, st)) || (rc = hm_upload(H, &H->sub_nodes, sub_nodes, st)) ||
            (rc = hm_upload(H, &H->top_up_off, top_up_off, st)) || (rc = hm_upload(H, &H->top_up, top_up, st)) ||
            (rc = hm_upload(H, &H->top_down_off, top_down_off, st)) ||
            (rc = hm_upload(H, &H->top_down, top_down, st)) ||
            (rc = hm_upload(H, &H->leaves, leaves, st)) || (rc = hm_upload(H, &H->nz_ptr, nz_ptr, st)) ||
            (rc = hm_upload(H, &H->nz_row, nz_row, st)) || (rc = hm_upload(H, &H->nz_col, nz_col, st)) ||
            (rc = hm_upload(H, &d_lam, R.lam, st)) || (rc = hm_upload(H, &d_w, R.w, st)))
            return fail(rc, "cluster tables");
        H->lo_d = d_lo;
        H->hi_d = d_hi;
        H->son_d = d_son;
        if ((rc = hm_alloc(H, &H->coef, (size_t)n * md)) || (rc = hm_alloc(H, &H->shift, (size_t)nn * md * md)) ||
            (rc = hm_alloc(H, &H->shiftT, (size_t)nn * md * md)) ||
            (rc = hm_alloc(H, &H->kmat, (size_t)nfar * md * md)) || (rc = hm_alloc(H, &H->xh, (size_t)nn * md)) ||
            (rc = hm_alloc(H, &H->yh, (size_t)nn * md)) ||
            (rc = hm_alloc(H, &H->Pb, (size_t)std::max(nfar, 1) * md)) || (rc = hm_alloc(H, &H->nz_val, (size_t)H->nnz)))
            return fail(rc, "cluster workspace");
        const DevTables& t = h->dev[pi];
        leaf_coef_kernel<<<blocks_for(n * md, 128), 128, 0, st>>>(n, d, H->m, md, H->perm, H->leaf_of, H->center,
                                                                  H->side, t.vod, t.v2c_ptr, t.v2c, t.cells, t.V,
                                                                  t.jac_orig, R.q, d_lam, d_w, H->coef);
        shift_kernel<<<blocks_for((int64_t)nn * md * md, 128), 128, 0, st>>>(nn, d, H->m, md, H->parent, H->center,
                                                                            H->side, H->shift, H->shiftT);
        if (nfar > 0)
            kmat_kernel<<<blocks_for((int64_t)nfar * md * md, 128), 128, 0, st>>>(
                nfar, d, H->m, md, d_far_sig, H->far_tau, H->center, H->side, -(d + 2.0 * s) / 2.0, H->kmat);
        count_launch(nfar > 0 ? 3 : 2);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(FL_ECUDA, std::string("cluster set-up: ") + cudaGetErrorString(e));
    } catch (const std::bad_alloc&) {
        return fail(FL_ENOMEM, "out of host memory");
    }
    *out = H;
    return FL_OK;
}

int fl_hmatrix_set_near(fl_hmatrix H, const double* A_dev, int64_t lda, void* stream) {
    if (!H) return FL_EINVAL;
    H->err.clear();
    if (!A_dev || lda < H->plan.n) return hm_fail(H, FL_EINVAL, "bad A / lda");
    if (cudaSetDevice(H->device) != cudaSuccess) return hm_fail(H, FL_ECUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    if (H->nnz > 0) {
        near_gather_kernel<<<blocks_for(H->nnz, 256), 256, 0, st>>>(H->nnz, H->nz_row, H->nz_col, A_dev, lda, H->nz_val);
        count_launch(1);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hm_fail(H, FL_ECUDA, std::string("near gather: ") + cudaGetErrorString(e));
    H->near_ready = true;
    H->dinv_ready = false;
    return FL_OK;
}

int fl_hmatrix_assemble_near(fl_hmatrix H, int precision, void* stream) {
    if (!H) return FL_EINVAL;
    H->err.clear();
    if (cudaSetDevice(H->device) != cudaSuccess) return hm_fail(H, FL_ECUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    fl_ctx* h = H->mesh;
    int rc = FL_OK;
    if (!H->hn_planned) {
        const int64_t b0 = H->bytes;
        try {
            fl::HNearPlan Q;
            std::string err;
            rc = fl::plan_hnear(h->plan[H->pi], H->plan, Q, err);
            if (rc != FL_OK) return hm_fail(H, rc, err);
            fl::HNearDev& q = H->hn;
            if ((rc = hm_upload(H, &q.tiles, Q.tiles, st)) || (rc = hm_upload(H, &q.toff, Q.toff, st)) ||
                (rc = hm_upload(H, &q.trow_ptr, Q.trow_ptr, st)) || (rc = hm_upload(H, &q.rowmask, Q.rowmask, st)) ||
                (rc = hm_upload(H, &q.F, Q.F, st)) ||
                (rc = hm_upload(H, &q.FN, Q.FN, st)) || (rc = hm_upload(H, &q.FLEN, Q.FLEN, st)) ||
                (rc = hm_upload(H, &q.ef_ptr, Q.ef_ptr, st)) || (rc = hm_upload(H, &q.ef_fac, Q.ef_fac, st)) ||
                (rc = hm_upload(H, &q.ef_cls, Q.ef_cls, st)))
                return rc;
            if ((rc = hm_alloc(H, &q.P, (size_t)Q.toff.back()))) return rc;
            q.ntiles = (int64_t)Q.tiles.size() / 2;
            H->hn_entries = Q.toff.back();
        } catch (const std::bad_alloc&) {
            return hm_fail(H, FL_ENOMEM, "out of host memory");
        }
        H->hn_bytes = H->bytes - b0;
        H->hn_planned = true;
    }
    rc = fl::assemble_hnear(h, H->pi, H->s, precision, H->hn, H->nnz, H->nz_row, H->nz_col, H->nz_val, st);
    if (rc != FL_OK) return hm_fail(H, rc, h->err);
    H->near_ready = true;
    H->dinv_ready = false;
    return FL_OK;
}

int fl_hmatrix_get_near(fl_hmatrix H, int64_t* nnz, int32_t* rowptr_dev, int32_t* col_dev, double* val_dev,
                        void* stream) {
    if (!H || !nnz) return FL_EINVAL;
    H->err.clear();
    *nnz = H->nnz;
    if (!rowptr_dev && !col_dev && !val_dev) return FL_OK;
    if (val_dev && !H->near_ready) return hm_fail(H, FL_EINVAL, "near field not set");
    if (cudaSetDevice(H->device) != cudaSuccess) return hm_fail(H, FL_ECUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (rowptr_dev)
        e = cudaMemcpyAsync(rowptr_dev, H->nz_ptr, (H->plan.n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && col_dev && H->nnz > 0)
        e = cudaMemcpyAsync(col_dev, H->nz_col, H->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && val_dev && H->nnz > 0)
        e = cudaMemcpyAsync(val_dev, H->nz_val, H->nnz * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return hm_fail(H, FL_ECUDA, std::string("near-field copy: ") + cudaGetErrorString(e));
    return FL_OK;
}

int fl_hmatrix_strong_form(fl_hmatrix H, const double* u_dev, int k_cell, int k_edge, int k_near, double* S_dev,
                           void* stream) {
    if (!H) return FL_EINVAL;
    H->err.clear();
    if (!u_dev || !S_dev) return hm_fail(H, FL_EINVAL, "NULL u or S");
    if (k_cell < 1 || k_cell > 16) return hm_fail(H, FL_EINVAL, "k_cell in [1, 16]");
    if (cudaSetDevice(H->device) != cudaSuccess) return hm_fail(H, FL_ECUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    fl_ctx* h = H->mesh;
    int rc = FL_OK;
    if (H->hsf_kc != k_cell) {
        const std::vector<int>* c2f = nullptr;
        int64_t nfac = 0;
        if ((rc = fl::sf_topology(h, H->pi, st, &c2f, &nfac)) != FL_OK) return hm_fail(H, rc, h->err);
        try {
            fl::HsfPlan Q;
            std::string err;
            rc = fl::plan_hsf(h->plan[H->pi], H->plan, *c2f, nfac, k_cell, Q, err);
            if (rc != FL_OK) return hm_fail(H, rc, err);
            fl::HsfDev& g = H->hsf;
            if ((rc = hm_upload(H, &g.gnode, Q.gnode, st)) || (rc = hm_upload(H, &g.gp_ptr, Q.gp_ptr, st)) ||
                (rc = hm_upload(H, &g.gp_idx, Q.gp_idx, st)) || (rc = hm_upload(H, &g.pgroup, Q.pgroup, st)) ||
                (rc = hm_upload(H, &g.plocal, Q.plocal, st)) || (rc = hm_upload(H, &g.gf_ptr, Q.gf_ptr, st)) ||
                (rc = hm_upload(H, &g.gf_fac, Q.gf_fac, st)) || (rc = hm_upload(H, &g.gbits, Q.gbits, st)) ||
                (rc = hm_upload(H, &g.dof_leaf, Q.dof_leaf, st)) || (rc = hm_upload(H, &g.gch, Q.gch, st)) ||
                (rc = hm_upload(H, &g.gpo, Q.gpo, st)) || (rc = hm_upload(H, &g.blk_g, Q.blk_g, st)) ||
                (rc = hm_upload(H, &g.blk_p0, Q.blk_p0, st)) || (rc = hm_upload(H, &g.blk_ch, Q.blk_ch, st)) ||
                (rc = hm_alloc(H, &g.cj, Q.gf_fac.size())) || (rc = hm_alloc(H, &g.part, (size_t)Q.nparts)))
                return rc;
            g.groups = Q.groups;
            g.words = Q.words;
            g.nparts = Q.nparts;
            g.nblocks = (int64_t)Q.blk_g.size();
            g.maxf = Q.maxf;
        } catch (const std::bad_alloc&) {
            return hm_fail(H, FL_ENOMEM, "out of host memory");
        }
        H->hsf_kc = k_cell;
    }
    // the far field of u at every node, then the strong form
    const int launches = fl::hm_enqueue(H, u_dev, nullptr, st, nullptr, true);
    if (launches < 0) return hm_fail(H, FL_ECUDA, "far-field passes");
    fl::count_launch(launches);
    fl::HsfDev g = H->hsf;
    g.m = H->m;
    g.md = H->md;
    g.yh = H->yh;
    g.center = H->center;
    g.side = H->side;
    rc = fl::strong_form_cluster(h, H->s, u_dev, k_cell, k_edge, k_near, g, S_dev, st);
    if (rc != FL_OK) return hm_fail(H, rc, h->err);
    return FL_OK;
}

int fl_hmatrix_br_indicators(fl_hmatrix H, const double* u_dev, const double* f_dev, int k_cell, int k_edge,
                             int k_near, double* eta_dev, double* S_dev, void* stream) {
    if (!H) return FL_EINVAL;
    H->err.clear();
    if (!eta_dev || !S_dev) return hm_fail(H, FL_EINVAL, "NULL eta or S");
    int rc = fl_hmatrix_strong_form(H, u_dev, k_cell, k_edge, k_near, S_dev, stream);
    if (rc != FL_OK) return rc;
    rc = fl::br_from_strong_form(H->mesh, H->s, f_dev, k_cell, S_dev, eta_dev, (cudaStream_t)stream);
    if (rc != FL_OK) return hm_fail(H, rc, H->mesh->err);
    return FL_OK;
}

int fl_hmatrix_near_info(fl_hmatrix H, int64_t* info) {
    if (!H || !info) return FL_EINVAL;
    info[0] = H->hn.ntiles;
    info[1] = H->hn_entries;
    info[2] = H->hn_bytes;
    return FL_OK;
}

}  // extern "C"

namespace fl {
namespace {
// The launches of one product: the near-field CSR product on `side` (forked from and joined
// back to `st`; on `st` itself when side is null), the upward pass, couplings and downward
// pass on `st`, then the leaf expansion, which adds the far field into y after the join.
// Returns the launch count, or -1.
// far_only: the upward pass, couplings and downward pass alone (H->yh then holds, per node, the far
// field of x expanded in the node's Chebyshev basis); y_dev and side are not used.
int hm_enqueue(fl_hm* H, const double* x_dev, double* y_dev, cudaStream_t st, cudaStream_t side,
               bool far_only) {
    const ClusterPlan& C = H->plan;
    const int64_t n = C.n;
    const int md = H->md, nn = C.nodes;
    int launches = 0;
    if (far_only) side = nullptr;
    if (side) {
        if (cudaEventRecord(H->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(side, H->ev_fork, 0) != cudaSuccess)
            return -1;
    }
    cudaStream_t ns = side ? side : st;
    if (!far_only) {
        near_spmv_kernel<<<blocks_for(n * 32, 256), 256, 0, ns>>>(n, H->nz_ptr, H->nz_col, H->nz_val, x_dev, y_dev);
        ++launches;
    }
    if (side && cudaEventRecord(H->ev_join, side) != cudaSuccess) return -1;
    up_leaf_kernel<<<blocks_for((int64_t)H->nleaves * md, 128), 128, 0, st>>>(H->nleaves, md, H->leaves, H->lo_d,
                                                                             H->hi_d, H->perm, H->coef, x_dev, H->xh);
    launches += 1;
    // upward pass: the subtrees below the split level, one block each, then the top in one block
    if (H->nsub > 0) {
        if (md == 16) up_sub_kernel<16><<<H->nsub, 256, 0, st>>>(H->sub_levels, md, H->sub_off, H->sub_nodes, H->son_d, H->shift, H->xh);
        else if (md == 36) up_sub_kernel<36><<<H->nsub, 256, 0, st>>>(H->sub_levels, md, H->sub_off, H->sub_nodes, H->son_d, H->shift, H->xh);
        else up_sub_kernel<0><<<H->nsub, 256, 0, st>>>(H->sub_levels, md, H->sub_off, H->sub_nodes, H->son_d, H->shift, H->xh);
        ++launches;
    }
    if (H->ntop_up > 0) {
        if (md == 16) up_top_kernel<16><<<1, 1024, 0, st>>>(H->ntop_up, md, H->top_up_off, H->top_up, H->son_d, H->shift, H->xh);
        else if (md == 36) up_top_kernel<36><<<1, 1024, 0, st>>>(H->ntop_up, md, H->top_up_off, H->top_up, H->son_d, H->shift, H->xh);
        else up_top_kernel<0><<<1, 1024, 0, st>>>(H->ntop_up, md, H->top_up_off, H->top_up, H->son_d, H->shift, H->xh);
        ++launches;
    }
    if (cudaMemsetAsync(H->yh, 0, (size_t)nn * md * sizeof(double), st) != cudaSuccess) return -1;
    if (H->nsig > 0) {
        const int nfar = (int)(H->plan.far.size() / 2);
        const dim3 g = blocks_for((int64_t)nfar * md, 128);
        if (md == 16) pair_product_kernel<16><<<g, 128, 0, st>>>(nfar, md, H->far_tau, H->kmat, H->xh, H->Pb);
        else if (md == 36) pair_product_kernel<36><<<g, 128, 0, st>>>(nfar, md, H->far_tau, H->kmat, H->xh, H->Pb);
        else pair_product_kernel<0><<<g, 128, 0, st>>>(nfar, md, H->far_tau, H->kmat, H->xh, H->Pb);
        couple_sum_kernel<<<blocks_for((int64_t)H->nsig * md, 128), 128, 0, st>>>(H->nsig, md, H->sig_nodes, H->far_ptr,
                                                                                 H->Pb, H->yh);
        launches += 2;
    }
    // downward pass: the top levels in one block, then the subtrees, one block each
    if (H->ntop_down > 0) {
        if (md == 16) down_top_kernel<16><<<1, 1024, 0, st>>>(H->ntop_down, md, H->top_down_off, H->top_down, H->parent, H->shiftT, H->yh);
        else if (md == 36) down_top_kernel<36><<<1, 1024, 0, st>>>(H->ntop_down, md, H->top_down_off, H->top_down, H->parent, H->shiftT, H->yh);
        else down_top_kernel<0><<<1, 1024, 0, st>>>(H->ntop_down, md, H->top_down_off, H->top_down, H->parent, H->shiftT, H->yh);
        ++launches;
    }
    if (H->nsub > 0 && H->sub_levels > 1) {
        if (md == 16) down_sub_kernel<16><<<H->nsub, 256, 0, st>>>(H->sub_levels, md, H->sub_off, H->sub_nodes, H->parent, H->shiftT, H->yh);
        else if (md == 36) down_sub_kernel<36><<<H->nsub, 256, 0, st>>>(H->sub_levels, md, H->sub_off, H->sub_nodes, H->parent, H->shiftT, H->yh);
        else down_sub_kernel<0><<<H->nsub, 256, 0, st>>>(H->sub_levels, md, H->sub_off, H->sub_nodes, H->parent, H->shiftT, H->yh);
        ++launches;
    }
    if (side && cudaStreamWaitEvent(st, H->ev_join, 0) != cudaSuccess) return -1;
    if (!far_only) {
        down_leaf_kernel<<<blocks_for(n, 128), 128, 0, st>>>(n, md, H->perm, H->leaf_of, H->coef, H->yh, -H->C, y_dev);
        ++launches;
    }
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}
}  // namespace
}  // namespace fl

extern "C" {

int fl_hmatrix_matvec(fl_hmatrix H, const double* x_dev, double* y_dev, void* stream) {
    if (!H) return FL_EINVAL;
    H->err.clear();
    if (!x_dev || !y_dev || x_dev == y_dev) return hm_fail(H, FL_EINVAL, "bad x / y (y must not be x)");
    if (!H->near_ready) return hm_fail(H, FL_EINVAL, "near field not set (fl_hmatrix_set_near)");
    if (cudaSetDevice(H->device) != cudaSuccess) return hm_fail(H, FL_ECUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    // a product is launched as the graph captured for this (x, y), captured on first use
    cudaGraphExec_t exec = nullptr;
    int launches = -1;
    for (const auto& g : H->graphs)
        if (g.x == x_dev && g.y == y_dev) {
            exec = g.exec;
            launches = g.launches;
        }
    if (!exec) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool capturing = st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
        cudaGetLastError();
        if (!H->cap && !capturing) {
            if (cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&H->side_st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&H->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&H->ev_join, cudaEventDisableTiming) != cudaSuccess)
                return hm_fail(H, FL_ECUDA, "product streams");
        }
        if (!capturing && H->graphs.size() < 8) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return hm_fail(H, FL_ECUDA, "graph capture");
            launches = fl::hm_enqueue(H, x_dev, y_dev, H->cap, H->side_st, false);
            const cudaError_t ec = cudaStreamEndCapture(H->cap, &graph);
            if (launches < 0 || ec != cudaSuccess || !graph) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return hm_fail(H, FL_ECUDA, "H-matrix product capture");
            }
            const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                cudaGetLastError();
                return hm_fail(H, FL_ECUDA, "H-matrix product graph");
            }
            H->graphs.push_back({x_dev, y_dev, exec, launches});
        }
    }
    if (exec) {
        if (cudaGraphLaunch(exec, st) != cudaSuccess) {
            cudaGetLastError();
            return hm_fail(H, FL_ECUDA, "H-matrix product graph launch");
        }
    } else {
        // inside a caller's capture, or more (x, y) pairs than kept graphs: launches on `st`
        launches = fl::hm_enqueue(H, x_dev, y_dev, st, nullptr, false);
        if (launches < 0) return hm_fail(H, FL_ECUDA, "H-matrix product launch");
    }
    count_launch(launches);
    return FL_OK;
}

int fl_hmatrix_info(fl_hmatrix H, int64_t* info) {
    if (!H || !info) return FL_EINVAL;
    info[0] = H->plan.nodes;
    info[1] = (int64_t)H->plan.far.size() / 2;
    info[2] = (int64_t)H->plan.near.size() / 2;
    info[3] = H->nnz;
    info[4] = H->bytes;
    info[5] = H->plan.depth;
    return FL_OK;
}

const char* fl_hmatrix_last_error(fl_hmatrix H) { return H ? H->err.c_str() : "null H-matrix handle"; }

int fl_hmatrix_solve(fl_hmatrix H, const double* b_dev, double* u_dev, const fl_solve_opts* o, fl_solve_info* info,
                     void* stream) {
    return fl_hmatrix_solve_shifted(H, 0.0, 1.0, b_dev, u_dev, o, info, stream);
}

int fl_hmatrix_solve_shifted(fl_hmatrix H, double alpha, double beta, const double* b_dev, double* u_dev,
                             const fl_solve_opts* o, fl_solve_info* info, void* stream) {
    if (!H) return FL_EINVAL;
    H->err.clear();
    if (!b_dev || !u_dev || b_dev == u_dev) return hm_fail(H, FL_EINVAL, "bad b / u");
    if (!(alpha >= 0.0) || !(beta > 0.0)) return hm_fail(H, FL_EINVAL, "alpha >= 0 and beta > 0 needed");
    if (!H->near_ready) return hm_fail(H, FL_EINVAL, "near field not set (fl_hmatrix_set_near)");
    fl_solve_opts d{};
    fl_default_solve_opts(&d);
    const fl_solve_opts& op = o ? *o : d;
    if (!(op.tol > 0.0) || op.maxit < 1) return hm_fail(H, FL_EINVAL, "tol must be > 0, maxit >= 1");
    if (cudaSetDevice(H->device) != cudaSuccess) return hm_fail(H, FL_ECUDA, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = H->plan.n;
    int rc;
    if (!H->cg_r) {
        if ((rc = hm_alloc(H, &H->cg_r, n)) || (rc = hm_alloc(H, &H->cg_z, n)) || (rc = hm_alloc(H, &H->cg_p, n)) ||
            (rc = hm_alloc(H, &H->cg_q, n)) || (rc = hm_alloc(H, &H->cg_dinv, n)) ||
            (rc = hm_alloc(H, &H->cg_part, 2 * HCG_BLOCKS)) || (rc = hm_alloc(H, &H->cg_scal, 4)))
            return rc;
        void* hp = nullptr;
        if (pool_host_alloc(&hp, 4 * sizeof(double)) != cudaSuccess) return hm_fail(H, FL_ENOMEM, "pinned scalars");
        H->cg_host = (double*)hp;
    }
    const fl::DevTables& mt = H->mesh->dev[H->pi];
    if (!H->dinv_ready || H->dinv_alpha != alpha || H->dinv_beta != beta) {
        hcg_diag_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, H->nz_ptr, H->nz_col, H->nz_val, alpha, beta, H->d,
                                                            mt.vod, mt.v2c_ptr, mt.v2c, mt.jac_orig, H->cg_dinv);
        count_launch();
        H->dinv_ready = true;
        H->dinv_alpha = alpha;
        H->dinv_beta = beta;
    }
    double* r = H->cg_r;
    double* z = H->cg_z;
    double* p = H->cg_p;
    double* q = H->cg_q;
    double* sc = H->cg_scal;  // [0] r.z (old), [1] r.z (new) / r.r, [2] p.q, [3] b.b
    double* hs = H->cg_host;
    auto dots = [&](const double* a, const double* b2, const double* c, const double* d2, double* out) {
        hcg_dots_kernel<<<HCG_BLOCKS, HCG_THREADS, 0, st>>>(n, a, b2, c, d2, H->cg_part);
        hcg_sum_kernel<<<1, 32, 0, st>>>(H->cg_part, out);
        count_launch(2);
    };
    hcg_start_kernel<<<HCG_BLOCKS, HCG_THREADS, 0, st>>>(n, b_dev, H->cg_dinv, u_dev, r, z, p);
    count_launch();
    dots(r, z, b_dev, b_dev, sc);  // sc[0] = r.z, sc[1] = b.b
    if (cudaMemcpyAsync(hs, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return hm_fail(H, FL_ECUDA, "solver scalars");
    const double bb = hs[1];
    fl_solve_info out{};
    out.outer_iterations = 1;
    out.status = FL_ENOTCONV;
    double rel = bb > 0.0 ? 1.0 : 0.0;
    if (bb == 0.0) out.status = FL_OK;
    int it = 0;
    while (out.status == FL_ENOTCONV && it < op.maxit) {
        if ((rc = fl_hmatrix_matvec(H, p, q, stream)) != FL_OK) return rc;
        if (alpha != 0.0 || beta != 1.0) {  // q = beta A p + alpha M p
            if ((rc = fl::mass_apply(H->mesh, H->s, 1, alpha, p, 1, beta, q, 1, q, 1, st)) != FL_OK)
                return hm_fail(H, rc, H->mesh->err);
        }
        dots(p, q, nullptr, nullptr, sc + 2);  // sc[2] = p.q
        hcg_update_kernel<<<HCG_BLOCKS, HCG_THREADS, 0, st>>>(n, sc, p, q, H->cg_dinv, u_dev, r, z);
        dots(r, z, r, r, sc + 1);  // sc[1] = r.z (new), sc[2] = r.r
        hcg_direction_kernel<<<HCG_BLOCKS, HCG_THREADS, 0, st>>>(n, sc, z, p);
        count_launch(2);
        ++it;
        if (cudaMemcpyAsync(hs, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return hm_fail(H, FL_ECUDA, "solver scalars");
        rel = std::sqrt(std::max(hs[2], 0.0) / bb);
        if (!(hs[1] > 0.0) && rel > op.tol) out.status = FL_ENOTSPD;
        else if (rel <= op.tol) out.status = FL_OK;
        // the direction kernel has moved beta's numerator: r.z (new) is the next old value
        if (cudaMemcpyAsync(sc, sc + 1, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return hm_fail(H, FL_ECUDA, "solver scalars");
    }
    out.iterations = it;
    out.rel_residual = rel;
    if (info) *info = out;
    return out.status;
}

}  // extern "C"
