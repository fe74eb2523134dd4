// Learned patch preconditioner and flexible conjugate gradients.
//
// Not in the paper.  The preconditioner is linear in the residual with a stencil that
// a small network computes from the geometry of each DOF's patch (the K nearest DOFs
// within two mesh edges):
//   g_i = ((x_{j_k} - x_i) / h_i, (y_{j_k} - y_i) / h_i)_k, log h_i, hop_i / 8, s
//   c_i = W3^T tanh(W2^T tanh(W1^T g_i + b1) + b2) + b3 + (1, 0, ..., 0)       (K + 1 values)
//   (M r)_i = (c_i0 r_i + sum_k c_ik r_{j_k}) / A_ii,   applied as (M + M^T) r / 2
// (h_i: mean edge length at the vertex, hop_i: mesh edges to the boundary, capped at 8).
// With W3 = b3 = 0 this is the Jacobi preconditioner, the initial state.  Training
// pairs (r = A e, e) give samples (g_i, x_i = normalised residual patch, t_i =
// e_i A_ii / sigma_i) and the loss mean (c(g_i) . x_i - t_i)^2 (for white-noise e the
// Frobenius fit of M to A^-1 on the pattern); forward, backward and Adam run in this
// file's kernels on float32 master weights; the stencil table is then computed with
// float16 weights and float32 sums.  Flexible CG uses it with the multigrid or Jacobi
// preconditioner as fallback; the float64 residual decides convergence.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "device.h"

struct fl_lp {
    int device = 0;
    fl_handle mesh = nullptr;  // not owned
    double s = 0.5;
    int64_t n = 0;
    int K = 12, F = 40, H = 64;  // F: length of a training sample row [g (2K + 3) | x (K + 1)]
    // patch tables (device)
    int* nbr = nullptr;     // n x K
    float* geo = nullptr;   // n x (2K + 3) geometry features
    float* coef = nullptr;  // n x (K + 1) stencil from the current parameters
    int *tptr = nullptr, *tsrc = nullptr;  // transpose incidence: DOF j <- (l * (K + 1) + k)
    // parameters: [W1 G x H | b1 H | W2 H x H | b2 H | W3 H x (K + 1) | b3 K + 1]
    int64_t nw = 0;
    float *w = nullptr, *m1 = nullptr, *m2 = nullptr, *g = nullptr;
    __half* w16 = nullptr;
    int adam_t = 0;
    // training set
    int64_t cap = 0, count = 0;
    float *X = nullptr, *T = nullptr;
    // scratch
    int64_t bcap = 0;
    float *Xb = nullptr, *Tb = nullptr, *H1 = nullptr, *H2 = nullptr, *D1 = nullptr, *D2 = nullptr, *DO = nullptr;
    float* dy = nullptr;
    float* loss = nullptr;
    double *vr = nullptr, *ve = nullptr, *vu = nullptr, *vx = nullptr;  // n-vectors
    float* sig = nullptr;
    float* diag = nullptr;   // A_ii of the bound matrix
    std::vector<void*> owned;
    std::string err;
};

namespace fl {
namespace lp {

static int fail(fl_lp* m, int code, const std::string& msg) {
    m->err = msg;
    return code;
}

template <typename T>
static T* dalloc(fl_lp* m, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    m->owned.push_back(p);
    return (T*)p;
}

static unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// counter-based generator (splitmix64, Steele, Lea & Flood 2014)
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// compiled network shape: K = 12 patch neighbours, hidden width 64
constexpr int KK = 12, HH = 64, FG = 2 * KK + 3, KO = KK + 1, FX = FG + KO;
constexpr int NW = FG * HH + HH + HH * HH + HH + HH * KO + KO;

// ------------------------------------------------------------------ samples --
// one thread per DOF: the sample row [g_i | x_i] (x: residual patch / sigma) and sigma
__global__ void features_kernel(int64_t n, const double* __restrict__ r, const int* __restrict__ nbr,
                                const float* __restrict__ geo, float* __restrict__ X, float* __restrict__ sig) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ss = r[i] * r[i];
    int cnt = 1;
    for (int k = 0; k < KK; ++k) {
        const int j = nbr[i * KK + k];
        if (j >= 0) {
            ss += r[j] * r[j];
            ++cnt;
        }
    }
    const double sg = sqrt(ss / cnt + 1e-30);
    float* x = X + i * FX;
    for (int f = 0; f < FG; ++f) x[f] = geo[i * FG + f];
    x[FG] = (float)(r[i] / sg);
    for (int k = 0; k < KK; ++k) {
        const int j = nbr[i * KK + k];
        x[FG + 1 + k] = (j >= 0) ? (float)(r[j] / sg) : 0.f;
    }
    sig[i] = (float)sg;
}

// targets t = e_i A_ii / sigma_i of the rows just written
__global__ void target_kernel(int64_t n, const double* e, const float* diag, const float* sig, float* T) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) T[i] = (float)(e[i] * (double)diag[i] / (double)sig[i]);
}

// ------------------------------------------------------------------ stencil --
// c_i from g_i with the network in float16 (shared memory) and float32 sums
__global__ void __launch_bounds__(128) coef_kernel(int64_t n, const float* __restrict__ geo,
                                                   const __half* __restrict__ w16, float* __restrict__ coef) {
    __shared__ __half wsh[NW];
    for (int e = threadIdx.x; e < NW; e += blockDim.x) wsh[e] = w16[e];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const __half* W1 = wsh;
    const __half* b1 = W1 + FG * HH;
    const __half* W2 = b1 + HH;
    const __half* b2 = W2 + HH * HH;
    const __half* W3 = b2 + HH;
    const __half* b3 = W3 + HH * KO;
    float g[FG];
#pragma unroll
    for (int f = 0; f < FG; ++f) g[f] = geo[i * FG + f];
    float h1[HH];
#pragma unroll
    for (int j = 0; j < HH; ++j) {
        float a = __half2float(b1[j]);
#pragma unroll
        for (int f = 0; f < FG; ++f) a = fmaf(g[f], __half2float(W1[f * HH + j]), a);
        h1[j] = tanhf(a);
    }
    float o[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) o[k] = __half2float(b3[k]);
#pragma unroll 1
    for (int q = 0; q < HH; ++q) {
        float a = __half2float(b2[q]);
#pragma unroll
        for (int j = 0; j < HH; ++j) a = fmaf(h1[j], __half2float(W2[j * HH + q]), a);
        const float h2 = tanhf(a);
#pragma unroll
        for (int k = 0; k < KO; ++k) o[k] = fmaf(h2, __half2float(W3[q * KO + k]), o[k]);
    }
    o[0] += 1.f;
#pragma unroll
    for (int k = 0; k < KO; ++k) coef[i * KO + k] = o[k];
}

// z = (M + M^T) r / 2 with (M r)_i = (c_i0 r_i + sum_k c_ik r_{j_k}) / A_ii
__global__ void apply_kernel(int64_t n, const double* __restrict__ r, const int* __restrict__ nbr,
                             const float* __restrict__ coef, const int* __restrict__ tptr,
                             const int* __restrict__ tsrc, const float* __restrict__ diag, double* __restrict__ z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = (double)coef[i * KO] * r[i];
    for (int k = 0; k < KK; ++k) {
        const int j = nbr[i * KK + k];
        if (j >= 0) a += (double)coef[i * KO + 1 + k] * r[j];
    }
    double b = 0.0;
    for (int e = tptr[i]; e < tptr[i + 1]; ++e) {
        const int src = tsrc[e];
        const int l = src / KO;
        b += (double)coef[src] * r[l] / (double)diag[l];
    }
    z[i] = 0.5 * (a / (double)diag[i] + b);
}

// ---------------------------------------------------------------- training --
// batch rows gathered from the training set by a counter-based draw
__global__ void gather_batch_kernel(int64_t B, const float* X, const float* T, int64_t count, uint64_t seed,
                                    uint64_t step, float* Xb, float* Tb) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t row = (int64_t)(splitmix64(seed ^ splitmix64(step * 0x100000001ull + (uint64_t)b)) % (uint64_t)count);
    for (int f = 0; f < FX; ++f) Xb[b * FX + f] = X[row * FX + f];
    Tb[b] = T[row];
}

// per sample: H1, H2, dO = dy x, dA2 = (W3 dO)(1 - H2^2), dA1 = (W2 dA2)(1 - H1^2), dy = 2 (y - t) / B
__global__ void __launch_bounds__(128) fwdbwd_kernel(int64_t B, const float* __restrict__ w,
                                                     const float* __restrict__ X, const float* __restrict__ T,
                                                     float* __restrict__ H1, float* __restrict__ H2,
                                                     float* __restrict__ D1, float* __restrict__ D2,
                                                     float* __restrict__ DO, float* __restrict__ dy) {
    __shared__ float wf[NW];
    for (int e = threadIdx.x; e < NW; e += blockDim.x) wf[e] = w[e];
    __syncthreads();
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= B) return;
    const float* W1 = wf;
    const float* b1 = W1 + FG * HH;
    const float* W2 = b1 + HH;
    const float* b2 = W2 + HH * HH;
    const float* W3 = b2 + HH;
    const float* b3 = W3 + HH * KO;
    const float* g = X + n * FX;
    const float* x = g + FG;
    float h1[HH];
#pragma unroll
    for (int j = 0; j < HH; ++j) {
        float a = b1[j];
#pragma unroll
        for (int f = 0; f < FG; ++f) a = fmaf(g[f], W1[f * HH + j], a);
        h1[j] = tanhf(a);
        H1[n * HH + j] = h1[j];
    }
    float o[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) o[k] = b3[k];
#pragma unroll 1
    for (int q = 0; q < HH; ++q) {
        float a = b2[q];
#pragma unroll
        for (int j = 0; j < HH; ++j) a = fmaf(h1[j], W2[j * HH + q], a);
        const float h2 = tanhf(a);
        H2[n * HH + q] = h2;
#pragma unroll
        for (int k = 0; k < KO; ++k) o[k] = fmaf(h2, W3[q * KO + k], o[k]);
    }
    o[0] += 1.f;
    float y = 0.f;
#pragma unroll
    for (int k = 0; k < KO; ++k) y = fmaf(o[k], x[k], y);
    const float gy = 2.f * (y - T[n]) / (float)B;
    dy[n] = gy;
    float dO[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        dO[k] = gy * x[k];
        DO[n * KO + k] = dO[k];
    }
    float d2[HH];
#pragma unroll 1
    for (int q = 0; q < HH; ++q) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < KO; ++k) a = fmaf(W3[q * KO + k], dO[k], a);
        const float h2 = H2[n * HH + q];
        D2[n * HH + q] = a * (1.f - h2 * h2);
    }
#pragma unroll
    for (int q = 0; q < HH; ++q) d2[q] = D2[n * HH + q];
#pragma unroll 1
    for (int j = 0; j < HH; ++j) {
        float a = 0.f;
#pragma unroll
        for (int q = 0; q < HH; ++q) a = fmaf(W2[j * HH + q], d2[q], a);
        D1[n * HH + j] = a * (1.f - h1[j] * h1[j]);
    }
}

// gradient rows, summed over the batch in sample order (deterministic); HH threads:
// blocks [0, FG): gW1 rows; [FG, FG+HH): gW2 rows; FG+HH: gb1; FG+HH+1: gb2;
// [FG+HH+2, FG+2HH+2): gW3 rows (KO threads); FG+2HH+2: gb3 (KO threads)
__global__ void grad_kernel(int64_t B, const float* __restrict__ X, const float* __restrict__ H1,
                            const float* __restrict__ H2, const float* __restrict__ D1, const float* __restrict__ D2,
                            const float* __restrict__ DO, float* __restrict__ g) {
    const int blk = blockIdx.x, j = threadIdx.x;
    float* gW1 = g;
    float* gb1 = gW1 + FG * HH;
    float* gW2 = gb1 + HH;
    float* gb2 = gW2 + HH * HH;
    float* gW3 = gb2 + HH;
    float* gb3 = gW3 + HH * KO;
    float a = 0.f;
    if (blk < FG) {
        for (int64_t n = 0; n < B; ++n) a = fmaf(X[n * FX + blk], D1[n * HH + j], a);
        gW1[blk * HH + j] = a;
    } else if (blk < FG + HH) {
        const int r = blk - FG;
        for (int64_t n = 0; n < B; ++n) a = fmaf(H1[n * HH + r], D2[n * HH + j], a);
        gW2[r * HH + j] = a;
    } else if (blk == FG + HH) {
        for (int64_t n = 0; n < B; ++n) a += D1[n * HH + j];
        gb1[j] = a;
    } else if (blk == FG + HH + 1) {
        for (int64_t n = 0; n < B; ++n) a += D2[n * HH + j];
        gb2[j] = a;
    } else if (blk < FG + 2 * HH + 2) {
        const int r = blk - (FG + HH + 2);
        if (j >= KO) return;
        for (int64_t n = 0; n < B; ++n) a = fmaf(H2[n * HH + r], DO[n * KO + j], a);
        gW3[r * KO + j] = a;
    } else {
        if (j >= KO) return;
        for (int64_t n = 0; n < B; ++n) a += DO[n * KO + j];
        gb3[j] = a;
    }
}

// loss = mean (y - t)^2 recovered from dy = 2 (y - t) / B: sum dy^2 B / 4
__global__ void loss_kernel(int64_t B, const float* dy, float* out) {
    __shared__ float sh[32];
    float s = 0.f;
    for (int64_t n = threadIdx.x; n < B; n += blockDim.x) s = fmaf(dy[n], dy[n], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
        *out = t * (float)B / 4.f;
    }
}

__global__ void adam_kernel(int64_t nw, float* w, const float* g, float* m1, float* m2, float lr, float b1c,
                            float b2c) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nw) return;
    const float gg = g[e];
    const float a = 0.9f * m1[e] + 0.1f * gg;
    const float b = 0.999f * m2[e] + 0.001f * gg * gg;
    m1[e] = a;
    m2[e] = b;
    w[e] -= lr * (a / b1c) / (sqrtf(b / b2c) + 1e-8f);
}

__global__ void to_half_kernel(int64_t nw, const float* w, __half* w16) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nw) w16[e] = __float2half_rn(w[e]);
}

// ------------------------------------------------------------- vector ops --
__global__ void sub_kernel(int64_t n, const double* a, const double* b, double* c) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] - b[i];
}
// x[i] ~ N(0, 1): Box-Muller on two splitmix64 draws of (seed, i)
__global__ void normal_kernel(int64_t n, uint64_t seed, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t a = splitmix64(seed ^ splitmix64(2 * (uint64_t)i)), b = splitmix64(seed ^ splitmix64(2 * (uint64_t)i + 1));
    const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0), u2 = ((b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    x[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
// e = -(x0 + d): the error of the iterate x0 + d of A x = 0 (solution 0)
__global__ void neg_sum_kernel(int64_t n, const double* a, const double* b, double* c) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) c[i] = -(a[i] + b[i]);
}
__global__ void neg_kernel(int64_t n, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = -x[i];
}
__global__ void diag_f_kernel(int64_t n, const double* A, int64_t lda, float* d) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = (float)A[i * lda + i];
}
__global__ void jacobi_kernel(int64_t n, const double* r, const float* d, double* z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = r[i] / (double)d[i];
}
constexpr int RB = 256;
__global__ void dotp_kernel(int64_t n, const double* a, const double* b, double* part) {
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
__global__ void dots_kernel(const double* part, int nparts, int count, double* out) {
    // out[c] = sum of part[c * nparts .. (c + 1) * nparts) in order
    const int c = threadIdx.x;
    if (c >= count) return;
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[c * nparts + i];
    out[c] = t;
}
// x += a p, r -= a q, a = sc[0] / sc[1] = (p.r) / (p.q)
__global__ void fcg_xr_kernel(int64_t n, const double* sc, double* x, double* r, const double* p, const double* q) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = sc[0] / sc[1];
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
}
// p = z + beta p with beta = -sc[2] / sc[1] (one-step flexible orthogonalisation); restart: beta = 0
__global__ void fcg_p_kernel(int64_t n, const double* sc, const double* z, double* p, int restart) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = restart ? z[i] : fma(-sc[2] / sc[1], p[i], z[i]);
}

}  // namespace lp
}  // namespace fl

namespace fl {
namespace lp {
// float16 copy of the parameters and the stencil table they give
static void refresh(fl_lp* m, cudaStream_t st) {
    to_half_kernel<<<nb(m->nw), 256, 0, st>>>(m->nw, m->w, m->w16);
    coef_kernel<<<nb(m->n, 128), 128, 0, st>>>(m->n, m->geo, m->w16, m->coef);
    fl::count_launch(2);
}
}  // namespace lp
}  // namespace fl

using namespace fl;
using namespace fl::lp;

extern "C" {

int fl_patches(fl_handle h, double s, int K, int32_t* nbr_host, double* hlen_host, int32_t* hop_host) {
    if (!h || K < 1 || K > 20) return FL_EINVAL;
    if (h->sym_K) return sym_unsupported(h, "fl_patches");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (P.dim != 2) return set_err(h, FL_ENOTIMPL, "patches are defined for 2D meshes");
    const int64_t nv = P.nv;
    std::vector<double> hl(nv, 0.0);
    for (int64_t v = 0; v < nv; ++v) {
        double sum = 0.0;
        const int c = P.nbr_ptr[v + 1] - P.nbr_ptr[v];
        for (int q = P.nbr_ptr[v]; q < P.nbr_ptr[v + 1]; ++q) {
            const int w = P.nbr[q];
            const double dx = P.V[2 * w] - P.V[2 * v], dy = P.V[2 * w + 1] - P.V[2 * v + 1];
            sum += std::sqrt(dx * dx + dy * dy);
        }
        hl[v] = c ? sum / c : 0.0;
    }
    std::vector<int> hop(nv, 8), frontier, next;
    for (int64_t v = 0; v < nv; ++v)
        if (P.onb[v]) {
            hop[v] = 0;
            frontier.push_back((int)v);
        }
    for (int d = 1; d <= 8 && !frontier.empty(); ++d) {
        next.clear();
        for (int v : frontier)
            for (int q = P.nbr_ptr[v]; q < P.nbr_ptr[v + 1]; ++q) {
                const int w = P.nbr[q];
                if (hop[w] > d) {
                    hop[w] = d;
                    next.push_back(w);
                }
            }
        frontier.swap(next);
    }
    std::vector<int> mark(nv, -1);
    std::vector<std::pair<double, int>> cand;
    for (int64_t i = 0; i < P.n; ++i) {
        const int v = P.vod[i];
        cand.clear();
        auto consider = [&](int w) {
            if (w == v || mark[w] == (int)i || P.dov[w] < 0) return;
            mark[w] = (int)i;
            const double dx = P.V[2 * w] - P.V[2 * v], dy = P.V[2 * w + 1] - P.V[2 * v + 1];
            cand.push_back({std::sqrt(dx * dx + dy * dy), w});
        };
        for (int q = P.nbr_ptr[v]; q < P.nbr_ptr[v + 1]; ++q) {
            const int w = P.nbr[q];
            consider(w);
            for (int q2 = P.nbr_ptr[w]; q2 < P.nbr_ptr[w + 1]; ++q2) consider(P.nbr[q2]);
        }
        std::sort(cand.begin(), cand.end());
        for (int k = 0; k < K; ++k) nbr_host[i * K + k] = (k < (int)cand.size()) ? P.dov[cand[k].second] : -1;
        if (hlen_host) hlen_host[i] = hl[v];
        if (hop_host) hop_host[i] = hop[v];
    }
    return FL_OK;
}

int fl_lp_create(fl_lp_handle* out, fl_handle mesh, double s, int K, int hidden, uint64_t seed) {
    if (!out || !mesh) return FL_EINVAL;
    if (mesh->sym_K) return sym_unsupported(mesh, "fl_lp_create");
    if (K != KK || hidden != HH) return FL_ENOTIMPL;  // the kernels are compiled for K = 12, width 64
    fl_lp* m = new (std::nothrow) fl_lp;
    if (!m) return FL_ENOMEM;
    cudaGetDevice(&m->device);
    m->mesh = mesh;
    m->s = s;
    m->K = K;
    m->H = hidden;
    m->F = FX;
    int64_t n = 0;
    int r = fl_num_dofs(mesh, s, &n);
    if (r != FL_OK) {
        delete m;
        return r;
    }
    m->n = n;
    std::vector<int32_t> nbr((size_t)n * K), hop(n);
    std::vector<double> hl(n);
    r = fl_patches(mesh, s, K, nbr.data(), hl.data(), hop.data());
    if (r != FL_OK) {
        delete m;
        return r;
    }
    std::vector<int32_t> vod(n);
    fl_dof_vertices(mesh, s, vod.data());
    const int pi = plan_for(mesh, s);
    const Plan& P = mesh->plan[pi];
    std::vector<float> geo((size_t)n * FG, 0.f);
    for (int64_t i = 0; i < n; ++i) {
        const int v = vod[i];
        for (int k = 0; k < K; ++k) {
            const int j = nbr[i * K + k];
            if (j < 0) continue;
            const int w = vod[j];
            geo[i * FG + 2 * k] = (float)((P.V[2 * w] - P.V[2 * v]) / hl[i]);
            geo[i * FG + 2 * k + 1] = (float)((P.V[2 * w + 1] - P.V[2 * v + 1]) / hl[i]);
        }
        geo[i * FG + 2 * K] = (float)std::log(hl[i]);
        geo[i * FG + 2 * K + 1] = (float)(hop[i] / 8.0);
        geo[i * FG + 2 * K + 2] = (float)s;
    }
    // transpose incidence: entry (l, k) of the stencil table acts on DOF j
    std::vector<int> tcnt(n + 1, 0);
    for (int64_t l = 0; l < n; ++l) {
        ++tcnt[l + 1];
        for (int k = 0; k < K; ++k)
            if (nbr[l * K + k] >= 0) ++tcnt[nbr[l * K + k] + 1];
    }
    for (int64_t j = 0; j < n; ++j) tcnt[j + 1] += tcnt[j];
    std::vector<int> tsrc(tcnt[n]);
    std::vector<int> fillp(tcnt.begin(), tcnt.end() - 1);
    for (int64_t l = 0; l < n; ++l) {
        tsrc[fillp[l]++] = (int)(l * KO);
        for (int k = 0; k < K; ++k) {
            const int j = nbr[l * K + k];
            if (j >= 0) tsrc[fillp[j]++] = (int)(l * KO + 1 + k);
        }
    }
    m->nw = NW;
    // parameters: hidden layers seeded (variance 1 / fan-in), output layer zero (Jacobi)
    std::vector<float> w(m->nw, 0.f);
    uint64_t ctr = seed;
    auto normal = [&]() {  // Box-Muller on two splitmix64 draws
        const double u1 = ((splitmix64(ctr++) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((splitmix64(ctr++) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int64_t e = 0; e < (int64_t)FG * HH; ++e) w[e] = (float)(normal() / std::sqrt((double)FG));
    const int64_t o2 = (int64_t)FG * HH + HH;
    for (int64_t e = 0; e < (int64_t)HH * HH; ++e) w[o2 + e] = (float)(normal() / std::sqrt((double)HH));
    m->nbr = dalloc<int>(m, nbr.size());
    m->geo = dalloc<float>(m, geo.size());
    m->coef = dalloc<float>(m, (size_t)n * KO);
    m->tptr = dalloc<int>(m, n + 1);
    m->tsrc = dalloc<int>(m, tsrc.size());
    m->w = dalloc<float>(m, m->nw);
    m->m1 = dalloc<float>(m, m->nw);
    m->m2 = dalloc<float>(m, m->nw);
    m->g = dalloc<float>(m, m->nw);
    m->w16 = dalloc<__half>(m, m->nw);
    m->loss = dalloc<float>(m, 1);
    m->vr = dalloc<double>(m, n);
    m->ve = dalloc<double>(m, n);
    m->vu = dalloc<double>(m, n);
    m->vx = dalloc<double>(m, n);
    m->sig = dalloc<float>(m, n);
    m->diag = dalloc<float>(m, n);
    if (!m->nbr || !m->geo || !m->coef || !m->tptr || !m->tsrc || !m->w || !m->m1 || !m->m2 || !m->g || !m->w16 ||
        !m->loss || !m->vr || !m->ve || !m->vu || !m->vx || !m->sig || !m->diag) {
        fl_lp_destroy(m);
        return FL_ENOMEM;
    }
    cudaMemcpy(m->nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(m->geo, geo.data(), geo.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(m->tptr, tcnt.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(m->tsrc, tsrc.data(), tsrc.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(m->w, w.data(), m->nw * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(m->m1, 0, m->nw * sizeof(float));
    cudaMemset(m->m2, 0, m->nw * sizeof(float));
    cudaMemset(m->diag, 0, n * sizeof(float));
    refresh(m, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        fl_lp_destroy(m);
        return FL_ECUDA;
    }
    *out = m;
    return FL_OK;
}

const char* fl_lp_last_error(fl_lp_handle m) { return m ? m->err.c_str() : ""; }

int64_t fl_lp_num_params(fl_lp_handle m) { return m ? m->nw : 0; }
int fl_lp_num_features(fl_lp_handle m) { return m ? m->F : 0; }
int64_t fl_lp_num_samples(fl_lp_handle m) { return m ? m->count : 0; }

int fl_lp_get_params(fl_lp_handle m, float* host) {
    if (!m || !host) return FL_EINVAL;
    return cudaMemcpy(host, m->w, m->nw * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? FL_OK : FL_ECUDA;
}

int fl_lp_set_params(fl_lp_handle m, const float* host) {
    if (!m || !host) return FL_EINVAL;
    if (cudaMemcpy(m->w, host, m->nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return FL_ECUDA;
    refresh(m, nullptr);
    return cudaDeviceSynchronize() == cudaSuccess ? FL_OK : FL_ECUDA;
}

// the diagonal the preconditioner divides by (and the training targets multiply by)
int fl_lp_stencil(fl_lp_handle m, float* host) {
    if (!m || !host) return FL_EINVAL;
    return cudaMemcpy(host, m->coef, (size_t)m->n * KO * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? FL_OK
               : FL_ECUDA;
}

int fl_lp_bind(fl_lp_handle m, const double* A_dev, int64_t lda, void* stream) {
    if (!m || !A_dev || lda < m->n) return FL_EINVAL;
    diag_f_kernel<<<nb(m->n), 256, 0, (cudaStream_t)stream>>>(m->n, A_dev, lda, m->diag);
    fl::count_launch();
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

int fl_lp_features(fl_lp_handle m, const double* r_dev, float* X_dev, float* sig_dev, void* stream) {
    if (!m || !r_dev || !X_dev || !sig_dev) return FL_EINVAL;
    features_kernel<<<nb(m->n), 256, 0, (cudaStream_t)stream>>>(m->n, r_dev, m->nbr, m->geo, X_dev, sig_dev);
    fl::count_launch();
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

int fl_lp_apply(fl_lp_handle m, const double* r_dev, double* z_dev, void* stream) {
    if (!m || !r_dev || !z_dev) return FL_EINVAL;
    apply_kernel<<<nb(m->n), 256, 0, (cudaStream_t)stream>>>(m->n, r_dev, m->nbr, m->coef, m->tptr, m->tsrc, m->diag,
                                                             z_dev);
    fl::count_launch();
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

static int ensure_batch(fl_lp* m, int64_t B) {
    if (m->bcap >= B) return FL_OK;
    const int F = m->F, H = m->H;
    m->DO = dalloc<float>(m, (size_t)B * KO);
    m->Xb = dalloc<float>(m, (size_t)B * F);
    m->Tb = dalloc<float>(m, B);
    m->H1 = dalloc<float>(m, (size_t)B * H);
    m->H2 = dalloc<float>(m, (size_t)B * H);
    m->D1 = dalloc<float>(m, (size_t)B * H);
    m->D2 = dalloc<float>(m, (size_t)B * H);
    m->dy = dalloc<float>(m, B);
    if (!m->Xb || !m->Tb || !m->H1 || !m->H2 || !m->D1 || !m->D2 || !m->DO || !m->dy) return FL_ENOMEM;
    m->bcap = B;
    return FL_OK;
}

static void fwd_bwd(fl_lp* m, int64_t B, const float* X, const float* T, cudaStream_t st) {
    fwdbwd_kernel<<<nb(B, 128), 128, 0, st>>>(B, m->w, X, T, m->H1, m->H2, m->D1, m->D2, m->DO, m->dy);
    grad_kernel<<<FG + 2 * HH + 3, HH, 0, st>>>(B, X, m->H1, m->H2, m->D1, m->D2, m->DO, m->g);
    loss_kernel<<<1, 256, 0, st>>>(B, m->dy, m->loss);
    fl::count_launch(3);
}

int fl_lp_loss_grad(fl_lp_handle m, int64_t B, const float* X_dev, const float* T_dev, float* loss_host,
                    float* grad_host, void* stream) {
    if (!m || B < 1 || !X_dev || !T_dev) return FL_EINVAL;
    if (ensure_batch(m, B) != FL_OK) return fail(m, FL_ENOMEM, "batch scratch");
    cudaStream_t st = (cudaStream_t)stream;
    fwd_bwd(m, B, X_dev, T_dev, st);
    if (loss_host) cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (grad_host) cudaMemcpyAsync(grad_host, m->g, m->nw * sizeof(float), cudaMemcpyDeviceToHost, st);
    return cudaStreamSynchronize(st) == cudaSuccess ? FL_OK : fail(m, FL_ECUDA, "gradient");
}

int fl_lp_add_pairs(fl_lp_handle m, const double* A_dev, int64_t lda, const double* E_dev, int64_t lde, int count,
                    void* stream) {
    if (!m || !A_dev || lda < m->n || !E_dev || lde < m->n || count < 0) return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = m->n;
    const int64_t need = m->count + (int64_t)count * n;
    if (need > m->cap) {
        const int64_t cap = std::max<int64_t>(need, 2 * m->cap);
        float* X = nullptr;
        float* T = nullptr;
        if (cudaMalloc((void**)&X, (size_t)cap * m->F * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&T, (size_t)cap * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            if (X) cudaFree(X);
            return fail(m, FL_ENOMEM, "training set");
        }
        if (m->count) {
            cudaMemcpyAsync(X, m->X, (size_t)m->count * m->F * sizeof(float), cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(T, m->T, (size_t)m->count * sizeof(float), cudaMemcpyDeviceToDevice, st);
        }
        cudaStreamSynchronize(st);
        if (m->X) cudaFree(m->X);
        if (m->T) cudaFree(m->T);
        m->X = X;
        m->T = T;
        m->cap = cap;
    }
    diag_f_kernel<<<nb(n), 256, 0, st>>>(n, A_dev, lda, m->diag);
    fl::count_launch();
    for (int c = 0; c < count; ++c) {
        const double* e = E_dev + (size_t)c * lde;
        if (fl::gemv(FL_F64, A_dev, lda, n, e, 1, m->vr, 1, nullptr, st) != cudaSuccess)
            return fail(m, FL_ECUDA, "residual of a pair");
        float* X = m->X + (size_t)m->count * m->F;
        features_kernel<<<nb(n), 256, 0, st>>>(n, m->vr, m->nbr, m->geo, X, m->sig);
        target_kernel<<<nb(n), 256, 0, st>>>(n, e, m->diag, m->sig, m->T + m->count);
        fl::count_launch(2);
        m->count += n;
    }
    return cudaGetLastError() == cudaSuccess ? FL_OK : fail(m, FL_ECUDA, "pairs");
}

int fl_lp_collect(fl_lp_handle m, const double* A_dev, int64_t lda, const double* b_dev, int nk, const int* ks,
                  void* stream) {
    if (!m || !A_dev || !b_dev || nk < 1 || !ks) return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = m->n;
    fl_solve_opts o;
    fl_default_solve_opts(&o);
    o.tol = 1e-11;
    fl_solve_info info;
    int r = fl_solve(m->mesh, n, A_dev, lda, b_dev, m->vu, &o, &info, stream);
    if (r != FL_OK && r != FL_ENOTCONV) return fail(m, r, "reference solve");
    for (int q = 0; q < nk; ++q) {
        o.tol = 1e-300;
        o.maxit = std::max(1, ks[q]);
        r = fl_solve(m->mesh, n, A_dev, lda, b_dev, m->vx, &o, &info, stream);  // Jacobi-PCG iterate x_k
        if (r != FL_OK && r != FL_ENOTCONV) return fail(m, r, "iterate");
        sub_kernel<<<nb(n), 256, 0, st>>>(n, m->vu, m->vx, m->ve);  // e_k = u - x_k
        fl::count_launch();
        r = fl_lp_add_pairs(m, A_dev, lda, m->ve, n, 1, stream);
        if (r != FL_OK) return r;
    }
    return FL_OK;
}

int fl_lp_collect_noise(fl_lp_handle m, const double* A_dev, int64_t lda, int count, int nk, const int* ks,
                        uint64_t seed, void* stream) {
    if (!m || !A_dev || lda < m->n || count < 1 || nk < 1 || !ks) return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = m->n;
    fl_solve_opts o;
    fl_default_solve_opts(&o);
    o.tol = 1e-300;
    fl_solve_info info;
    for (int c = 0; c < count; ++c) {
        normal_kernel<<<nb(n), 256, 0, st>>>(n, splitmix64(seed + (uint64_t)c), m->vu);  // x0
        fl::count_launch();
        // b' = -A x0: Jacobi-PCG on A d = b' from 0 is CG on A x = 0 from x0, with x = x0 + d
        if (fl::gemv(FL_F64, A_dev, lda, n, m->vu, 1, m->vr, 1, nullptr, st) != cudaSuccess)
            return fail(m, FL_ECUDA, "start residual");
        neg_kernel<<<nb(n), 256, 0, st>>>(n, m->vr);
        fl::count_launch();
        for (int q = 0; q < nk; ++q) {
            if (ks[q] <= 0) {
                cudaMemcpyAsync(m->ve, m->vu, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
                neg_kernel<<<nb(n), 256, 0, st>>>(n, m->ve);  // e = -x0
                fl::count_launch();
            } else {
                o.maxit = ks[q];
                const int r = fl_solve(m->mesh, n, A_dev, lda, m->vr, m->vx, &o, &info, stream);
                if (r != FL_OK && r != FL_ENOTCONV) return fail(m, r, "iterate");
                neg_sum_kernel<<<nb(n), 256, 0, st>>>(n, m->vu, m->vx, m->ve);
                fl::count_launch();
            }
            const int r = fl_lp_add_pairs(m, A_dev, lda, m->ve, n, 1, stream);
            if (r != FL_OK) return r;
        }
    }
    return FL_OK;
}

int fl_lp_train(fl_lp_handle m, int steps, int64_t batch, float lr, uint64_t seed, float* loss_host, void* stream) {
    if (!m || steps < 1 || batch < 1 || !(lr > 0)) return FL_EINVAL;
    if (m->count < 1) return fail(m, FL_EINVAL, "no training pairs");
    if (ensure_batch(m, batch) != FL_OK) return fail(m, FL_ENOMEM, "batch scratch");
    cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < steps; ++k) {
        gather_batch_kernel<<<nb(batch), 256, 0, st>>>(batch, m->X, m->T, m->count, seed, (uint64_t)k, m->Xb, m->Tb);
        fl::count_launch();
        fwd_bwd(m, batch, m->Xb, m->Tb, st);
        ++m->adam_t;
        const float b1c = 1.f - std::pow(0.9f, (float)m->adam_t), b2c = 1.f - std::pow(0.999f, (float)m->adam_t);
        adam_kernel<<<nb(m->nw), 256, 0, st>>>(m->nw, m->w, m->g, m->m1, m->m2, lr, b1c, b2c);
        fl::count_launch();
    }
    refresh(m, st);
    if (loss_host) cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    return cudaStreamSynchronize(st) == cudaSuccess ? FL_OK : fail(m, FL_ECUDA, "training");
}

void fl_lp_destroy(fl_lp_handle m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    for (void* p : m->owned) cudaFree(p);
    if (m->X) cudaFree(m->X);
    if (m->T) cudaFree(m->T);
    delete m;
}

// ---------------------------------------------------------- flexible CG --
int fl_fcg_solve(fl_handle h, int64_t n, const double* A_dev, int64_t lda, const double* b_dev, double* u_dev,
                 fl_lp_handle lp, fl_mg_handle mg, double tol, int maxit, fl_fcg_info* info, void* stream) {
    if (!h || !A_dev || !b_dev || !u_dev || n < 1 || lda < n || !(tol > 0) || maxit < 1) return FL_EINVAL;
    if (lp && lp->n != n) return set_err(h, FL_EINVAL, "learned preconditioner built for another size");
    cudaStream_t st = (cudaStream_t)stream;
    // workspace: r, z, p, q, t, diag (as float), partial sums, scalars
    std::vector<void*> mine;
    auto al = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        mine.push_back(p);
        return p;
    };
    double* r = (double*)al(n * 8);
    double* z = (double*)al(n * 8);
    double* p = (double*)al(n * 8);
    double* q = (double*)al(n * 8);
    double* t = (double*)al(n * 8);
    float* dg = (float*)al(n * 4);
    double* part = (double*)al(4 * RB * 8);
    double* sc = (double*)al(8 * 8);
    double* hs = nullptr;
    auto release = [&]() {
        for (void* v : mine) cudaFree(v);
        if (hs) cudaFreeHost(hs);
    };
    if (!r || !z || !p || !q || !t || !dg || !part || !sc || cudaMallocHost((void**)&hs, 8 * sizeof(double)) != cudaSuccess) {
        release();
        return set_err(h, FL_ENOMEM, "flexible CG workspace");
    }
    const unsigned g = nb(n);
    diag_f_kernel<<<g, 256, 0, st>>>(n, A_dev, lda, dg);
    fl::count_launch();
    if (lp) fl_lp_bind(lp, A_dev, lda, stream);
    // preconditioner in use: 2 learned, 1 multigrid, 0 Jacobi
    int mode = lp ? 2 : (mg ? 1 : 0);
    int fallback_at = -1;
    auto precond = [&](const double* rin, double* zout) -> int {
        if (mode == 2) return fl_lp_apply(lp, rin, zout, stream);
        if (mode == 1) return fl::mg_precondition(mg, rin, zout, st);
        jacobi_kernel<<<g, 256, 0, st>>>(n, rin, dg, zout);
        fl::count_launch();
        return FL_OK;
    };
    // several dot products in one pass of partial sums
    auto dots = [&](std::initializer_list<std::pair<const double*, const double*>> pr, double* out) {
        int c = 0;
        for (const auto& ab : pr) {
            dotp_kernel<<<RB, 256, 0, st>>>(n, ab.first, ab.second, part + c * RB);
            ++c;
        }
        dots_kernel<<<1, 32, 0, st>>>(part, RB, c, out);
        fl::count_launch(c + 1);
    };
    cudaMemsetAsync(u_dev, 0, n * sizeof(double), st);
    cudaMemcpyAsync(r, b_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    int rc = precond(r, z);
    if (rc != FL_OK) {
        release();
        return set_err(h, rc, "preconditioner");
    }
    cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    dots({{r, r}}, sc + 4);  // sc[4] = b.b
    cudaMemcpyAsync(hs + 4, sc + 4, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        release();
        return set_err(h, FL_ECUDA, "flexible CG start");
    }
    const double bb = hs[4];
    double rr = bb, rr_window = bb;
    int it = 0, status = (bb == 0.0) ? FL_OK : FL_ENOTCONV, restart = 0, since = 0;
    while (status == FL_ENOTCONV && it < maxit) {
        if (fl::gemv(FL_F64, A_dev, lda, n, p, 1, q, 1, nullptr, st) != cudaSuccess) {
            release();
            return set_err(h, FL_ECUDA, "matvec");
        }
        dots({{p, r}, {p, q}}, sc);  // sc[0] = p.r, sc[1] = p.q
        fcg_xr_kernel<<<g, 256, 0, st>>>(n, sc, u_dev, r, p, q);
        fl::count_launch();
        rc = precond(r, z);
        if (rc != FL_OK) {
            release();
            return set_err(h, rc, "preconditioner");
        }
        dots({{z, q}, {r, r}, {z, r}}, sc + 2);  // sc[2] = z.q, sc[3] = r.r, sc[4] = z.r
        cudaMemcpyAsync(hs, sc, 5 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            release();
            return set_err(h, FL_ECUDA, "flexible CG step");
        }
        ++it;
        ++since;
        if (!(hs[1] > 0.0)) {
            status = FL_ENOTSPD;
            break;
        }
        rr = hs[3];
        if (rr <= tol * tol * bb) {
            status = FL_OK;
            break;
        }
        // stall or a preconditioned residual that is not a descent direction: fall back
        const bool bad = !std::isfinite(hs[4]) || !(hs[4] > 0.0) || !std::isfinite(hs[2]);
        const bool slow = since >= 10 && rr > 0.81 * rr_window;  // < 10 % residual reduction over 10 steps
        if (since >= 10 && !slow) {
            rr_window = rr;
            since = 0;
        }
        if (mode != 0 && (bad || slow) && !(mode == 1 && !lp)) {
            mode = (mode == 2 && mg) ? 1 : 0;
            if (fallback_at < 0) fallback_at = it;
            precond(r, z);
            restart = 1;
            rr_window = rr;
            since = 0;
        } else if (bad) {
            status = FL_ENOTSPD;
            break;
        }
        fcg_p_kernel<<<g, 256, 0, st>>>(n, sc, z, p, restart);
        fl::count_launch();
        restart = 0;
    }
    // the float64 residual decides: b - A u recomputed
    fl::gemv(FL_F64, A_dev, lda, n, u_dev, 1, t, 1, nullptr, st);
    sub_kernel<<<g, 256, 0, st>>>(n, b_dev, t, t);
    fl::count_launch();
    dots({{t, t}}, sc + 5);
    cudaMemcpyAsync(hs + 5, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    const double rel = bb > 0 ? std::sqrt(hs[5] / bb) : 0.0;
    if (status == FL_OK && rel > tol * 1.01) status = FL_ENOTCONV;
    if (info) {
        info->iterations = it;
        info->fallback_at = fallback_at;
        info->final_preconditioner = mode;
        info->rel_residual = rel;
        info->status = status;
    }
    release();
    return status;
}

}  // extern "C"
