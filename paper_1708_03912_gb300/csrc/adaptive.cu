// Adaptive refinement on the device (Section 4 and Appendix A of arXiv:1708.03912): the
// strong form (-Delta)^s u_h at the points of a cell rule, the Babuska-Rheinboldt indicators
// and maximum marking.  The refinement of the marked cells is host code (refine.cpp).
//
// Lemma 4.1 writes (-Delta)^s u_h(x), x inside the cell K0, as regular integrals over cell
// boundaries (eq. (8); eq. (9), with a logarithmic kernel, when s = 1 - d/2).  With
// m = d + 2s - 2, n_K the outward normal of K and C = C(d, s):
//   (-Delta)^s u_h(x) / C = (1/m) int_{dK0} n.grad u_K0 |x-y|^{-m} - u(x)/(2s) int_{dK0} n.(x-y) |x-y|^{-d-2s}
//       + sum_{K != K0} [ 1/(2sm) int_{dK} n.grad u_K |x-y|^{-m} - 1/(2s) int_{dK} u(y) n.(x-y) |x-y|^{-d-2s} ].
// Here the sum is gathered by facet instead of by cell.  Both sides of a facet see the same
// quadrature points, so the discrete sums agree up to rounding:
//   * a facet e not on dK0 between K+ and K- (n_e outward of K+) contributes
//     1/(2sm) int_e n_e.(grad u_K+ - grad u_K-) |x-y|^{-m}, the jump of the normal derivative:
//     the u(y) terms of its two sides cancel, u_h being continuous;
//   * a boundary facet not on dK0 contributes 1/(2sm) int_e n.grad u_K |x-y|^{-m}
//     - 1/(2s) int_e u(y) n.(x-y) |x-y|^{-d-2s}; the second part vanishes unless boundary
//     vertices carry degrees of freedom;
//   * a facet e of K0 with neighbour K' (n0 outward of K0) contributes
//     int_e [(1/m) n0.grad u_K0 - 1/(2sm) n0.grad u_K'] |x-y|^{-m}
//     - 1/(2s) int_e (u(x) - u(y)) n0.(x-y) |x-y|^{-d-2s}, with u(x) - u(y) = grad u_K0.(x-y)
//     (u_h is linear on K0); on the boundary, without K', the first bracket keeps its first
//     term and u(x) - u(y) becomes u(x).
// In the log case |x-y|^{-m} / m becomes log(1/|x-y|) (and 1/(2sm) becomes 1/(2s)).  The
// facets of K0 are integrated by Gauss-Legendre of order k_near, all others by order k_edge
// (1D: the facets are points).
//
// Kernels: sf_prep (cell gradients and the points, in the planner's spatial cell order),
// sf_facet (per facet and Gauss point: the point and its coefficient), sf_far_dw (2D with s in
// {1/4, 1/2, 3/4}: the sum over the facets that share no vertex with K0, in double-word
// arithmetic on the float32 pipe, coordinates relative to an origin per block), sf_far_f64
// (other s, and 1D: the same facets in float64), sf_near (float64: the facets of K0, the other
// facets through a vertex of K0 -- the ones close to x, where double-word coordinates, good to
// 2^-48 of their size, would lose the relative accuracy of x - y -- and the sum of the parts).
// Every sum runs in a fixed order: the result is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "cluster.h"
#include "context.h"
#include "device.h"

namespace fl {
namespace {

#define SF_TRY(...)                 \
    do {                            \
        int r_ = (__VA_ARGS__);     \
        if (r_ != FL_OK) return r_; \
    } while (0)
#define SF_CUDA(h, x)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (x);                                                                             \
        if (e_ != cudaSuccess) return set_err(h, FL_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int SF_THREADS = 128;
constexpr int SF_TREC = 512;   // facet points per shared-memory tile
constexpr int SF_MAXK_CELL = 16, SF_MAXK_EDGE = 32, SF_MAXK_NEAR = 64;

double frac_const(int d, double s) {
    // C(d, s) = 2^{2s} s Gamma((d + 2s)/2) / (pi^{d/2} Gamma(1 - s))
    return std::pow(2.0, 2.0 * s) * s * std::tgamma((d + 2.0 * s) / 2.0) /
           (std::pow(M_PI, d / 2.0) * std::tgamma(1.0 - s));
}

// ------------------------------------------------------------------ kernels --

// gradients of u_h on every cell (original order) and the cell-rule points (internal order)
__global__ void sf_prep_kernel(int64_t nc, int d, int q, const int* __restrict__ perm, const int* __restrict__ cells,
                               const double* __restrict__ V, const int* __restrict__ dov, const double* __restrict__ u,
                               const double* __restrict__ lam, double* __restrict__ grad, double* __restrict__ X) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int K = perm[k];
    const int* c = cells + (int64_t)K * (d + 1);
    double uv[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j <= d; ++j) {
        const int i = dov[c[j]];
        uv[j] = i >= 0 ? u[i] : 0.0;
    }
    if (d == 1) {
        const double x0 = V[c[0]], x1 = V[c[1]];
        grad[K] = (uv[1] - uv[0]) / (x1 - x0);
        for (int a = 0; a < q; ++a) X[k * q + a] = x0 + lam[a] * (x1 - x0);
    } else {
        const double p0x = V[2 * c[0]], p0y = V[2 * c[0] + 1];
        const double e1x = V[2 * c[1]] - p0x, e1y = V[2 * c[1] + 1] - p0y;
        const double e2x = V[2 * c[2]] - p0x, e2y = V[2 * c[2] + 1] - p0y;
        const double du1 = uv[1] - uv[0], du2 = uv[2] - uv[0];
        const double det = e1x * e2y - e1y * e2x;
        grad[2 * K] = (du1 * e2y - du2 * e1y) / det;
        grad[2 * K + 1] = (e1x * du2 - e2x * du1) / det;
        for (int a = 0; a < q; ++a) {
            const double l1 = lam[2 * a], l2 = lam[2 * a + 1];
            X[2 * (k * q + a)] = p0x + l1 * e1x + l2 * e2x;
            X[2 * (k * q + a) + 1] = p0y + l1 * e1y + l2 * e2y;
        }
    }
}

// per facet e and Gauss point g: the point y, cA = w |e| J_e cA_scale (J_e the jump of the
// normal derivative, the one-sided value on the boundary) and, on boundary facets,
// cB = w |e| u(y) cB_scale
__global__ void sf_facet_kernel(int64_t nfac, int64_t nint, int d, int ke, const int* __restrict__ fac,
                                const double* __restrict__ fn, const double* __restrict__ V, const int* __restrict__ dov,
                                const double* __restrict__ u, const double* __restrict__ grad,
                                const double* __restrict__ te, const double* __restrict__ we, double cA_scale,
                                double cB_scale, int termB, double* __restrict__ yrec, double* __restrict__ crec,
                                double* __restrict__ brec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nfac * ke) return;
    const int64_t e = i / ke;
    const int g = (int)(i - e * ke);
    const int a = fac[4 * e], b = fac[4 * e + 1], kp = fac[4 * e + 2], km = fac[4 * e + 3];
    const double* n = fn + e * (d + 1);
    const double L = n[d];
    double J = 0.0;
    for (int c = 0; c < d; ++c) J += n[c] * (grad[(int64_t)kp * d + c] - (km >= 0 ? grad[(int64_t)km * d + c] : 0.0));
    double w, t = 0.0;
    if (d == 1) {
        yrec[i] = V[a];
        w = 1.0;
    } else {
        t = te[g];
        const double ax = V[2 * a], ay = V[2 * a + 1];
        yrec[2 * i] = ax + t * (V[2 * b] - ax);
        yrec[2 * i + 1] = ay + t * (V[2 * b + 1] - ay);
        w = we[g] * L;
    }
    crec[i] = w * J * cA_scale;
    if (termB && e >= nint) {
        const int ia = dov[a], ib = dov[b];
        const double ua = ia >= 0 ? u[ia] : 0.0, ub = ib >= 0 ? u[ib] : 0.0;
        const double uy = d == 1 ? ua : (1.0 - t) * ua + t * ub;
        brec[(e - nint) * ke + g] = w * uy * cB_scale;
    }
}

// One term of the double-word facet sum: acc += c |x-y|^{-PWK/2} (BND: c n.(x-y) |x-y|^{-PWK/2}),
// x = (xh + xl, yh + yl) and the facet point y relative to the same origin.
template <int PWK, bool BND>
__device__ __forceinline__ void sf_term(dw& acc, dw xr, dw yr, float4 y, dw c, float4 nn) {
    // x - y.  TwoSum of the high parts, then the low parts' difference added and the pair
    // renormalised by Fast2Sum: the low parts can make up as much as the high parts' difference
    // when the points are close, and dropping that would cost the square its accuracy.  Fast2Sum
    // is exact here: either the high parts are within a factor 2 (their difference is exact, a
    // nonzero multiple of the smaller one's ulp, which the low parts' difference does not
    // exceed in exponent), or the difference dwarfs the low parts, or it is zero.
    dw dx = two_sum(xr.h, -y.x);
    dx = fast_two_sum(dx.h, __fadd_rn(dx.l, __fsub_rn(xr.l, y.y)));
    dw dy = two_sum(yr.h, -y.z);
    dy = fast_two_sum(dy.h, __fadd_rn(dy.l, __fsub_rn(yr.l, y.w)));
    const dw r2 = dw_add(dw_sqr(dx), dw_sqr(dy));
    dw k = dw_kpow<PWK>(r2);
    if constexpr (BND) {
        const dw nd = dw_add(dw_mul(dw{nn.x, nn.y}, dx), dw_mul(dw{nn.z, nn.w}, dy));
        k = dw_mul(k, nd);
    }
    dw_mac(acc, c, k);
}

// Sum over the facet points of facets [f_begin, f_end) that share no vertex with the point's own
// cell (those are summed in float64 by sf_near_kernel), 2D, double-word.  BND = false: c |x-y|^{-2s} with PWK = 4s; BND = true (boundary facets,
// term with u(y)): c n.(x-y) |x-y|^{-2-2s} with PWK = 4 + 4s.  Each thread takes R points of
// the block's range (stride SF_THREADS); blockIdx.y picks the facet chunk.  KE > 0 fixes the
// Gauss order on the facets at compile time (ke must equal it), 0 takes ke.  A facet that no
// lane of the warp owns (nearly all of them) runs without per-point tests.
template <int PWK, bool BND, int R, int KE>
__global__ void __launch_bounds__(SF_THREADS) sf_far_dw_kernel(
    int64_t npts, int q, const double* __restrict__ X, const int* __restrict__ perm, const int* __restrict__ cells,
    const int* __restrict__ fac, int ke, int64_t f_begin, int64_t f_end, int64_t fac_per_chunk,
    const double* __restrict__ yrec, const double* __restrict__ crec, const double* __restrict__ fn,
    double* __restrict__ part) {
    __shared__ float4 sy[SF_TREC];
    __shared__ float2 sc[SF_TREC];
    __shared__ float4 sn[BND ? SF_TREC : 1];
    __shared__ int2 sab[SF_TREC];  // facet end points
    const int kq = KE > 0 ? KE : ke;
    const int64_t pb = (int64_t)blockIdx.x * SF_THREADS * R;
    // origin of the block: its first point
    const double ox = X[2 * pb], oy = X[2 * pb + 1];
    dw xr[R], yr[R], acc[R];
    int v0[R], v1[R], v2[R];  // the vertices of the point's cell
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t p = pb + r * SF_THREADS + threadIdx.x;
        acc[r] = {0.f, 0.f};
        if (p < npts) {
            xr[r] = dw_from(X[2 * p] - ox);
            yr[r] = dw_from(X[2 * p + 1] - oy);
            const int K = perm[p / q];
            v0[r] = cells[3 * K];
            v1[r] = cells[3 * K + 1];
            v2[r] = cells[3 * K + 2];
        } else {
            xr[r] = {0.f, 0.f};
            yr[r] = {0.f, 0.f};
            v0[r] = v1[r] = v2[r] = -1;
        }
    }
    const int64_t fb = f_begin + (int64_t)blockIdx.y * fac_per_chunk;
    const int64_t fe = min(f_end, fb + fac_per_chunk);
    const int fpt = SF_TREC / kq;
    const float4 nn0 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t f = fb; f < fe; f += fpt) {
        const int nf = (int)min((int64_t)fpt, fe - f);
        __syncthreads();
        for (int i = threadIdx.x; i < nf * kq; i += SF_THREADS) {
            const int64_t gi = f * kq + i;
            const dw yx = dw_from(yrec[2 * gi] - ox), yy = dw_from(yrec[2 * gi + 1] - oy);
            sy[i] = make_float4(yx.h, yx.l, yy.h, yy.l);
            const dw c = dw_from(BND ? crec[gi - f_begin * kq] : crec[gi]);
            sc[i] = make_float2(c.h, c.l);
            if constexpr (BND) {
                const int64_t e = f + i / kq;
                const dw nx = dw_from(fn[3 * e]), ny = dw_from(fn[3 * e + 1]);
                sn[i] = make_float4(nx.h, nx.l, ny.h, ny.l);
            }
        }
        for (int i = threadIdx.x; i < nf; i += SF_THREADS) sab[i] = make_int2(fac[4 * (f + i)], fac[4 * (f + i) + 1]);
        __syncthreads();
        for (int j = 0; j < nf; ++j) {
            const int2 ab = sab[j];
            bool use[R], all = true;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                use[r] = ab.x != v0[r] && ab.x != v1[r] && ab.x != v2[r] && ab.y != v0[r] && ab.y != v1[r] &&
                         ab.y != v2[r];
                all = all && use[r];
            }
            if (__all_sync(0xffffffffu, all)) {
#pragma unroll
                for (int g = 0; g < kq; ++g) {
                    const float4 y = sy[j * kq + g];
                    const float2 c2 = sc[j * kq + g];
                    const float4 nn = BND ? sn[j * kq + g] : nn0;
#pragma unroll
                    for (int r = 0; r < R; ++r) sf_term<PWK, BND>(acc[r], xr[r], yr[r], y, dw{c2.x, c2.y}, nn);
                }
            } else {
                for (int g = 0; g < kq; ++g) {
                    const float4 y = sy[j * kq + g];
                    const float2 c2 = sc[j * kq + g];
                    const float4 nn = BND ? sn[j * kq + g] : nn0;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (use[r]) sf_term<PWK, BND>(acc[r], xr[r], yr[r], y, dw{c2.x, c2.y}, nn);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = dw_renorm(acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t p = pb + r * SF_THREADS + threadIdx.x;
        if (p < npts) part[(int64_t)blockIdx.y * npts + p] = dw_to(acc[r]);
    }
}

// The same sum in float64 for any s and for 1D: c |x-y|^{-m} (log case: c log(1/|x-y|)) on every
// facet that shares no vertex with the point's cell, plus cB n.(x-y) |x-y|^{-d-2s} on boundary
// facets when termB.
__global__ void __launch_bounds__(SF_THREADS) sf_far_f64_kernel(
    int64_t npts, int q, int d, const double* __restrict__ X, const int* __restrict__ perm, const int* __restrict__ cells,
    const int* __restrict__ fac,
    int ke, int64_t nfac, int64_t nint, int64_t fac_per_chunk, const double* __restrict__ yrec,
    const double* __restrict__ crec, const double* __restrict__ brec, const double* __restrict__ fn, int termB, double m,
    double pB, int logc, double* __restrict__ part) {
    const int64_t p = (int64_t)blockIdx.x * SF_THREADS + threadIdx.x;
    if (p >= npts) return;
    const int nfc = d + 1;
    const int K = perm[p / q];
    int vk[3] = {-1, -1, -1};
    for (int j = 0; j < nfc; ++j) vk[j] = cells[(int64_t)K * nfc + j];
    const double x0 = X[p * d], x1 = d == 2 ? X[p * d + 1] : 0.0;
    const int64_t fb = (int64_t)blockIdx.y * fac_per_chunk;
    const int64_t fe = min(nfac, fb + fac_per_chunk);
    double acc = 0.0;
    for (int64_t e = fb; e < fe; ++e) {
        const int a = fac[4 * e], b = fac[4 * e + 1];
        if (a == vk[0] || a == vk[1] || a == vk[2] || b == vk[0] || b == vk[1] || b == vk[2]) continue;
        for (int g = 0; g < ke; ++g) {
            const int64_t i = e * ke + g;
            const double dx = x0 - yrec[i * d], dy = d == 2 ? x1 - yrec[i * d + 1] : 0.0;
            const double r2 = dx * dx + dy * dy;
            acc += crec[i] * (logc ? -0.5 * log(r2) : pow(r2, -0.5 * m));
            if (termB && e >= nint) {
                const double* n = fn + e * (d + 1);
                const double nd = n[0] * dx + (d == 2 ? n[1] * dy : 0.0);
                acc += brec[(e - nint) * ke + g] * nd * pow(r2, -0.5 * pB);
            }
        }
    }
    part[(int64_t)blockIdx.y * npts + p] = acc;
}

// the facets of the point's own cell (float64, order k_near), the other facets that share a
// vertex with it (float64, order k_edge: the close ones, whose difference x - y double-word
// coordinates would resolve only to 2^-48 of the coordinates), and the sum of all parts:
// S[K q + a] = C (near + sum over chunks of part)
__global__ void sf_near_kernel(int64_t npts, int q, int d, const double* __restrict__ X, const double* __restrict__ lam,
                               const int* __restrict__ perm, const int* __restrict__ cells, const double* __restrict__ V,
                               const int* __restrict__ dov, const double* __restrict__ u,
                               const double* __restrict__ grad, const int* __restrict__ c2f,
                               const int* __restrict__ fac, const double* __restrict__ fn, int kn,
                               const double* __restrict__ tn, const double* __restrict__ wn,
                               const int* __restrict__ v2e_ptr, const int* __restrict__ v2e, int ke, int64_t nint,
                               int termB, const double* __restrict__ yrec, const double* __restrict__ crec,
                               const double* __restrict__ brec, double s, double m, double pB, int logc, int nparts,
                               const double* __restrict__ part, double C, double* __restrict__ S) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const int64_t kint = p / q;
    const int a = (int)(p - kint * q);
    const int K0 = perm[kint];
    const int nfc = d + 1;
    const double x0 = X[p * d], x1 = d == 2 ? X[p * d + 1] : 0.0;
    // u(x) from the cell's nodal values
    const int* c = cells + (int64_t)K0 * nfc;
    double ux = 0.0;
    {
        double l[3];
        if (d == 1) {
            l[0] = 1.0 - lam[a];
            l[1] = lam[a];
        } else {
            l[1] = lam[2 * a];
            l[2] = lam[2 * a + 1];
            l[0] = 1.0 - l[1] - l[2];
        }
        for (int j = 0; j < nfc; ++j) {
            const int i = dov[c[j]];
            ux += l[j] * (i >= 0 ? u[i] : 0.0);
        }
    }
    const double g0x = grad[(int64_t)K0 * d], g0y = d == 2 ? grad[(int64_t)K0 * d + 1] : 0.0;
    const double cown = logc ? 1.0 : 1.0 / m;
    const double cnbr = logc ? 1.0 / (2.0 * s) : 1.0 / (2.0 * s * m);
    double near = 0.0;
    for (int j = 0; j < nfc; ++j) {
        const int e = c2f[(int64_t)K0 * nfc + j];
        const int va = fac[4 * e], vb = fac[4 * e + 1], kp = fac[4 * e + 2], km = fac[4 * e + 3];
        const double* n = fn + (int64_t)e * (d + 1);
        const double sg = kp == K0 ? 1.0 : -1.0;
        const int Kn = kp == K0 ? km : kp;
        const double n0x = sg * n[0], n0y = d == 2 ? sg * n[1] : 0.0;
        double cg = cown * (n0x * g0x + n0y * g0y);
        if (Kn >= 0)
            cg -= cnbr * (n0x * grad[(int64_t)Kn * d] + (d == 2 ? n0y * grad[(int64_t)Kn * d + 1] : 0.0));
        const int ng = d == 1 ? 1 : kn;
        for (int g = 0; g < ng; ++g) {
            double yx, yy = 0.0, w;
            if (d == 1) {
                yx = V[va];
                w = 1.0;
            } else {
                const double t = tn[g];
                const double ax = V[2 * va], ay = V[2 * va + 1];
                yx = ax + t * (V[2 * vb] - ax);
                yy = ay + t * (V[2 * vb + 1] - ay);
                w = wn[g] * n[d];
            }
            const double dx = x0 - yx, dy = x1 - yy;
            const double r2 = dx * dx + dy * dy;
            const double k0 = logc ? -0.5 * log(r2) : pow(r2, -0.5 * m);
            const double k1 = pow(r2, -0.5 * pB);
            const double nd = n0x * dx + n0y * dy;
            const double du = Kn >= 0 ? g0x * dx + g0y * dy : ux;
            near += w * (cg * k0 - du * nd * k1 / (2.0 * s));
        }
    }
    // the vertex star: facets through one vertex of K0 that are not its own (in 1D there are none)
    for (int j = 0; j < nfc && d == 2; ++j) {
        for (int qq = v2e_ptr[c[j]]; qq < v2e_ptr[c[j] + 1]; ++qq) {
            const int e = v2e[qq];
            if (e == c2f[(int64_t)K0 * 3] || e == c2f[(int64_t)K0 * 3 + 1] || e == c2f[(int64_t)K0 * 3 + 2]) continue;
            const double* n = fn + (int64_t)e * 3;
            for (int g = 0; g < ke; ++g) {
                const int64_t i = (int64_t)e * ke + g;
                const double dx = x0 - yrec[2 * i], dy = x1 - yrec[2 * i + 1];
                const double r2 = dx * dx + dy * dy;
                near += crec[i] * pow(r2, -0.5 * m);
                if (termB && e >= nint) near += brec[(e - nint) * ke + g] * (n[0] * dx + n[1] * dy) * pow(r2, -0.5 * pB);
            }
        }
    }
    double acc = 0.0;
    for (int r = 0; r < nparts; ++r) acc += part[(int64_t)r * npts + p];
    S[(int64_t)K0 * q + a] = C * (acc + near);
}

// ------------------------------------------------ strong form by the cluster method --
// (Section 6: for a point x0 of cell K0 and sigma the leaf of K0's DOF closest to x0,
// u = u_N + u_F with u_N on the DOFs of sigma's inadmissible partners; the strong form of u_N
// is Lemma 4.1's, that of u_F is -C int k(x0, y) u_F(y) dy = -C sum_alpha L_alpha^sigma(x0)
// yh_sigma[alpha] with the far-field coefficients of the H-matrix product of u.)

constexpr int HSF_FCH = 2048;  // facets per chunk of the far kernel

__device__ __forceinline__ bool hsf_near(const uint32_t* bits, int leaf) {
    return (bits[leaf >> 5] >> (leaf & 31)) & 1u;
}

// nodal value of the near part of u at vertex v (0 off the near DOFs)
__device__ __forceinline__ double hsf_u(int v, const int* dov, const double* u, const int* dof_leaf,
                                        const uint32_t* bits) {
    const int i = dov[v];
    return (i >= 0 && hsf_near(bits, dof_leaf[i])) ? u[i] : 0.0;
}

// gradient of the near part on the (original) cell K, 2D; the expressions of sf_prep_kernel
__device__ void hsf_grad(int K, const int* cells, const double* V, const int* dov, const double* u,
                         const int* dof_leaf, const uint32_t* bits, double& gx, double& gy) {
    const int* c = cells + (int64_t)K * 3;
    const double u0 = hsf_u(c[0], dov, u, dof_leaf, bits), u1 = hsf_u(c[1], dov, u, dof_leaf, bits),
                 u2 = hsf_u(c[2], dov, u, dof_leaf, bits);
    const double p0x = V[2 * c[0]], p0y = V[2 * c[0] + 1];
    const double e1x = V[2 * c[1]] - p0x, e1y = V[2 * c[1] + 1] - p0y;
    const double e2x = V[2 * c[2]] - p0x, e2y = V[2 * c[2] + 1] - p0y;
    const double du1 = u1 - u0, du2 = u2 - u0;
    const double det = e1x * e2y - e1y * e2x;
    gx = (du1 * e2y - du2 * e1y) / det;
    gy = (e1x * du2 - e2x * du1) / det;
}

// per group and facet of its list: the jump of the near part's normal derivative times 1/(2sm)
__global__ void hsf_jump_kernel(const int64_t* __restrict__ gf_ptr, const int* __restrict__ gf_fac,
                                const uint32_t* __restrict__ gbits, int words, const int* __restrict__ fac,
                                const double* __restrict__ fn, const int* __restrict__ cells,
                                const double* __restrict__ V, const int* __restrict__ dov,
                                const double* __restrict__ u, const int* __restrict__ dof_leaf, double cA_scale,
                                double* __restrict__ cj) {
    const int g = blockIdx.y;
    const int64_t idx = gf_ptr[g] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= gf_ptr[g + 1]) return;
    const uint32_t* bits = gbits + (int64_t)g * words;
    const int e = gf_fac[idx];
    const int kp = fac[4 * e + 2], km = fac[4 * e + 3];
    double gx, gy;
    hsf_grad(kp, cells, V, dov, u, dof_leaf, bits, gx, gy);
    double J = fn[3 * e] * gx + fn[3 * e + 1] * gy;
    if (km >= 0) {
        hsf_grad(km, cells, V, dov, u, dof_leaf, bits, gx, gy);
        J -= fn[3 * e] * gx + fn[3 * e + 1] * gy;
    }
    cj[idx] = J * cA_scale;
}

// The far facets of each point's group (those sharing no vertex with the point's cell),
// double-word as in sf_far_dw_kernel: block = (group, 128 of its points, a chunk of its facets).
template <int PWK>
__global__ void __launch_bounds__(SF_THREADS) hsf_far_dw_kernel(
    const int* __restrict__ blk_g, const int* __restrict__ blk_p0, const int* __restrict__ blk_ch,
    const int* __restrict__ gp_ptr, const int* __restrict__ gp_idx, const int64_t* __restrict__ gf_ptr,
    const int* __restrict__ gf_fac, const int64_t* __restrict__ gpo, int q, const double* __restrict__ X,
    const int* __restrict__ perm, const int* __restrict__ cells, const int* __restrict__ fac,
    const double* __restrict__ fn, int ke, const double* __restrict__ yrec, const double* __restrict__ we,
    const double* __restrict__ cj, double* __restrict__ part) {
    __shared__ float4 sy[SF_TREC];
    __shared__ float2 sc[SF_TREC];
    __shared__ int2 sab[SF_TREC];
    const int b = blockIdx.x;
    const int g = blk_g[b], ch = blk_ch[b];
    const int ng = gp_ptr[g + 1] - gp_ptr[g];
    const int i = blk_p0[b] + threadIdx.x;
    const bool valid = i < ng;
    const int p0 = gp_idx[gp_ptr[g] + blk_p0[b]];
    const double ox = X[2 * (int64_t)p0], oy = X[2 * (int64_t)p0 + 1];
    dw xr = {0.f, 0.f}, yr = {0.f, 0.f}, acc = {0.f, 0.f};
    int v0 = -1, v1 = -1, v2 = -1;
    if (valid) {
        const int p = gp_idx[gp_ptr[g] + i];
        xr = dw_from(X[2 * (int64_t)p] - ox);
        yr = dw_from(X[2 * (int64_t)p + 1] - oy);
        const int K = perm[p / q];
        v0 = cells[3 * K];
        v1 = cells[3 * K + 1];
        v2 = cells[3 * K + 2];
    }
    const int64_t fb = gf_ptr[g] + (int64_t)ch * HSF_FCH;
    const int64_t fe = min(gf_ptr[g + 1], fb + HSF_FCH);
    const int fpt = SF_TREC / ke;
    const float4 nn0 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t f = fb; f < fe; f += fpt) {
        const int nf = (int)min((int64_t)fpt, fe - f);
        __syncthreads();
        for (int t = threadIdx.x; t < nf * ke; t += SF_THREADS) {
            const int64_t idx = f + t / ke;
            const int gq = t - (t / ke) * ke;
            const int e = gf_fac[idx];
            const int64_t gi = (int64_t)e * ke + gq;
            const dw yx = dw_from(yrec[2 * gi] - ox), yy = dw_from(yrec[2 * gi + 1] - oy);
            sy[t] = make_float4(yx.h, yx.l, yy.h, yy.l);
            const dw c = dw_from(we[gq] * fn[3 * e + 2] * cj[idx]);
            sc[t] = make_float2(c.h, c.l);
        }
        for (int t = threadIdx.x; t < nf; t += SF_THREADS) {
            const int e = gf_fac[f + t];
            sab[t] = make_int2(fac[4 * e], fac[4 * e + 1]);
        }
        __syncthreads();
        for (int j = 0; j < nf; ++j) {
            const int2 ab = sab[j];
            const bool use = ab.x != v0 && ab.x != v1 && ab.x != v2 && ab.y != v0 && ab.y != v1 && ab.y != v2;
            if (__all_sync(0xffffffffu, use)) {
                for (int gq = 0; gq < ke; ++gq) {
                    const float2 c2 = sc[j * ke + gq];
                    sf_term<PWK, false>(acc, xr, yr, sy[j * ke + gq], dw{c2.x, c2.y}, nn0);
                }
            } else if (use) {
                for (int gq = 0; gq < ke; ++gq) {
                    const float2 c2 = sc[j * ke + gq];
                    sf_term<PWK, false>(acc, xr, yr, sy[j * ke + gq], dw{c2.x, c2.y}, nn0);
                }
            }
            acc = dw_renorm(acc);
        }
    }
    if (valid) part[gpo[g] + (int64_t)ch * ng + i] = dw_to(acc);
}

// r2^{-s} and r2^{-(1+s)} for s = pw0 / 4 (pw0 in {1, 2, 3}) through t = r2^{-1/2}: products of t
// and sqrt(t) in place of two general powers
__device__ __forceinline__ void hsf_pows(double r2, int pw0, double& k0, double& k1) {
    const double t = rsqrt(r2);
    const double t2 = t * t;
    if (pw0 == 2) {
        k0 = t;
        k1 = t2 * t;
    } else {
        const double q = sqrt(t);
        if (pw0 == 1) {
            k0 = q;
            k1 = t2 * q;
        } else {
            k0 = t * q;
            k1 = t2 * t * q;
        }
    }
}

__device__ __forceinline__ double hsf_cheb_node(double c, double L, int m, int k) {
    return c + 0.5 * L * cos((2.0 * (k + 1) - 1.0) * M_PI / (2.0 * m));
}

// per point: the facets of its cell and the other facets through its vertices for the near part
// (float64, as sf_near_kernel with the near part's values), the far-kernel chunks of its group in
// order, and the far field -sum_alpha L_alpha^sigma(x0) yh_sigma[alpha]; S[K0 q + a] = C (...)
__global__ void hsf_near_kernel(int64_t npts, int q, const double* __restrict__ X, const double* __restrict__ lam,
                                const int* __restrict__ perm, const int* __restrict__ cells,
                                const double* __restrict__ V, const int* __restrict__ dov, const double* __restrict__ u,
                                const int* __restrict__ c2f, const int* __restrict__ fac, const double* __restrict__ fn,
                                int kn, const double* __restrict__ tn, const double* __restrict__ wn,
                                const int* __restrict__ v2e_ptr, const int* __restrict__ v2e, int ke,
                                const double* __restrict__ yrec, const double* __restrict__ we,
                                const int* __restrict__ pgroup, const int* __restrict__ plocal,
                                const uint32_t* __restrict__ gbits, int words, const int* __restrict__ dof_leaf,
                                const int* __restrict__ gnode, const int* __restrict__ gp_ptr,
                                const int64_t* __restrict__ gf_ptr, const int* __restrict__ gf_fac,
                                const double* __restrict__ cj,
                                const int* __restrict__ gch, const int64_t* __restrict__ gpo,
                                const double* __restrict__ part, int m, int md, const double* __restrict__ yh,
                                const double* __restrict__ center, const double* __restrict__ side, double s,
                                double mexp, int pw0, double C, double* __restrict__ S) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const int64_t kint = p / q;
    const int a = (int)(p - kint * q);
    const int K0 = perm[kint];
    const int g = pgroup[p];
    const uint32_t* bits = gbits + (int64_t)g * words;
    const double x0 = X[2 * p], x1 = X[2 * p + 1];
    const int* c = cells + (int64_t)K0 * 3;
    double ux;
    {
        const double l1 = lam[2 * a], l2 = lam[2 * a + 1], l0 = 1.0 - l1 - l2;
        ux = l0 * hsf_u(c[0], dov, u, dof_leaf, bits) + l1 * hsf_u(c[1], dov, u, dof_leaf, bits) +
             l2 * hsf_u(c[2], dov, u, dof_leaf, bits);
    }
    double g0x, g0y;
    hsf_grad(K0, cells, V, dov, u, dof_leaf, bits, g0x, g0y);
    const double cown = 1.0 / mexp, cnbr = 1.0 / (2.0 * s * mexp);
    double near = 0.0;
    for (int j = 0; j < 3; ++j) {
        const int e = c2f[(int64_t)K0 * 3 + j];
        const int va = fac[4 * e], vb = fac[4 * e + 1], kp = fac[4 * e + 2], km = fac[4 * e + 3];
        const double* n = fn + (int64_t)e * 3;
        const double sg = kp == K0 ? 1.0 : -1.0;
        const int Kn = kp == K0 ? km : kp;
        const double n0x = sg * n[0], n0y = sg * n[1];
        double cg = cown * (n0x * g0x + n0y * g0y);
        if (Kn >= 0) {
            double gx, gy;
            hsf_grad(Kn, cells, V, dov, u, dof_leaf, bits, gx, gy);
            cg -= cnbr * (n0x * gx + n0y * gy);
        }
        for (int gq = 0; gq < kn; ++gq) {
            const double t = tn[gq];
            const double ax = V[2 * va], ay = V[2 * va + 1];
            const double yx = ax + t * (V[2 * vb] - ax), yy = ay + t * (V[2 * vb + 1] - ay);
            const double w = wn[gq] * n[2];
            const double dx = x0 - yx, dy = x1 - yy;
            const double r2 = dx * dx + dy * dy;
            double k0, k1;
            hsf_pows(r2, pw0, k0, k1);
            const double nd = n0x * dx + n0y * dy;
            const double du = Kn >= 0 ? g0x * dx + g0y * dy : ux;
            near += w * (cg * k0 - du * nd * k1 / (2.0 * s));
        }
    }
    // the other facets through K0's vertices: their jumps from the group's list (ascending facet ids;
    // a facet absent from it touches no near DOF, its jump is zero)
    const int64_t fl0 = gf_ptr[g], fl1 = gf_ptr[g + 1];
    for (int j = 0; j < 3; ++j) {
        for (int qq = v2e_ptr[c[j]]; qq < v2e_ptr[c[j] + 1]; ++qq) {
            const int e = v2e[qq];
            if (e == c2f[(int64_t)K0 * 3] || e == c2f[(int64_t)K0 * 3 + 1] || e == c2f[(int64_t)K0 * 3 + 2]) continue;
            int64_t lo = fl0, hi = fl1;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (gf_fac[mid] < e) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= fl1 || gf_fac[lo] != e) continue;
            const double cjv = cj[lo];
            for (int gq = 0; gq < ke; ++gq) {
                const int64_t i = (int64_t)e * ke + gq;
                const double dx = x0 - yrec[2 * i], dy = x1 - yrec[2 * i + 1];
                double k0, k1;
                hsf_pows(dx * dx + dy * dy, pw0, k0, k1);
                near += we[gq] * fn[3 * e + 2] * cjv * k0;
            }
        }
    }
    double acc = 0.0;
    const int ng = gp_ptr[g + 1] - gp_ptr[g];
    const int il = plocal[p];
    for (int ch = 0; ch < gch[g]; ++ch) acc += part[gpo[g] + (int64_t)ch * ng + il];
    double farf = 0.0;
    const int cn = gnode[g];
    if (cn >= 0) {
        double lx[12], ly[12], nx[12], ny[12];
        const double cx = center[2 * (int64_t)cn], cy = center[2 * (int64_t)cn + 1], L = side[cn];
        for (int k = 0; k < m; ++k) {  // the nodes once (the same values as node by node)
            nx[k] = hsf_cheb_node(cx, L, m, k);
            ny[k] = hsf_cheb_node(cy, L, m, k);
        }
        for (int k = 0; k < m; ++k) {
            double vx = 1.0, vy = 1.0;
            for (int l = 0; l < m; ++l)
                if (l != k) {
                    vx *= (x0 - nx[l]) / (nx[k] - nx[l]);
                    vy *= (x1 - ny[l]) / (ny[k] - ny[l]);
                }
            lx[k] = vx;
            ly[k] = vy;
        }
        const double* y = yh + (int64_t)cn * md;
        for (int k0 = 0; k0 < m; ++k0) {
            double r = 0.0;
            for (int k1 = 0; k1 < m; ++k1) r += ly[k1] * y[k0 * m + k1];
            farf += lx[k0] * r;
        }
    }
    S[(int64_t)K0 * q + a] = C * (acc + near - farf);
}

// per cell: h_K^{2s} sum_a W_a (f(x_a) - S_a)^2
__global__ void br_cell_kernel(int64_t nc, int d, int q, const int* __restrict__ cells, const double* __restrict__ V,
                               const double* __restrict__ jac, const double* __restrict__ lam,
                               const double* __restrict__ w, const double* __restrict__ f, const double* __restrict__ S,
                               double two_s, double* __restrict__ err) {
    const int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= nc) return;
    const int* c = cells + K * (d + 1);
    double h;
    if (d == 1) {
        h = V[c[1]] - V[c[0]];
    } else {
        h = 0.0;
        for (int j = 0; j < 3; ++j) {
            const int a = c[j], b = c[(j + 1) % 3];
            h = fmax(h, hypot(V[2 * b] - V[2 * a], V[2 * b + 1] - V[2 * a + 1]));
        }
    }
    double sum = 0.0;
    for (int a = 0; a < q; ++a) {
        double fx = 1.0;
        if (f) {
            if (d == 1) {
                fx = (1.0 - lam[a]) * f[c[0]] + lam[a] * f[c[1]];
            } else {
                const double l1 = lam[2 * a], l2 = lam[2 * a + 1];
                fx = (1.0 - l1 - l2) * f[c[0]] + l1 * f[c[1]] + l2 * f[c[2]];
            }
        }
        const double r = fx - S[K * q + a];
        sum += w[a] * jac[K] * r * r;
    }
    err[K] = pow(h, two_s) * sum;
}

// per DOF: eta_i = sqrt(sum over the cells around its vertex)
__global__ void br_dof_kernel(int64_t n, const int* __restrict__ vod, const int64_t* __restrict__ v2c_ptr,
                              const int* __restrict__ v2c, const double* __restrict__ err, double* __restrict__ eta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = vod[i];
    double acc = 0.0;
    for (int64_t k = v2c_ptr[v]; k < v2c_ptr[v + 1]; ++k) acc += err[v2c[k]];
    eta[i] = sqrt(acc);
}

// one block: *thr = theta max_i eta_i
__global__ void mark_max_kernel(int64_t n, const double* __restrict__ eta, double theta, double* __restrict__ thr) {
    __shared__ double red[32];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, eta[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) *thr = theta * mx;
    }
}

__global__ void mark_dof_kernel(int64_t n, const double* __restrict__ eta, const double* __restrict__ thr,
                                uint8_t* __restrict__ marks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) marks[i] = eta[i] >= *thr ? 1 : 0;
}

__global__ void mark_cell_kernel(int64_t nc, int nvpc, const int* __restrict__ cells, const int* __restrict__ dov,
                                 const double* __restrict__ eta, const double* __restrict__ thr,
                                 uint8_t* __restrict__ marks) {
    const int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= nc) return;
    uint8_t m = 0;
    for (int j = 0; j < nvpc; ++j) {
        const int i = dov[cells[K * nvpc + j]];
        if (i >= 0 && eta[i] >= *thr) m = 1;
    }
    marks[K] = m;
}

// ------------------------------------------------------------------ host --

int dev_alloc(fl_ctx* h, void** dst, size_t bytes) {
    *dst = nullptr;
    cudaError_t e = pool_dev_alloc(dst, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("adaptive tables: ") + cudaGetErrorString(e));
    h->bufs.push_back({*dst, bytes});
    h->ws_bytes += (int64_t)bytes;
    return FL_OK;
}

template <typename X>
int upload(fl_ctx* h, X** dst, const std::vector<X>& src, cudaStream_t st) {
    SF_TRY(dev_alloc(h, (void**)dst, src.size() * sizeof(X)));
    if (!src.empty()) {
        SF_CUDA(h, cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice, st));
        SF_CUDA(h, cudaStreamSynchronize(st));
    }
    h->h2d_bytes += (int64_t)(src.size() * sizeof(X));
    return FL_OK;
}

// Facets of the mesh for the strong form: interior facets first (the lower cell id is K+),
// then boundary facets; cell -> facets in the cell's own order (2D edges v0v1, v1v2, v2v0;
// 1D left, right end).
struct SfFac {
    int a, b, kp, km;
    double n[2], len;
};

// host part: the facet list and cell -> facets (FL_EINVAL for a non-conforming mesh)
int sf_build_facets(const Plan& P, std::vector<SfFac>& F, std::vector<int>& c2f_local, std::string& err) {
    const int d = P.dim, nvpc = P.nvpc;
    const int64_t nc = P.nc;
    using Fac = SfFac;
    F.clear();
    c2f_local.assign(nc * nvpc, -1);
    if (d == 1) {
        // facet per vertex; K+ = the cell whose right end it is (normal +1)
        std::vector<int> right(P.nv, -1), left(P.nv, -1);
        for (int64_t K = 0; K < nc; ++K) {
            left[P.C[K * 2]] = (int)K;
            right[P.C[K * 2 + 1]] = (int)K;
        }
        std::vector<int> fid(P.nv, -1);
        for (int pass = 0; pass < 2; ++pass)
            for (int64_t v = 0; v < P.nv; ++v) {
                const bool interior = left[v] >= 0 && right[v] >= 0;
                if (interior != (pass == 0) || (left[v] < 0 && right[v] < 0)) continue;
                Fac f{};
                f.a = f.b = (int)v;
                if (right[v] >= 0) {
                    f.kp = right[v];
                    f.km = left[v];
                    f.n[0] = 1.0;
                } else {
                    f.kp = left[v];
                    f.km = -1;
                    f.n[0] = -1.0;
                }
                f.len = 1.0;
                fid[v] = (int)F.size();
                F.push_back(f);
            }
        for (int64_t K = 0; K < nc; ++K) {
            c2f_local[K * 2] = fid[P.C[K * 2]];
            c2f_local[K * 2 + 1] = fid[P.C[K * 2 + 1]];
        }
    } else {
        // (edge key, cell, local edge) sorted: the cells of an edge are adjacent, lower cell first
        struct Ent {
            uint64_t key;
            int K, j;
        };
        std::vector<Ent> ent((size_t)nc * 3);
        for (int64_t K = 0; K < nc; ++K)
            for (int j = 0; j < 3; ++j) {
                const int a = P.C[K * 3 + j], b = P.C[K * 3 + (j + 1) % 3];
                ent[(size_t)K * 3 + j] = {((uint64_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b), (int)K, j};
            }
        std::sort(ent.begin(), ent.end(), [](const Ent& x, const Ent& y) {
            return x.key < y.key || (x.key == y.key && (x.K < y.K || (x.K == y.K && x.j < y.j)));
        });
        // per edge: its first entry and its size; numbering: interior facets by (K+, local edge),
        // then boundary facets the same way
        std::vector<std::pair<std::pair<int, int>, size_t>> lst[2];
        for (size_t i = 0; i < ent.size();) {
            size_t e = i + 1;
            while (e < ent.size() && ent[e].key == ent[i].key) ++e;
            if (e - i > 2) {
                err = "non-conforming mesh: an edge in more than two cells";
                return FL_EINVAL;
            }
            lst[e - i == 2 ? 0 : 1].push_back({{ent[i].K, ent[i].j}, i});
            i = e;
        }
        for (int pass = 0; pass < 2; ++pass) {
            std::sort(lst[pass].begin(), lst[pass].end());
            for (const auto& it : lst[pass]) {
                const size_t i0 = it.second;
                const bool two = pass == 0;
                const int K = ent[i0].K, j = ent[i0].j;
                Fac f{};
                f.a = P.C[(int64_t)K * 3 + j];
                f.b = P.C[(int64_t)K * 3 + (j + 1) % 3];
                f.kp = K;
                f.km = two ? ent[i0 + 1].K : -1;
                const double ex = P.V[2 * f.b] - P.V[2 * f.a], ey = P.V[2 * f.b + 1] - P.V[2 * f.a + 1];
                f.len = std::hypot(ex, ey);
                // counter-clockwise cells: the outward normal is the edge vector turned clockwise
                f.n[0] = ey / f.len;
                f.n[1] = -ex / f.len;
                const int id = (int)F.size();
                F.push_back(f);
                c2f_local[(int64_t)K * 3 + j] = id;
                if (two) c2f_local[(int64_t)ent[i0 + 1].K * 3 + ent[i0 + 1].j] = id;
            }
        }
    }
    return FL_OK;
}

int ensure_sf_topology(fl_ctx* h, int pi, cudaStream_t st) {
    DevTables& t = h->dev[pi];
    if (t.sf_ready) return FL_OK;
    const Plan& P = h->plan[pi];
    const int d = P.dim;
    std::vector<SfFac> F;
    std::vector<int> c2f_local;
    {
        std::string err;
        const int rc = sf_build_facets(P, F, c2f_local, err);
        if (rc != FL_OK) return set_err(h, rc, err);
    }
    int64_t nint = 0;
    for (const auto& f : F) nint += f.km >= 0;
    std::vector<int> fac(F.size() * 4);
    std::vector<double> fn(F.size() * (d + 1));
    for (size_t e = 0; e < F.size(); ++e) {
        fac[4 * e] = F[e].a;
        fac[4 * e + 1] = F[e].b;
        fac[4 * e + 2] = F[e].kp;
        fac[4 * e + 3] = F[e].km;
        for (int c = 0; c < d; ++c) fn[e * (d + 1) + c] = F[e].n[c];
        fn[e * (d + 1) + d] = F[e].len;
    }
    SF_CUDA(h, cudaSetDevice(h->device));
    SF_TRY(upload(h, &t.sf_fac, fac, st));
    SF_TRY(upload(h, &t.sf_fn, fn, st));
    SF_TRY(upload(h, &t.sf_c2f, c2f_local, st));
    t.sf_c2f_host = c2f_local;
    // vertex -> facets through it (2D)
    std::vector<int> v2e_ptr(P.nv + 1, 0), v2e;
    if (d == 2) {
        for (const auto& f : F) ++v2e_ptr[f.a + 1], ++v2e_ptr[f.b + 1];
        for (int64_t v = 0; v < P.nv; ++v) v2e_ptr[v + 1] += v2e_ptr[v];
        v2e.resize(v2e_ptr[P.nv]);
        std::vector<int> fill(v2e_ptr.begin(), v2e_ptr.end() - 1);
        for (size_t e = 0; e < F.size(); ++e) {
            v2e[fill[F[e].a]++] = (int)e;
            v2e[fill[F[e].b]++] = (int)e;
        }
    }
    SF_TRY(upload(h, &t.sf_v2e_ptr, v2e_ptr, st));
    SF_TRY(upload(h, &t.sf_v2e, v2e, st));
    SF_TRY(upload(h, &t.sf_perm, P.perm, st));
    t.sf_nfac = (int64_t)F.size();
    t.sf_nint = nint;
    t.sf_ready = true;
    return FL_OK;
}

// rule tables: cell rule (lam q*d, w q), edge rule (t, w: k_edge), near rule (t, w: k_near)
int ensure_sf_rules(fl_ctx* h, int pi, int kc, int ke, int kn, cudaStream_t st) {
    DevTables& t = h->dev[pi];
    if (t.sf_rule && t.sf_rule_key[0] == kc && t.sf_rule_key[1] == ke && t.sf_rule_key[2] == kn) return FL_OK;
    const Plan& P = h->plan[pi];
    const Rule R = make_rule(P.dim, kc);
    std::vector<double> tab(R.lam);
    tab.insert(tab.end(), R.w.begin(), R.w.end());
    std::vector<double> x, w;
    gauss01(ke, x, w);
    tab.insert(tab.end(), x.begin(), x.end());
    tab.insert(tab.end(), w.begin(), w.end());
    gauss01(kn, x, w);
    tab.insert(tab.end(), x.begin(), x.end());
    tab.insert(tab.end(), w.begin(), w.end());
    if (tab.size() > t.sf_rule_cap) {
        SF_TRY(dev_alloc(h, (void**)&t.sf_rule, tab.size() * sizeof(double)));
        t.sf_rule_cap = tab.size();
    }
    SF_CUDA(h, cudaMemcpyAsync(t.sf_rule, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    SF_CUDA(h, cudaStreamSynchronize(st));
    t.sf_rule_key[0] = kc;
    t.sf_rule_key[1] = ke;
    t.sf_rule_key[2] = kn;
    return FL_OK;
}

int ensure_ws(fl_ctx* h, size_t bytes) {
    if (bytes <= h->sf_ws_bytes) return FL_OK;
    if (h->sf_ws) {
        SF_CUDA(h, cudaDeviceSynchronize());
        pool_dev_free(h->sf_ws);
        h->sf_ws = nullptr;
        h->sf_ws_bytes = 0;
    }
    cudaError_t e = pool_dev_alloc(&h->sf_ws, bytes);
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("adaptive workspace: ") + cudaGetErrorString(e));
    h->sf_ws_bytes = bytes;
    return FL_OK;
}

// s in {1/4, 1/2, 3/4} as 4s, else 0
int quarter(double s) {
    for (int k = 1; k <= 3; ++k)
        if (s == k / 4.0) return k;
    return 0;
}

template <int PW0, int R>
void launch_far_dw_r(dim3 grid, int64_t npts, int q, const double* X, const int* perm, const int* cells,
                     const int* fac, int ke, int64_t fb, int64_t fe, int64_t fpc, const double* yrec,
                     const double* crec, const double* fn, double* part, cudaStream_t st) {
    if (ke == 4)
        sf_far_dw_kernel<PW0, false, R, 4><<<grid, SF_THREADS, 0, st>>>(npts, q, X, perm, cells, fac, ke, fb, fe, fpc,
                                                                         yrec, crec, fn, part);
    else
        sf_far_dw_kernel<PW0, false, R, 0><<<grid, SF_THREADS, 0, st>>>(npts, q, X, perm, cells, fac, ke, fb, fe, fpc,
                                                                         yrec, crec, fn, part);
}

template <int PW0>
void launch_far_dw(int R, dim3 grid, int64_t npts, int q, const double* X, const int* perm, const int* cells,
                   const int* fac, int ke, int64_t fb, int64_t fe, int64_t fpc, const double* yrec,
                   const double* crec, const double* fn, double* part, cudaStream_t st) {
    if (R == 2)
        launch_far_dw_r<PW0, 2>(grid, npts, q, X, perm, cells, fac, ke, fb, fe, fpc, yrec, crec, fn, part, st);
    else
        launch_far_dw_r<PW0, 1>(grid, npts, q, X, perm, cells, fac, ke, fb, fe, fpc, yrec, crec, fn, part, st);
}

template <int PW>
void launch_bnd_dw(dim3 grid, int64_t npts, int q, const double* X, const int* perm, const int* cells,
                   const int* fac, int ke, int64_t fb, int64_t fe, int64_t fpc, const double* yrec,
                   const double* brec, const double* fn, double* part, cudaStream_t st) {
    sf_far_dw_kernel<PW, true, 1, 0><<<grid, SF_THREADS, 0, st>>>(npts, q, X, perm, cells, fac, ke, fb, fe, fpc, yrec,
                                                                   brec, fn, part);
}

}  // namespace

int strong_form(fl_ctx* h, double s, const double* u, int kc, int ke, int kn, double* S, cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!u || !S) return set_err(h, FL_EINVAL, "NULL u or S");
    if (kc < 1 || kc > SF_MAXK_CELL || ke < 1 || ke > SF_MAXK_EDGE || kn < 1 || kn > SF_MAXK_NEAR)
        return set_err(h, FL_EINVAL, "k_cell in [1,16], k_edge in [1,32], k_near in [1,64]");
    SF_CUDA(h, cudaSetDevice(h->device));
    SF_TRY(ensure_device_tables(h, pi, st));
    SF_TRY(ensure_sf_topology(h, pi, st));
    SF_TRY(ensure_sf_rules(h, pi, kc, ke, kn, st));
    DevTables& t = h->dev[pi];
    const int d = P.dim;
    const int64_t nc = P.nc, nfac = t.sf_nfac, nint = t.sf_nint, nb = nfac - nint;
    const int q = d == 1 ? kc : kc * kc;
    const int64_t npts = nc * q;
    const int ke_eff = d == 1 ? 1 : ke;
    const double m = d + 2.0 * s - 2.0, pB = d + 2.0 * s;
    const int logc = std::fabs(m) < 1e-14;
    const double cA_scale = logc ? 1.0 / (2.0 * s) : 1.0 / (2.0 * s * m);
    const double cB_scale = -1.0 / (2.0 * s);
    // boundary values of u_h are zero unless boundary vertices are degrees of freedom
    bool termB = false;
    for (int64_t v = 0; v < P.nv && !termB; ++v) termB = P.onb[v] && P.dov[v] >= 0;
    const int pw0 = d == 2 ? quarter(s) : 0;
    const bool use_dw = pw0 > 0 && !h->far_f64_pipe;
    // chunks of facets so that the grid fills the device
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    // two points per thread once the grid fills the device (four measured slower: 80 registers)
    const int R = use_dw && npts >= (int64_t)sms * SF_THREADS * 8 ? 2 : 1;
    const int64_t bx = (npts + (int64_t)SF_THREADS * R - 1) / ((int64_t)SF_THREADS * R);
    const int64_t want = (int64_t)sms * 8;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(64, (want + bx - 1) / bx));
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, nfac / 16));
    const int64_t fpc = (nfac + chunks - 1) / chunks;
    int64_t bchunks = 0, bfpc = 1;
    if (use_dw && termB && nb > 0) {
        bchunks = std::max<int64_t>(1, std::min<int64_t>(16, std::min<int64_t>((want + bx - 1) / bx, nb)));
        bfpc = (nb + bchunks - 1) / bchunks;
    }
    const int64_t nparts = chunks + bchunks;
    // workspace: grad, X, yrec, crec, brec, part
    const size_t n_grad = nc * d, n_X = npts * d, n_y = nfac * ke_eff * d, n_c = nfac * ke_eff,
                 n_b = std::max<int64_t>(nb, 1) * ke_eff, n_part = nparts * npts;
    const size_t total = (n_grad + n_X + n_y + n_c + n_b + n_part + 8 * 6) * sizeof(double);
    SF_TRY(ensure_ws(h, total));
    double* base = (double*)h->sf_ws;
    auto take = [&](size_t n) {
        double* p = base;
        base += (n + 7) / 8 * 8;
        return p;
    };
    double* grad = take(n_grad);
    double* X = take(n_X);
    double* yrec = take(n_y);
    double* crec = take(n_c);
    double* brec = take(n_b);
    double* part = take(n_part);
    const double* lam = t.sf_rule;
    const Rule Rc = make_rule(d, kc);  // sizes only
    const double* wc = t.sf_rule + Rc.lam.size();
    const double* te = wc + Rc.w.size();
    const double* we = te + ke;
    const double* tn = we + ke;
    const double* wn = tn + kn;
    (void)wc;
    if (nc > 0) {
        sf_prep_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(nc, d, q, t.sf_perm, t.cells, t.V, t.dov, u, lam,
                                                                     grad, X);
        count_launch();
        const int64_t nrec = nfac * ke_eff;
        sf_facet_kernel<<<(unsigned)((nrec + 127) / 128), 128, 0, st>>>(nfac, nint, d, ke_eff, t.sf_fac, t.sf_fn, t.V,
                                                                        t.dov, u, grad, te, we, cA_scale, cB_scale,
                                                                        termB ? 1 : 0, yrec, crec, brec);
        count_launch();
        if (use_dw) {
            const dim3 grid((unsigned)bx, (unsigned)chunks);
            switch (pw0) {
                case 1: launch_far_dw<1>(R, grid, npts, q, X, t.sf_perm, t.cells, t.sf_fac, ke, 0, nfac, fpc, yrec, crec, t.sf_fn, part, st); break;
                case 2: launch_far_dw<2>(R, grid, npts, q, X, t.sf_perm, t.cells, t.sf_fac, ke, 0, nfac, fpc, yrec, crec, t.sf_fn, part, st); break;
                default: launch_far_dw<3>(R, grid, npts, q, X, t.sf_perm, t.cells, t.sf_fac, ke, 0, nfac, fpc, yrec, crec, t.sf_fn, part, st); break;
            }
            count_launch();
            if (bchunks > 0) {
                const int64_t bx1 = (npts + SF_THREADS - 1) / SF_THREADS;
                const dim3 g2((unsigned)bx1, (unsigned)bchunks);
                double* bpart = part + chunks * npts;
                switch (pw0) {
                    case 1: launch_bnd_dw<5>(g2, npts, q, X, t.sf_perm, t.cells, t.sf_fac, ke, nint, nfac, bfpc, yrec, brec, t.sf_fn, bpart, st); break;
                    case 2: launch_bnd_dw<6>(g2, npts, q, X, t.sf_perm, t.cells, t.sf_fac, ke, nint, nfac, bfpc, yrec, brec, t.sf_fn, bpart, st); break;
                    default: launch_bnd_dw<7>(g2, npts, q, X, t.sf_perm, t.cells, t.sf_fac, ke, nint, nfac, bfpc, yrec, brec, t.sf_fn, bpart, st); break;
                }
                count_launch();
            }
        } else {
            const dim3 grid((unsigned)((npts + SF_THREADS - 1) / SF_THREADS), (unsigned)chunks);
            sf_far_f64_kernel<<<grid, SF_THREADS, 0, st>>>(npts, q, d, X, t.sf_perm, t.cells, t.sf_fac, ke_eff, nfac, nint, fpc,
                                                           yrec, crec, brec, t.sf_fn, termB ? 1 : 0, m, pB, logc, part);
            count_launch();
        }
        sf_near_kernel<<<(unsigned)((npts + 127) / 128), 128, 0, st>>>(
            npts, q, d, X, lam, t.sf_perm, t.cells, t.V, t.dov, u, grad, t.sf_c2f, t.sf_fac, t.sf_fn, kn, tn, wn,
            t.sf_v2e_ptr, t.sf_v2e, ke_eff, nint, termB ? 1 : 0, yrec, crec, brec, s, m, pB, logc, (int)nparts, part,
            frac_const(d, s), S);
        count_launch();
    }
    SF_CUDA(h, cudaGetLastError());
    return FL_OK;
}

int sf_facets_host(const Plan& P, std::vector<int>& c2f, std::vector<int>& fac_vert, int64_t* nfac) {
    std::vector<SfFac> F;
    std::string err;
    const int rc = sf_build_facets(P, F, c2f, err);
    if (rc != FL_OK) return rc;
    fac_vert.resize(F.size() * 2);
    for (size_t e = 0; e < F.size(); ++e) {
        fac_vert[2 * e] = F[e].a;
        fac_vert[2 * e + 1] = F[e].b;
    }
    *nfac = (int64_t)F.size();
    return FL_OK;
}

int sf_topology(fl_ctx* h, int pi, cudaStream_t st, const std::vector<int>** c2f, int64_t* nfac) {
    SF_CUDA(h, cudaSetDevice(h->device));
    SF_TRY(ensure_device_tables(h, pi, st));
    SF_TRY(ensure_sf_topology(h, pi, st));
    *c2f = &h->dev[pi].sf_c2f_host;
    *nfac = h->dev[pi].sf_nfac;
    return FL_OK;
}

int plan_hsf(const Plan& P, const ClusterPlan& C, const std::vector<int>& c2f, int64_t nfac, int kc, HsfPlan& Q,
             std::string& err) {
    Q = HsfPlan();
    if (P.dim != 2) {
        err = "the cluster strong form is 2D";
        return FL_ENOTIMPL;
    }
    const int64_t nc = P.nc, n = P.n;
    const Rule R = make_rule(2, kc);
    const int q = R.q;
    Q.kc = kc;
    Q.npts = nc * q;
    // leaves in node order; the leaf of every DOF
    std::vector<int> lidx(C.nodes, -1), leaves;
    for (int a = 0; a < C.nodes; ++a)
        if (C.son[2 * a] < 0) {
            lidx[a] = (int)leaves.size();
            leaves.push_back(a);
        }
    const int nl = (int)leaves.size();
    Q.words = (nl + 31) / 32;
    Q.dof_leaf.assign(n, -1);
    std::vector<int> dof_node(n, -1);
    for (int a : leaves)
        for (int p = C.lo[a]; p < C.hi[a]; ++p) {
            Q.dof_leaf[C.perm[p]] = lidx[a];
            dof_node[C.perm[p]] = a;
        }
    // each point's group: the leaf of its cell's DOF closest to it (ties: lower DOF), or the group
    // of cells without DOFs
    std::vector<int> gof_node(C.nodes, -1);
    std::vector<int> pnode(Q.npts, -1);
    bool any_free = false;
    for (int64_t k = 0; k < nc; ++k) {
        const int K = P.perm[k];
        const int* c = &P.C[(int64_t)K * 3];
        const double p0x = P.V[2 * c[0]], p0y = P.V[2 * c[0] + 1];
        const double e1x = P.V[2 * c[1]] - p0x, e1y = P.V[2 * c[1] + 1] - p0y;
        const double e2x = P.V[2 * c[2]] - p0x, e2y = P.V[2 * c[2] + 1] - p0y;
        for (int a = 0; a < q; ++a) {
            const double l1 = R.lam[2 * a], l2 = R.lam[2 * a + 1];
            const double x = p0x + l1 * e1x + l2 * e2x, y = p0y + l1 * e1y + l2 * e2y;
            int best = -1;
            double bd = 0.0;
            for (int j = 0; j < 3; ++j) {
                const int i = P.dov[c[j]];
                if (i < 0) continue;
                const double dx = P.V[2 * c[j]] - x, dy = P.V[2 * c[j] + 1] - y;
                const double dd = dx * dx + dy * dy;
                if (best < 0 || dd < bd || (dd == bd && i < best)) {
                    best = i;
                    bd = dd;
                }
            }
            pnode[k * q + a] = best >= 0 ? dof_node[best] : -1;
            any_free = any_free || best < 0;
        }
    }
    for (int64_t p = 0; p < Q.npts; ++p)
        if (pnode[p] >= 0) gof_node[pnode[p]] = 1;
    for (int a : leaves)
        if (gof_node[a] > 0) {
            gof_node[a] = Q.groups++;
            Q.gnode.push_back(a);
        }
    const int free_group = any_free ? Q.groups++ : -1;
    if (any_free) Q.gnode.push_back(-1);
    if (Q.groups > 65535) {
        err = "more than 65535 point groups";
        return FL_ENOTIMPL;
    }
    const int G = Q.groups;
    Q.pgroup.resize(Q.npts);
    Q.plocal.resize(Q.npts);
    Q.gp_ptr.assign(G + 1, 0);
    for (int64_t p = 0; p < Q.npts; ++p) {
        Q.pgroup[p] = pnode[p] >= 0 ? gof_node[pnode[p]] : free_group;
        ++Q.gp_ptr[Q.pgroup[p] + 1];
    }
    for (int g = 0; g < G; ++g) Q.gp_ptr[g + 1] += Q.gp_ptr[g];
    Q.gp_idx.resize(Q.npts);
    {
        std::vector<int> fill(Q.gp_ptr.begin(), Q.gp_ptr.end() - 1);
        for (int64_t p = 0; p < Q.npts; ++p) {
            const int g = Q.pgroup[p];
            Q.plocal[p] = fill[g] - Q.gp_ptr[g];
            Q.gp_idx[fill[g]++] = (int)p;
        }
    }
    // per group: near leaves and the facets of the cells touching a near DOF
    std::vector<std::vector<int>> partners(C.nodes);
    for (size_t b = 0; b + 1 < C.near.size(); b += 2) partners[C.near[b]].push_back(C.near[b + 1]);
    Q.gbits.assign((size_t)G * Q.words, 0u);
    Q.gf_ptr.assign(G + 1, 0);
    // in parallel over ranges of groups, the lists concatenated in group order
    const int nthr = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    const int gchunk = (G + nthr - 1) / nthr;
    std::vector<std::vector<int>> lists(nthr);
    std::vector<std::vector<int64_t>> lens(nthr);
    auto work = [&](int th) {
        const int g0 = th * gchunk, g1 = std::min(G, g0 + gchunk);
        if (g0 >= g1) return;
        std::vector<int> cmark(nc, -1), fmark(nfac, -1), fl;
        for (int g = g0; g < g1; ++g) {
            uint32_t* bits = &Q.gbits[(size_t)g * Q.words];
            fl.clear();
            if (Q.gnode[g] < 0) {
                for (int l = 0; l < nl; ++l) bits[l >> 5] |= 1u << (l & 31);
                for (int64_t e = 0; e < nfac; ++e) fl.push_back((int)e);
            } else {
                for (int tau : partners[Q.gnode[g]]) {
                    const int l = lidx[tau];
                    bits[l >> 5] |= 1u << (l & 31);
                    for (int pp = C.lo[tau]; pp < C.hi[tau]; ++pp) {
                        const int v = P.vod[C.perm[pp]];
                        for (int r = P.v2c_ptr[v]; r < P.v2c_ptr[v + 1]; ++r) {
                            const int K = P.v2c[r];
                            if (cmark[K] == g) continue;
                            cmark[K] = g;
                            for (int j = 0; j < 3; ++j) {
                                const int e = c2f[(int64_t)K * 3 + j];
                                if (fmark[e] == g) continue;
                                fmark[e] = g;
                                fl.push_back(e);
                            }
                        }
                    }
                }
                std::sort(fl.begin(), fl.end());
            }
            lists[th].insert(lists[th].end(), fl.begin(), fl.end());
            lens[th].push_back((int64_t)fl.size());
        }
    };
    {
        std::vector<std::thread> th;
        for (int t = 1; t < nthr; ++t) th.emplace_back(work, t);
        work(0);
        for (auto& x : th) x.join();
    }
    {
        int g = 0;
        for (int t = 0; t < nthr; ++t) {
            Q.gf_fac.insert(Q.gf_fac.end(), lists[t].begin(), lists[t].end());
            for (int64_t L : lens[t]) {
                Q.gf_ptr[g + 1] = Q.gf_ptr[g] + L;
                Q.maxf = std::max<int64_t>(Q.maxf, L);
                ++g;
            }
        }
    }
    // far-kernel blocks: (group, 128 points, facet chunk); partial sums per group: points x chunks
    Q.gch.resize(G);
    Q.gpo.resize(G);
    int64_t off = 0;
    for (int g = 0; g < G; ++g) {
        const int64_t nf = Q.gf_ptr[g + 1] - Q.gf_ptr[g];
        const int ng = Q.gp_ptr[g + 1] - Q.gp_ptr[g];
        Q.gch[g] = (int)std::max<int64_t>(1, (nf + HSF_FCH - 1) / HSF_FCH);
        Q.gpo[g] = off;
        off += (int64_t)ng * Q.gch[g];
        for (int p0 = 0; p0 < ng; p0 += SF_THREADS)
            for (int ch = 0; ch < Q.gch[g]; ++ch) {
                Q.blk_g.push_back(g);
                Q.blk_p0.push_back(p0);
                Q.blk_ch.push_back(ch);
            }
    }
    Q.nparts = off;
    return FL_OK;
}

int strong_form_cluster(fl_ctx* h, double s, const double* u, int kc, int ke, int kn, const HsfDev& g, double* S,
                        cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!u || !S) return set_err(h, FL_EINVAL, "NULL u or S");
    if (P.dim != 2) return set_err(h, FL_ENOTIMPL, "the cluster strong form is 2D");
    if (kc < 1 || kc > SF_MAXK_CELL || ke < 1 || ke > SF_MAXK_EDGE || kn < 1 || kn > SF_MAXK_NEAR)
        return set_err(h, FL_EINVAL, "k_cell in [1,16], k_edge in [1,32], k_near in [1,64]");
    const int pw0 = quarter(s);
    if (pw0 == 0) return set_err(h, FL_ENOTIMPL, "the cluster strong form takes s in {1/4, 1/2, 3/4}");
    for (int64_t v = 0; v < P.nv; ++v)
        if (P.onb[v] && P.dov[v] >= 0) return set_err(h, FL_ENOTIMPL, "the cluster strong form takes interior DOFs");
    SF_CUDA(h, cudaSetDevice(h->device));
    SF_TRY(ensure_device_tables(h, pi, st));
    SF_TRY(ensure_sf_topology(h, pi, st));
    SF_TRY(ensure_sf_rules(h, pi, kc, ke, kn, st));
    DevTables& t = h->dev[pi];
    const int64_t nc = P.nc, nfac = t.sf_nfac, nint = t.sf_nint;
    const int q = kc * kc;
    const int64_t npts = nc * q;
    const double mexp = 2.0 * s;
    const double cA_scale = 1.0 / (2.0 * s * mexp);
    // workspace: grad (unused values), X, yrec, crec, brec (geometry of the facet points)
    const size_t n_grad = nc * 2, n_X = npts * 2, n_y = nfac * ke * 2, n_c = nfac * ke, n_b = ke;
    SF_TRY(ensure_ws(h, (n_grad + n_X + n_y + n_c + n_b + 8 * 5) * sizeof(double)));
    double* base = (double*)h->sf_ws;
    auto take = [&](size_t n) {
        double* p = base;
        base += (n + 7) / 8 * 8;
        return p;
    };
    double* grad = take(n_grad);
    double* X = take(n_X);
    double* yrec = take(n_y);
    double* crec = take(n_c);
    double* brec = take(n_b);
    const double* lam = t.sf_rule;
    const Rule Rc = make_rule(2, kc);
    const double* wc = t.sf_rule + Rc.lam.size();
    const double* te = wc + Rc.w.size();
    const double* we = te + ke;
    const double* tn = we + ke;
    const double* wn = tn + kn;
    if (nc == 0) return FL_OK;
    sf_prep_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(nc, 2, q, t.sf_perm, t.cells, t.V, t.dov, u, lam, grad, X);
    const int64_t nrec = nfac * ke;
    sf_facet_kernel<<<(unsigned)((nrec + 127) / 128), 128, 0, st>>>(nfac, nint, 2, ke, t.sf_fac, t.sf_fn, t.V, t.dov, u,
                                                                    grad, te, we, 1.0, 0.0, 0, yrec, crec, brec);
    count_launch(2);
    // near parts' jumps per group and facet
    if (g.groups > 0 && g.maxf > 0) {
        const dim3 grid((unsigned)((g.maxf + 127) / 128), (unsigned)g.groups);
        hsf_jump_kernel<<<grid, 128, 0, st>>>(g.gf_ptr, g.gf_fac, g.gbits, g.words, t.sf_fac, t.sf_fn, t.cells, t.V,
                                              t.dov, u, g.dof_leaf, cA_scale, g.cj);
        count_launch();
    }
    if (g.nblocks > 0) {
        const unsigned nb = (unsigned)g.nblocks;
#define HSF_FAR(PW)                                                                                                   \
    hsf_far_dw_kernel<PW><<<nb, SF_THREADS, 0, st>>>(g.blk_g, g.blk_p0, g.blk_ch, g.gp_ptr, g.gp_idx, g.gf_ptr,      \
                                                     g.gf_fac, g.gpo, q, X, t.sf_perm, t.cells, t.sf_fac, t.sf_fn, ke, \
                                                     yrec, we, g.cj, g.part)
        if (pw0 == 1) HSF_FAR(1);
        else if (pw0 == 2) HSF_FAR(2);
        else HSF_FAR(3);
#undef HSF_FAR
        count_launch();
    }
    hsf_near_kernel<<<(unsigned)((npts + 127) / 128), 128, 0, st>>>(
        npts, q, X, lam, t.sf_perm, t.cells, t.V, t.dov, u, t.sf_c2f, t.sf_fac, t.sf_fn, kn, tn, wn, t.sf_v2e_ptr,
        t.sf_v2e, ke, yrec, we, g.pgroup, g.plocal, g.gbits, g.words, g.dof_leaf, g.gnode, g.gp_ptr, g.gf_ptr,
        g.gf_fac, g.cj, g.gch, g.gpo,
        g.part, g.m, g.md, g.yh, g.center, g.side, s, mexp, pw0, frac_const(2, s), S);
    count_launch();
    SF_CUDA(h, cudaGetLastError());
    return FL_OK;
}

int br_from_strong_form(fl_ctx* h, double s, const double* f, int kc, const double* S, double* eta, cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!eta || !S) return set_err(h, FL_EINVAL, "NULL eta or S");
    const int d = P.dim;
    const int q = d == 1 ? kc : kc * kc;
    const int64_t nc = P.nc;
    DevTables& t = h->dev[pi];
    void* scratch = nullptr;
    cudaError_t e = pool_dev_alloc(&scratch, std::max<size_t>(nc * sizeof(double), 16));
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("indicator scratch: ") + cudaGetErrorString(e));
    double* err = (double*)scratch;
    const Rule Rc = make_rule(d, kc);
    const double* lam = t.sf_rule;
    const double* wc = t.sf_rule + Rc.lam.size();
    br_cell_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(nc, d, q, t.cells, t.V, t.jac_orig, lam, wc, f, S,
                                                                 2.0 * s, err);
    count_launch();
    if (P.n > 0) {
        br_dof_kernel<<<(unsigned)((P.n + 127) / 128), 128, 0, st>>>(P.n, t.vod, t.v2c_ptr, t.v2c, err, eta);
        count_launch();
    }
    int r = FL_OK;
    e = cudaGetLastError();
    if (e != cudaSuccess) r = set_err(h, FL_ECUDA, std::string("indicator kernels: ") + cudaGetErrorString(e));
    const cudaError_t es = cudaStreamSynchronize(st);
    pool_dev_free(scratch);
    if (r == FL_OK && es != cudaSuccess) r = set_err(h, FL_ECUDA, std::string("indicators: ") + cudaGetErrorString(es));
    return r;
}

int br_indicators(fl_ctx* h, double s, const double* u, const double* f, int kc, int ke, int kn, double* eta,
                  double* S_out, cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!eta) return set_err(h, FL_EINVAL, "NULL eta");
    if (kc < 1 || kc > SF_MAXK_CELL) return set_err(h, FL_EINVAL, "k_cell in [1,16]");
    const int d = P.dim;
    const int q = d == 1 ? kc : kc * kc;
    const int64_t nc = P.nc;
    // S (caller's or scratch) and the per-cell errors live after the strong-form workspace
    double* S = S_out;
    double* err = nullptr;
    void* scratch = nullptr;
    const size_t extra = ((S_out ? 0 : nc * q) + nc) * sizeof(double);
    cudaError_t e = pool_dev_alloc(&scratch, std::max<size_t>(extra, 16));
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("indicator scratch: ") + cudaGetErrorString(e));
    if (!S) S = (double*)scratch;
    err = (double*)scratch + (S_out ? 0 : nc * q);
    int r = strong_form(h, s, u, kc, ke, kn, S, st);
    if (r == FL_OK) {
        DevTables& t = h->dev[pi];
        const Rule Rc = make_rule(d, kc);
        const double* lam = t.sf_rule;
        const double* wc = t.sf_rule + Rc.lam.size();
        br_cell_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(nc, d, q, t.cells, t.V, t.jac_orig, lam, wc, f, S,
                                                                     2.0 * s, err);
        count_launch();
        if (P.n > 0) {
            br_dof_kernel<<<(unsigned)((P.n + 127) / 128), 128, 0, st>>>(P.n, t.vod, t.v2c_ptr, t.v2c, err, eta);
            count_launch();
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) r = set_err(h, FL_ECUDA, std::string("indicator kernels: ") + cudaGetErrorString(e));
    }
    // the scratch block goes back to the pool once the stream has used it
    cudaError_t es = cudaStreamSynchronize(st);
    pool_dev_free(scratch);
    if (r == FL_OK && es != cudaSuccess) r = set_err(h, FL_ECUDA, std::string("indicators: ") + cudaGetErrorString(es));
    return r;
}

int mark_max(fl_ctx* h, double s, const double* eta, double theta, uint8_t* dof_marks, uint8_t* cell_marks,
             cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!eta || (!dof_marks && !cell_marks)) return set_err(h, FL_EINVAL, "NULL eta, or no output");
    if (!(theta > 0.0 && theta <= 1.0)) return set_err(h, FL_EINVAL, "theta must lie in (0, 1]");
    SF_CUDA(h, cudaSetDevice(h->device));
    SF_TRY(ensure_device_tables(h, pi, st));
    SF_TRY(ensure_ws(h, std::max<size_t>(h->sf_ws_bytes, 64)));
    DevTables& t = h->dev[pi];
    double* thr = (double*)h->sf_ws;
    mark_max_kernel<<<1, 1024, 0, st>>>(P.n, eta, theta, thr);
    count_launch();
    if (dof_marks && P.n > 0) {
        mark_dof_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, st>>>(P.n, eta, thr, dof_marks);
        count_launch();
    }
    if (cell_marks) {
        mark_cell_kernel<<<(unsigned)((P.nc + 255) / 256), 256, 0, st>>>(P.nc, P.nvpc, t.cells, t.dov, eta, thr,
                                                                        cell_marks);
        count_launch();
    }
    SF_CUDA(h, cudaGetLastError());
    return FL_OK;
}

}  // namespace fl
