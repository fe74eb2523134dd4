// Dense stiffness matrix of the integral fractional Laplacian by element-pair
// quadrature (arXiv:1708.03912, Sections 2, 3, 5; Appendix B for the orders).
//
// Pipeline of fl_assemble (all on the caller's stream, fixed summation orders):
//   prep_points    quadrature offsets x_a - c_K of the far rule per cell
//   far_tile       separated pairs at vertex-graph distance >= 2: one warp per
//                  32x32 tile of cells (lane = column cell, loop over row cells),
//                  off-diagonal 3x3 blocks into lane-private shared memory, then a
//                  per-tile partial block over the tile's local DOF lists; row/column
//                  sums of the kernel for the diagonal blocks
//   near_pairs     separated pairs at distance 1 (order k_near), one thread each
//   touch_pairs    common-edge / common-vertex pairs, float64, one thread each
//   bnd_far        element x far boundary facet sums (2D), one warp per 32 cells
//   element        per cell, in two parts: the identical pair, near pairs and
//                  touching/near facets (no far-field input, runs beside far_tile),
//                  then the diagonal block from the far row sums and far facets
//   gather_csr     sparse near-field values from the contribution slots
//   compose        dense A = far partials (fixed order) + near-field values
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "cluster.h"
#include "context.h"
#include "device.h"

namespace fl {

#define FL_CUDA_TRY(h, x)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) return set_err(h, FL_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int set_err(fl_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

// ------------------------------------------------------------------ tables --

template <typename T, int Q, int NV>
struct FarRule {
    T w[Q];           // reference weights
    T wphi[Q * NV];   // reference weight x shape value
    T wpair[Q * NV];  // the same, as [b / 2][v][b % 2] (pairs of points for packed float32)
};

// ------------------------------------------------------------- far field --
template <typename T>
struct FarArgs {
    const double* cen;
    const T* pts;
    const double* jac;
    const char* hasdof;
    const int* loc;
    const int* ex_ptr;
    const int* ex_idx;
    const int* tiles;
    const int64_t* toff;
    const int* L_ptr;
    const int* inc_ptr;
    const int* inc_ent;
    T* P;
    T* Pd;      // [cell][block][point] row sums; null: not wanted (the cluster method's near field)
    int64_t nc;
    int64_t nblk;
    T expo;
};

// offsets x_a - c_K of the far rule in the arithmetic type T
template <typename T, int D>
__global__ void prep_points(const double* cvx, const double* cen, const double* lam, int q, int64_t nc, T* pts) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const double* v = cvx + k * (D + 1) * D;
    for (int a = 0; a < q; ++a) {
        for (int d = 0; d < D; ++d) {
            double x;
            if (D == 1) x = v[0] + lam[a] * (v[1] - v[0]);
            else x = v[d] + lam[2 * a] * (v[2 + d] - v[d]) + lam[2 * a + 1] * (v[4 + d] - v[d]);
            pts[(k * q + a) * D + d] = (T)(x - cen[k * D + d]);
        }
    }
}

// |x - y|^{2e} for two squared distances at once (packed float32 multiplies).
template <int PW>
__device__ __forceinline__ float2 kpow2(float2 r2, float2 e) {
    if constexpr (PW == 4 || PW == 6) {
        const float2 t = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 t2 = __fmul2_rn(t, t);
        if constexpr (PW == 4) return t2;
        else return __fmul2_rn(t2, t);
    } else {
        const float2 l = __fmul2_rn(make_float2(lg2_approx(r2.x), lg2_approx(r2.y)), e);
        return make_float2(ex2_approx(l.x), ex2_approx(l.y));
    }
}

// Sum of 16 values over the 32 lanes of a warp, scattered: halving exchanges (16, 8,
// 4, 2 lanes apart) leave lane l with the partial total of point point_of_lane16(l) over
// its half, quarter, ... of the warp; a last exchange with lane l ^ 1 completes it (lanes
// l and l ^ 1 then hold the same total).  16 shuffles in all, in a fixed order.
__device__ __forceinline__ int point_of_lane16(int lane) {
    return (((lane >> 4) & 1) << 3) | (((lane >> 3) & 1) << 2) | (((lane >> 2) & 1) << 1) | ((lane >> 1) & 1);
}
template <typename T>
__device__ __forceinline__ T reduce_scatter16(T (&v)[16], int lane) {
#pragma unroll
    for (int h = 8, bit = 16; h >= 1; h >>= 1, bit >>= 1) {
        const bool upper = (lane & bit) != 0;  // keeps the upper half of the current values
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const T send = upper ? v[k] : v[k + h];
            const T keep = upper ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int D, typename T, int Q, int PW>
__global__ void __launch_bounds__(32) far_tile_kernel(const FarArgs<T> A, const FarRule<T, Q, D + 1> R, int maxL) {
    constexpr int NV = D + 1;
    constexpr int QW = (Q + 31) / 32;
    // Q = 16: the per-point row sums are reduced once per row cell by a 16-value
    // reduce-scatter across the warp instead of one warp sum per point
    constexpr bool MR = (Q == 16);
    // float32, 2D, 16 points, PW in {0, 4, 6}: points b and b + 1 evaluated as one packed pair
    constexpr bool PK = MR && D == 2 && sizeof(T) == 4 && (PW == 0 || PW == 4 || PW == 6);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int tix = blockIdx.x;
    const int I = A.tiles[2 * tix], J = A.tiles[2 * tix + 1];
    const int nLI = A.L_ptr[I + 1] - A.L_ptr[I];
    const int nLJ = A.L_ptr[J + 1] - A.L_ptr[J];
    const int64_t nc = A.nc;
    const int64_t K0 = (int64_t)I * 32, Kt0 = (int64_t)J * 32;
    const int nI = (int)min((int64_t)32, nc - K0);

    double* sCen = reinterpret_cast<double*>(smem_raw);      // 32*D
    double* sJac = sCen + 32 * D;                             // 32
    T* sPts = reinterpret_cast<T*>(sJac + 32);                // 32*Q*D (MR: sU[a][lane], Q*32)
    T* sD = sPts + 32 * Q * (MR ? 1 : D);                     // 32*Q (diagonal tile)
    T* priv = sD + 32 * Q;                                    // NV*maxL*32
    int* sLoc = reinterpret_cast<int*>(priv + NV * maxL * 32);  // 32*NV
    int* sHas = sLoc + 32 * NV;                               // 32

    if constexpr (!MR)
        for (int i = lane; i < nI * Q * D; i += 32) sPts[i] = A.pts[K0 * Q * D + i];
    T* sU = sPts;
    for (int i = lane; i < nI * D; i += 32) sCen[i] = A.cen[K0 * D + i];
    for (int i = lane; i < nI * NV; i += 32) sLoc[i] = A.loc[K0 * NV + i];
    if (lane < nI) {
        sJac[lane] = A.jac[K0 + lane];
        sHas[lane] = A.hasdof[K0 + lane];
    }
    for (int i = lane; i < NV * nLI * 32; i += 32) priv[i] = T(0);
    for (int i = lane; i < 32 * Q; i += 32) sD[i] = T(0);
    __syncwarp();

    const int64_t Kt = Kt0 + lane;
    const bool valid = Kt < nc;
    T pj[Q][D];
    double cj[D];
    T wj = T(0);
    bool hj = false;
    int ep = 0, ee = 0;
    if (valid) {
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int d = 0; d < D; ++d) pj[b][d] = A.pts[(Kt * Q + b) * D + d];
#pragma unroll
        for (int d = 0; d < D; ++d) cj[d] = A.cen[Kt * D + d];
        wj = (T)A.jac[Kt];
        hj = A.hasdof[Kt] != 0;
        ep = A.ex_ptr[Kt];
        ee = A.ex_ptr[Kt + 1];
    } else {
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int d = 0; d < D; ++d) pj[b][d] = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) cj[d] = 0.0;
    }
    T S[Q];
    T pn[Q];  // |y_b - c_J|^2
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        S[b] = T(0);
        T q = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) q = fma(pj[b][d], pj[b][d], q);
        pn[b] = q;
    }
    // an inactive lane's row cell is moved so far that |x - y|^2 overflows to +inf and the
    // kernel value is exactly 0 (no per-evaluation select)
    const T far_away = sizeof(T) == 8 ? T(1e200) : T(1e30);
    float2 pn2[MR ? Q / 2 : 1], py0[MR ? Q / 2 : 1], py1[MR ? Q / 2 : 1], S2[MR ? Q / 2 : 1];
    float2 wp[MR ? Q / 2 : 1][NV];
    if constexpr (PK) {
#pragma unroll
        for (int c = 0; c < Q / 2; ++c) {
            pn2[c] = make_float2((float)pn[2 * c], (float)pn[2 * c + 1]);
            py0[c] = make_float2((float)pj[2 * c][0], (float)pj[2 * c + 1][0]);
            py1[c] = make_float2((float)pj[2 * c][D - 1], (float)pj[2 * c + 1][D - 1]);
            S2[c] = make_float2(0.f, 0.f);
#pragma unroll
            for (int v = 0; v < NV; ++v)
                wp[c][v] = make_float2((float)R.wpair[(c * NV + v) * 2], (float)R.wpair[(c * NV + v) * 2 + 1]);
        }
    }

    for (int kk = 0; kk < nI; ++kk) {
        const int64_t K = K0 + kk;
        bool act = valid && (I != J || kk < lane);
        if (act) {
            while (ep < ee && A.ex_idx[ep] < K) ++ep;
            if (ep < ee && A.ex_idx[ep] == K) act = false;
        }
        act = act && (hj || sHas[kk] != 0);
        const bool any = __any_sync(0xffffffffu, act);
        T myD[QW];
#pragma unroll
        for (int w = 0; w < QW; ++w) myD[w] = T(0);
        T myDa = T(0);  // MR: the row sum of point a_of_lane (lanes with bit 0 clear)
        if (any) {
            T dct[D];
#pragma unroll
            for (int d = 0; d < D; ++d) dct[d] = act ? (T)(sCen[kk * D + d] - cj[d]) : far_away;
            const T wK = (T)sJac[kk];
            T off[NV][NV];
#pragma unroll
            for (int i = 0; i < NV; ++i)
#pragma unroll
                for (int j = 0; j < NV; ++j) off[i][j] = T(0);
            if constexpr (PK) {
                const float2 e2 = make_float2((float)A.expo, (float)A.expo);
                const T* px = A.pts + K * Q * D;
                float nx0 = __ldg(px), nx1 = __ldg(px + 1);  // offsets of point 0, then prefetched
#pragma unroll 2
                for (int a = 0; a < Q; ++a) {
                    const float x0 = (float)dct[0] + nx0, x1 = (float)dct[1] + nx1;
                    if (a + 1 < Q) {
                        nx0 = __ldg(px + (a + 1) * D);
                        nx1 = __ldg(px + (a + 1) * D + 1);
                    }
                    const float xn = fmaf(x0, x0, x1 * x1);
                    const float2 xnn = make_float2(xn, xn);
                    const float2 xm0 = make_float2(-2.f * x0, -2.f * x0), xm1 = make_float2(-2.f * x1, -2.f * x1);
                    const float wa = (float)(R.w[a] * wK);
                    const float2 wa2 = make_float2(wa, wa);
                    float2 tp[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) tp[v] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < Q / 2; ++c) {
                        float2 r2 = __fadd2_rn(xnn, pn2[c]);
                        r2 = __ffma2_rn(xm0, py0[c], r2);
                        r2 = __ffma2_rn(xm1, py1[c], r2);
                        const float2 kv = kpow2<PW>(r2, e2);
#pragma unroll
                        for (int v = 0; v < NV; ++v) tp[v] = __ffma2_rn(wp[c][v], kv, tp[v]);
                        S2[c] = __ffma2_rn(wa2, kv, S2[c]);
                    }
                    T t[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) t[v] = (T)(tp[v].x + tp[v].y);
                    T u = t[0];
#pragma unroll
                    for (int v = 1; v < NV; ++v) u += t[v];
                    sU[a * 32 + lane] = u * wj;
#pragma unroll
                    for (int i = 0; i < NV; ++i)
#pragma unroll
                        for (int j = 0; j < NV; ++j) off[i][j] = fma(R.wphi[a * NV + i], t[j], off[i][j]);
                }
            } else {
#pragma unroll 1
            for (int a = 0; a < Q; ++a) {
                // |x_a - y_b|^2 = |x_a|^2 + |y_b|^2 - 2 x_a.y_b, offsets from c_J (|x_a| and
                // |y_b| are within a few cell diameters of |x_a - y_b| for separated pairs)
                T xm[D];
                T xn = T(0);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const T x = dct[d] + (MR ? __ldg(A.pts + (K * Q + a) * D + d) : sPts[(kk * Q + a) * D + d]);
                    xn = fma(x, x, xn);
                    xm[d] = T(-2) * x;
                }
                T t[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) t[v] = T(0);
                const T wa = R.w[a] * wK;
#pragma unroll
                for (int b = 0; b < Q; ++b) {
                    T r2 = xn + pn[b];
#pragma unroll
                    for (int d = 0; d < D; ++d) r2 = fma(xm[d], pj[b][d], r2);
                    const T kv = kpow<PW>(r2, A.expo);
#pragma unroll
                    for (int v = 0; v < NV; ++v) t[v] = fma(R.wphi[b * NV + v], kv, t[v]);
                    S[b] = fma(wa, kv, S[b]);
                }
                T u = t[0];
#pragma unroll
                for (int v = 1; v < NV; ++v) u += t[v];
                if constexpr (MR) {
                    sU[a * 32 + lane] = u * wj;
                } else {
                    u = warp_sum(u * wj);
#pragma unroll
                    for (int w = 0; w < QW; ++w)
                        if (a == w * 32 + lane) myD[w] = u;
                }
#pragma unroll
                for (int i = 0; i < NV; ++i)
#pragma unroll
                    for (int j = 0; j < NV; ++j) off[i][j] = fma(R.wphi[a * NV + i], t[j], off[i][j]);
            }
            }
            if constexpr (MR) {
                __syncwarp();
                T v16[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v16[q] = sU[q * 32 + lane];
                myDa = reduce_scatter16(v16, lane);
            }
            if (act) {
                const T sc = wK * wj;
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    const int li = sLoc[kk * NV + i];
                    if (li >= 0) {
#pragma unroll
                        for (int j = 0; j < NV; ++j) priv[(j * nLI + li) * 32 + lane] += off[i][j] * sc;
                    }
                }
            }
        }
        // row sums of cell K from this tile's columns
        if constexpr (MR) {
            if ((lane & 1) == 0) {
                const int a = point_of_lane16(lane);
                if (I == J) sD[kk * Q + a] += myDa;
                else if (A.Pd) A.Pd[((int64_t)K * A.nblk + J) * Q + a] = myDa;
            }
            __syncwarp();  // sU is rewritten by the next row cell
            continue;
        }
#pragma unroll
        for (int w = 0; w < QW; ++w) {
            const int a = w * 32 + lane;
            if (a < Q) {
                if (I == J) sD[kk * Q + a] += myD[w];
                else if (A.Pd) A.Pd[((int64_t)K * A.nblk + J) * Q + a] = myD[w];
            }
        }
    }
    __syncwarp();
    if constexpr (PK) {
#pragma unroll
        for (int c = 0; c < Q / 2; ++c) {
            S[2 * c] = (T)S2[c].x;
            S[2 * c + 1] = (T)S2[c].y;
        }
    }
    if (valid && A.Pd) {
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            T v = S[b];
            if (I == J) v += sD[lane * Q + b];
            A.Pd[((int64_t)Kt * A.nblk + I) * Q + b] = v;
        }
    }
    // partial block over the local DOF lists of blocks I and J
    T* Pt = A.P + A.toff[tix];
    const int pJ = A.L_ptr[J];
    for (int idx = lane; idx < nLI * nLJ; idx += 32) {
        const int li = idx / nLJ, lj = idx - li * nLJ;
        T acc = T(0);
        for (int q = A.inc_ptr[pJ + lj]; q < A.inc_ptr[pJ + lj + 1]; ++q) {
            const int e = A.inc_ent[q];
            const int l = e / NV, j = e - l * NV;
            acc += priv[(j * nLI + li) * 32 + l];
        }
        Pt[idx] = acc;
    }
}

// ------------------------------------------------------------ near pairs --
// Separated pairs at vertex-graph distance 1 with the order-k_near rule; one thread
// per unordered pair.  Writes the off-diagonal block (scaled by -C) into the
// contribution slots and the per-point row sums of both cells into Dn.
template <int D, typename T, int PW>
__global__ void near_pair_kernel(int nnear, const int* np_a, const int* np_b, const double* cvx, const double* cen,
                                 const double* jac, const double* rule, RuleOffsets ro, T expo, double C,
                                 double* contrib, int64_t slot0, double* Dn) {
    constexpr int NV = D + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnear) return;
    const int q = ro.qn;
    const double* lam = rule + ro.near_lam;
    const double* w = rule + ro.near_w;
    const double* phi = rule + ro.near_phi;
    const int ka = np_a[p], kb = np_b[p];
    // offsets of the vertices from the centroids, edge vectors, centroid difference
    T e0a[D], e1a[D], e2a[D], e0b[D], e1b[D], e2b[D], dc[D];
    const double* va = cvx + (int64_t)ka * NV * D;
    const double* vb = cvx + (int64_t)kb * NV * D;
    for (int d = 0; d < D; ++d) {
        e0a[d] = (T)(va[d] - cen[(int64_t)ka * D + d]);
        e0b[d] = (T)(vb[d] - cen[(int64_t)kb * D + d]);
        e1a[d] = (T)(va[D + d] - va[d]);
        e1b[d] = (T)(vb[D + d] - vb[d]);
        e2a[d] = (D == 2) ? (T)(va[2 * D + d] - va[d]) : T(0);
        e2b[d] = (D == 2) ? (T)(vb[2 * D + d] - vb[d]) : T(0);
        dc[d] = (T)(cen[(int64_t)ka * D + d] - cen[(int64_t)kb * D + d]);
    }
    double S[MAXQ_NEAR];
    for (int b = 0; b < q; ++b) S[b] = 0.0;
    double off[NV][NV];
    for (int i = 0; i < NV; ++i)
        for (int j = 0; j < NV; ++j) off[i][j] = 0.0;
    const double ja = jac[ka], jb = jac[kb];
    double* Da = Dn + ((int64_t)p * 2 + 0) * q;
    double* Db = Dn + ((int64_t)p * 2 + 1) * q;
    for (int a = 0; a < q; ++a) {
        T xa[D];
        for (int d = 0; d < D; ++d) {
            xa[d] = dc[d] + e0a[d] + (T)lam[a * D] * e1a[d];
            if (D == 2) xa[d] += (T)lam[a * D + 1] * e2a[d];
        }
        T t[NV];
        for (int v = 0; v < NV; ++v) t[v] = T(0);
        const T wa = (T)w[a];
        for (int b = 0; b < q; ++b) {
            T r2 = T(0);
            for (int d = 0; d < D; ++d) {
                T yb = e0b[d] + (T)lam[b * D] * e1b[d];
                if (D == 2) yb += (T)lam[b * D + 1] * e2b[d];
                T df = xa[d] - yb;
                r2 = fma(df, df, r2);
            }
            T kv = kpow<PW>(r2, expo);
            for (int v = 0; v < NV; ++v) t[v] = fma((T)(w[b] * phi[b * NV + v]), kv, t[v]);
            S[b] += (double)(wa * kv);
        }
        double u = 0.0;
        for (int v = 0; v < NV; ++v) u += (double)t[v];
        Da[a] = jb * u;
        for (int i = 0; i < NV; ++i)
            for (int j = 0; j < NV; ++j) off[i][j] += w[a] * phi[a * NV + i] * (double)t[j];
    }
    for (int b = 0; b < q; ++b) Db[b] = ja * S[b];
    double* out = contrib + slot0 + (int64_t)p * NV * NV;
    for (int i = 0; i < NV; ++i)
        for (int j = 0; j < NV; ++j) out[i * NV + j] = -C * ja * jb * off[i][j];
}

// Same computation with the order-6 rule as compile-time tables in the arithmetic
// type: per evaluation only float (or only double) operations, S in registers.
template <typename T, int QN, int D>
struct NearRule {
    T lam[QN * D];
    T w[QN];
    T wphi[QN * (D + 1)];
};

template <int D, typename T, int PW, int QN>
__global__ void near_pair_fast(int nnear, const int* np_a, const int* np_b, const double* cvx, const double* cen,
                               const double* jac, const NearRule<T, QN, D> R, T expo, double C, double* contrib,
                               int64_t slot0, double* Dn) {
    constexpr int NV = D + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnear) return;
    const int ka = np_a[p], kb = np_b[p];
    T e0a[D], e1a[D], e2a[D], e0b[D], e1b[D], e2b[D], dc[D];
    const double* va = cvx + (int64_t)ka * NV * D;
    const double* vb = cvx + (int64_t)kb * NV * D;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        e0a[d] = (T)(va[d] - cen[(int64_t)ka * D + d]);
        e0b[d] = (T)(vb[d] - cen[(int64_t)kb * D + d]);
        e1a[d] = (T)(va[D + d] - va[d]);
        e1b[d] = (T)(vb[D + d] - vb[d]);
        if constexpr (D == 2) {
            e2a[d] = (T)(va[2 * D + d] - va[d]);
            e2b[d] = (T)(vb[2 * D + d] - vb[d]);
        } else {
            e2a[d] = T(0);
            e2b[d] = T(0);
        }
        dc[d] = (T)(cen[(int64_t)ka * D + d] - cen[(int64_t)kb * D + d]);
    }
    T S[QN];
#pragma unroll
    for (int b = 0; b < QN; ++b) S[b] = T(0);
    T off[NV][NV];
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int j = 0; j < NV; ++j) off[i][j] = T(0);
    const double ja = jac[ka], jb = jac[kb];
    double* Da = Dn + ((int64_t)p * 2 + 0) * QN;
    double* Db = Dn + ((int64_t)p * 2 + 1) * QN;
#pragma unroll 1
    for (int a = 0; a < QN; ++a) {
        T xa[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            xa[d] = dc[d] + e0a[d] + R.lam[a * D] * e1a[d];
            if constexpr (D == 2) xa[d] += R.lam[a * D + 1] * e2a[d];
        }
        T t[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) t[v] = T(0);
        const T wa = R.w[a];
#pragma unroll
        for (int b = 0; b < QN; ++b) {
            T r2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                T yb = e0b[d] + R.lam[b * D] * e1b[d];
                if constexpr (D == 2) yb += R.lam[b * D + 1] * e2b[d];
                const T df = xa[d] - yb;
                r2 = fma(df, df, r2);
            }
            const T kv = kpow<PW>(r2, expo);
#pragma unroll
            for (int v = 0; v < NV; ++v) t[v] = fma(R.wphi[b * NV + v], kv, t[v]);
            S[b] = fma(wa, kv, S[b]);
        }
        T u = t[0];
#pragma unroll
        for (int v = 1; v < NV; ++v) u += t[v];
        Da[a] = jb * (double)u;
#pragma unroll
        for (int i = 0; i < NV; ++i)
#pragma unroll
            for (int j = 0; j < NV; ++j) off[i][j] = fma(R.wphi[a * NV + i], t[j], off[i][j]);
    }
#pragma unroll
    for (int b = 0; b < QN; ++b) Db[b] = ja * (double)S[b];
    double* out = contrib + slot0 + (int64_t)p * NV * NV;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int j = 0; j < NV; ++j) out[i * NV + j] = -C * ja * jb * (double)off[i][j];
}

// ---------------------------------------------------------- touching pairs --
// Common edge / common vertex pairs (2D) and common vertex pairs (1D), one warp per
// pair: lanes take the points of the (per-s) table in a strided order, then a
// butterfly sum gives every lane the same totals.
// Tables hold the angular / Duffy points with the exact radial factor folded into
// their weights.  T is the arithmetic type: float64 in the parity mode; float32 in
// the mixed mode (float32 tables and relative coordinates, the per-pair scale applied
// in float64), where the float64 version is bound by the slow float64 pipe.
template <typename T>
__device__ __forceinline__ T touch_pow(T x, T e) {
    if constexpr (sizeof(T) == 8) return pow(x, e);
    else return kpow<0>(x, e);
}

template <typename T, int PW>
__global__ void touch_pair_kernel(int ntp, int dim, const int* tp_type, const int* tp_vert, const int* tp_cell,
                                  const int64_t* tp_slot, const double* V, const double* jac_orig,
                                  const T* rule, RuleOffsets ro, double s, double C, double* contrib) {
    const int lane = threadIdx.x & 31;
    const int p = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (p >= ntp) return;
    const int type = tp_type[p];
    const int* tv = tp_vert + 5 * p;
    double* out = contrib + tp_slot[p];
    const double jK = jac_orig[tp_cell[2 * p]], jM = jac_orig[tp_cell[2 * p + 1]];
    if (type == 2) {  // 1D common vertex: [a, v, b], h1 = left, h2 = right
        const T* tb = rule + ro.t_1d;
        const T h1 = (T)jK, h2 = (T)jM;
        const T e = (T)(-1.0 - 2.0 * s);
        T acc[6] = {};
        for (int m = lane; m < ro.n_1d; m += 32) {
            const T eta = tb[2 * m], wt = tb[2 * m + 1];
            const T d1[3] = {T(1), T(-1) + eta, -eta};
            const T d2[3] = {eta, T(1) - eta, T(-1)};
            const T k1 = wt * touch_pow<T>(h1 + h2 * eta, e), k2 = wt * touch_pow<T>(h1 * eta + h2, e);
            int q = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = i; j < 3; ++j) acc[q++] += k1 * d1[i] * d1[j] + k2 * d2[i] * d2[j];
        }
        for (int q = 0; q < 6; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
            const double sc = C * jK * jM / (3.0 - 2.0 * s);
            int q = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = i; j < 3; ++j, ++q) out[i * 3 + j] = out[j * 3 + i] = sc * (double)acc[q];
        }
        return;
    }
    const T e2 = (T)(-(1.0 + s));
    if (type == 0) {  // common edge [P,Q], thirds R (K) and Rt (M)
        const double *P_ = V + 2 * tv[0], *Q_ = V + 2 * tv[1], *R_ = V + 2 * tv[2], *Rt = V + 2 * tv[3];
        const T a[2] = {(T)(Q_[0] - P_[0]), (T)(Q_[1] - P_[1])};
        const T b[2] = {(T)(R_[0] - Q_[0]), (T)(R_[1] - Q_[1])};
        const T c[2] = {(T)(-(Rt[0] - Q_[0])), (T)(-(Rt[1] - Q_[1]))};
        const T* tb = rule + ro.t_edge;
        T acc[10] = {};
        for (int m = lane; m < ro.n_edge; m += 32) {
            const T* r = tb + 8 * m;  // dphi[4], w1, w2, w3, weight
            const T x = a[0] * r[4] + b[0] * r[5] + c[0] * r[6];
            const T y = a[1] * r[4] + b[1] * r[5] + c[1] * r[6];
            const T f = r[7] * kpow<PW>(x * x + y * y, e2);
            int q = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T fi = f * r[i];
#pragma unroll
                for (int j = i; j < 4; ++j) acc[q++] += fi * r[j];
            }
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
            const double sc = C * jK * jM / ((3.0 - 2.0 * s) * (4.0 - 2.0 * s));
            int q = 0;
            for (int i = 0; i < 4; ++i)
                for (int j = i; j < 4; ++j, ++q) out[i * 4 + j] = out[j * 4 + i] = sc * (double)acc[q];
        }
    } else {  // common vertex P: K = (P,Q,R), M = (P,Qt,Rt)
        const double *P_ = V + 2 * tv[0], *Q_ = V + 2 * tv[1], *R_ = V + 2 * tv[2], *Qt = V + 2 * tv[3], *Rt = V + 2 * tv[4];
        const T a1[2] = {(T)(Q_[0] - P_[0]), (T)(Q_[1] - P_[1])};
        const T a2[2] = {(T)(R_[0] - Q_[0]), (T)(R_[1] - Q_[1])};
        const T a3[2] = {(T)(-(Qt[0] - P_[0])), (T)(-(Qt[1] - P_[1]))};
        const T a4[2] = {(T)(-(Rt[0] - Qt[0])), (T)(-(Rt[1] - Qt[1]))};
        const T* tb = rule + ro.t_vert;
        T acc[15] = {};
        for (int m = lane; m < ro.n_vert; m += 32) {
            const T* r = tb + 10 * m;  // dphi[5], x1, x2, y1, y2, weight
            const T x = a1[0] * r[5] + a2[0] * r[6] + a3[0] * r[7] + a4[0] * r[8];
            const T y = a1[1] * r[5] + a2[1] * r[6] + a3[1] * r[7] + a4[1] * r[8];
            const T f = r[9] * kpow<PW>(x * x + y * y, e2);
            int q = 0;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const T fi = f * r[i];
#pragma unroll
                for (int j = i; j < 5; ++j) acc[q++] += fi * r[j];
            }
        }
#pragma unroll
        for (int q = 0; q < 15; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
            const double sc = C * jK * jM / (4.0 - 2.0 * s);
            int q = 0;
            for (int i = 0; i < 5; ++i)
                for (int j = i; j < 5; ++j, ++q) out[i * 5 + j] = out[j * 5 + i] = sc * (double)acc[q];
        }
    }
}

// ------------------------------------------------------ boundary, far facets --
// 2D: for each cell the sums B_a = Σ_e Σ_b w_b n_e·(x_a - y_b) |x_a - y_b|^{-2-2s}
// over all boundary facets not listed as touching/near for that cell.  A block of
// BND_WARPS warps serves 32 cells (lane = cell); warp w takes the facets f = w, w +
// BND_WARPS, ...; the per-warp sums are added in warp order.  Facet data come from a
// compact per-facet record (start point, edge, normal and length, float64).
constexpr int BND_WARPS = 4;


__global__ void facet_records_kernel(int64_t nf, const int* F, const double* FN, const double* FLEN, const double* V,
                                     FacetRec* out) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double* E0 = V + 2 * F[2 * f];
    const double* E1 = V + 2 * F[2 * f + 1];
    FacetRec r;
    r.e0x = E0[0];
    r.e0y = E0[1];
    r.ex = E1[0] - E0[0];
    r.ey = E1[1] - E0[1];
    r.nx = FN[2 * f];
    r.ny = FN[2 * f + 1];
    r.len = FLEN[f];
    r.pad = 0.0;
    out[f] = r;
}

template <typename T, int Q, int PW>
__global__ void __launch_bounds__(32 * BND_WARPS) bnd_far_kernel(int64_t nc, int64_t nf, const double* cen, const T* pts,
                                                                  const char* hasdof, const int* ef_ptr,
                                                                  const int* ef_fac, const FacetRec* FR,
                                                                  const double* F64, const double* rule, RuleOffsets ro,
                                                                  T expo, double* Bf) {
    __shared__ double part[BND_WARPS][Q][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = k < nc && hasdof[k];
    T xa[Q][2];
    double c[2] = {0.0, 0.0};
    int ep = 0, ee = 0;
    if (valid) {
        for (int a = 0; a < Q; ++a) {
            xa[a][0] = pts[(k * Q + a) * 2];
            xa[a][1] = pts[(k * Q + a) * 2 + 1];
        }
        c[0] = cen[2 * k];
        c[1] = cen[2 * k + 1];
        ep = ef_ptr[k];
        ee = ef_ptr[k + 1];
    } else {
        for (int a = 0; a < Q; ++a) xa[a][0] = xa[a][1] = T(0);
    }
    const int kf = ro.kf;
    const double* gt = rule + ro.glf_t;
    const double* gw = rule + ro.glf_w;
    double B[Q];
    T Bp[Q];
    for (int a = 0; a < Q; ++a) B[a] = 0.0, Bp[a] = T(0);
    int since = 0;
    const bool any = __any_sync(0xffffffffu, valid);
    for (int64_t f = wid; any && f < nf; f += BND_WARPS) {
        bool act = valid;
        if (act) {
            while (ep < ee && ef_fac[ep] < f) ++ep;
            if (ep < ee && ef_fac[ep] == f) act = false;
        }
        const FacetRec r = FR[f];
        const T ex = (T)r.ex, ey = (T)r.ey, nx = (T)r.nx, ny = (T)r.ny;
        T dcx = (T)(c[0] - r.e0x), dcy = (T)(c[1] - r.e0y);
        if (!act) {  // far away and zero-weighted: every value stays finite
            dcx = T(1.0e3);
            dcy = T(1.0e3);
        }
        const T L = act ? (T)r.len : T(0);
        for (int b = 0; b < kf; ++b) {
            const T tb = (T)gt[b], wb = (T)gw[b] * L;
            const T yx = tb * ex, yy = tb * ey;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const T dx = dcx + xa[a][0] - yx, dy = dcy + xa[a][1] - yy;
                const T kv = kpow<PW>(fma(dx, dx, dy * dy), expo);
                Bp[a] = fma(wb * (nx * dx + ny * dy), kv, Bp[a]);
            }
        }
        if (++since == 32) {
            for (int a = 0; a < Q; ++a) B[a] += (double)Bp[a], Bp[a] = T(0);
            since = 0;
        }
    }
    for (int a = 0; a < Q; ++a) part[wid][a][lane] = B[a] + (double)Bp[a];
    __syncthreads();
    if (wid == 0 && valid)
        for (int a = 0; a < Q; ++a) {
            double acc = 0.0;
            for (int w = 0; w < BND_WARPS; ++w) acc += part[w][a][lane];
            Bf[k * Q + a] = acc;
        }
}

// ------------------------------------------------------------- per element --
struct ElemArgs {
    int dim;
    int64_t nc, nblk, nf, nnear;
    const double* cvx;
    const double* cen;
    const double* jac;
    const char* hasdof;
    const void* Pd;     // T
    int pd_is_float;
    const double* Dn;
    const int* enp_ptr;
    const int* enp_ent;
    const double* Bf;
    const int* ef_ptr;
    const int* ef_fac;
    const int* ef_cls;
    const int* F;
    const double* FN;
    const double* FLEN;
    const double* V;
    const int* corner;  // nc*nvpc original vertex ids in internal order
    const double* rule;
    const float* rule32;  // float32 tables in the mixed mode (identical pair and 2D facet powers in float32), else null
    RuleOffsets ro;
    double s, C;
    double C2s;             // C / (2s)
    double r2s, r3s, r4s;   // 1 / (2 - 2s), 1 / (3 - 2s), 1 / (4 - 2s)
    int regional;
    double* contrib;
    int64_t slot0;
    double* eblk;  // nc x 6: the far-independent part of each cell's block (PART 1 -> PART 2)
    // 1: the cluster method's near field.  The ef lists then hold, per cell K, the facets of the
    // boundary of N(K) (K, its touching cells and those at vertex-graph distance 1), classes 0-3
    // (0 = far), with normals pointing into N(K), in place of the boundary facets of Omega; there
    // are no far row sums (nblk = 0) and no Bf: the far pairs' diagonal-block terms and the
    // boundary term are the integral over that boundary (divergence theorem), its class-0
    // facets at the far rule's points in PART 2 (2D) or in the facet loop (1D).
    int cluster;
};

// One warp per cell with DOFs.  Lanes take quadrature points (or partner blocks)
// in a strided order; the upper triangle of the local block is summed over lanes
// with a butterfly at the end.
__device__ __forceinline__ int tri_index(int i, int j, int NV) {  // i <= j
    return i * NV - i * (i - 1) / 2 + (j - i);
}

// s += x with the running compensation c (Kahan); no reassociation is applied to it.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// |x - y|^{2e} from r2 = |x - y|^2 for the 2D boundary facets: float64, or in the mixed
// mode float32 (the float64 power is the slow pipe's work; the geometry stays float64).
template <int PW>
__device__ __forceinline__ double facet_pow(double r2, double e, bool f32) {
    if (f32) {
        constexpr int PWF = (PW == 4 || PW == 6) ? PW : 0;
        return (double)kpow<PWF>((float)r2, (float)e);
    }
    return kpow<PW>(r2, e);
}

// The block blk (upper triangle, 6 values in 2D) stays in registers: the dimension is a
// template parameter and every update of it uses a compile-time index.
// PART 1: everything that does not need the far field (near pairs and facets, identical
// pair, touching facets), summed over the warp into A.eblk[k]; it runs while the far
// tile kernel runs, on the float64 pipe that kernel leaves idle.  PART 2: the diagonal
// block from the far row sums and far facets, plus A.eblk[k], into the contribution slots.
template <int PW, int D, int PART>
__global__ void element_kernel(ElemArgs A) {
    constexpr int NV = D + 1;
    const int lane = threadIdx.x & 31;
    const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (k >= A.nc || !A.hasdof[k]) return;
    const RuleOffsets& ro = A.ro;
    const double* rule = A.rule;
    const double s = A.s, C = A.C;
    const double* v = A.cvx + k * NV * D;
    const double jk = A.jac[k];
    double blk[6] = {};
    const int qf = ro.qf, qn = ro.qn;
    // diagonal block from the far row sums and far facets.  Lanes own (point a, half h)
    // and add the partner blocks B = h, h+2, h+4, ... in a fixed order with four
    // independent accumulators; the two halves are then added.
    if constexpr (PART == 2) {
        const double* w = rule + ro.far_w;
        const double* phi = rule + ro.far_phi;
        const int npass = (qf + 15) / 16;
        for (int pass = 0; pass < npass; ++pass) {
            const int a = pass * 16 + (lane & 15), hb = lane >> 4;
            double Dk = 0.0;
            if (a < qf) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int64_t B = hb;
                if (A.pd_is_float) {
                    // compensated (Kahan) float32 sums: float64 accuracy without the slow pipe
                    const float* Pd = (const float*)A.Pd + k * A.nblk * qf + a;
                    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
                    for (; B + 6 < A.nblk; B += 8) {
                        kahan_add(f0, c0, Pd[B * qf]);
                        kahan_add(f1, c1, Pd[(B + 2) * qf]);
                        kahan_add(f2, c2, Pd[(B + 4) * qf]);
                        kahan_add(f3, c3, Pd[(B + 6) * qf]);
                    }
                    for (; B < A.nblk; B += 2) kahan_add(f0, c0, Pd[B * qf]);
                    s0 = (double)f0 - (double)c0;
                    s1 = (double)f1 - (double)c1;
                    s2 = (double)f2 - (double)c2;
                    s3 = (double)f3 - (double)c3;
                } else {
                    const double* Pd = (const double*)A.Pd + k * A.nblk * qf + a;
                    for (; B + 6 < A.nblk; B += 8) {
                        s0 += Pd[B * qf];
                        s1 += Pd[(B + 2) * qf];
                        s2 += Pd[(B + 4) * qf];
                        s3 += Pd[(B + 6) * qf];
                    }
                    for (; B < A.nblk; B += 2) s0 += Pd[B * qf];
                }
                Dk = (s0 + s1) + (s2 + s3);
            }
            const double other = __shfl_xor_sync(0xffffffffu, Dk, 16);
            Dk = (hb == 0) ? Dk + other : other + Dk;
            if (hb == 0 && a < qf) {
                double bf = 0.0;
                if (D == 2 && !A.regional && !A.cluster) bf = A.Bf[k * qf + a];
                if (D == 2 && A.cluster) {
                    // class-0 facets of the boundary of N(K) at far-rule point a, k_far-point Gauss rule
                    const double* lam = rule + ro.far_lam;
                    const double* gt = rule + ro.glf_t;
                    const double* gw = rule + ro.glf_w;
                    double xa[2];
                    for (int d = 0; d < 2; ++d)
                        xa[d] = v[d] + lam[a * 2] * (v[2 + d] - v[d]) + lam[a * 2 + 1] * (v[4 + d] - v[d]);
                    for (int q = A.ef_ptr[k]; q < A.ef_ptr[k + 1]; ++q) {
                        if (A.ef_cls[q] != 0) continue;
                        const int f = A.ef_fac[q];
                        const double* E0 = A.V + 2 * A.F[2 * f];
                        const double* E1 = A.V + 2 * A.F[2 * f + 1];
                        double acc = 0.0;
                        for (int b = 0; b < ro.kf; ++b) {
                            const double dx = xa[0] - (E0[0] + gt[b] * (E1[0] - E0[0]));
                            const double dy = xa[1] - (E0[1] + gt[b] * (E1[1] - E0[1]));
                            acc += gw[b] * A.FLEN[f] * (A.FN[2 * f] * dx + A.FN[2 * f + 1] * dy) *
                                   facet_pow<PW>(dx * dx + dy * dy, -(1.0 + s), false);
                        }
                        bf += acc;
                    }
                }
                const double f = jk * w[a] * (C * Dk + A.C2s * bf);
#pragma unroll
                for (int i = 0; i < NV; ++i)
#pragma unroll
                    for (int j = i; j < NV; ++j) blk[tri_index(i, j, NV)] += f * phi[a * NV + i] * phi[a * NV + j];
            }
        }
    }
    if constexpr (PART == 1) {
    // near pairs (both roles) and near boundary facets, order-k_near points
    {
        const double* w = rule + ro.near_w;
        const double* phi = rule + ro.near_phi;
        const double* lam = rule + ro.near_lam;
        for (int a = lane; a < qn; a += 32) {
            double Dk = 0.0, D1 = 0.0;
            const int q0 = A.enp_ptr[k], q1 = A.enp_ptr[k + 1];
            int q = q0;
            for (; q + 1 < q1; q += 2) {
                Dk += A.Dn[(int64_t)A.enp_ent[q] * qn + a];
                D1 += A.Dn[(int64_t)A.enp_ent[q + 1] * qn + a];
            }
            if (q < q1) Dk += A.Dn[(int64_t)A.enp_ent[q] * qn + a];
            Dk += D1;
            double Bn = 0.0;
            if (!A.regional) {
                double xa[2] = {0.0, 0.0};
                for (int d = 0; d < D; ++d) {
                    xa[d] = v[d] + lam[a * D] * (v[D + d] - v[d]);
                    if (D == 2) xa[d] += lam[a * D + 1] * (v[2 * D + d] - v[d]);
                }
                for (int q = A.ef_ptr[k]; q < A.ef_ptr[k + 1]; ++q) {
                    if (A.ef_cls[q] != 1) continue;
                    const int f = A.ef_fac[q];
                    if (D == 1) {
                        const double dx = xa[0] - A.V[A.F[f]];
                        Bn += A.FN[f] * dx * pow(dx * dx, -(1.0 + 2.0 * s) / 2.0);
                    } else {
                        const double* E0 = A.V + 2 * A.F[2 * f];
                        const double* E1 = A.V + 2 * A.F[2 * f + 1];
                        const double* gt = rule + ro.gln_t;
                        const double* gw = rule + ro.gln_w;
                        double acc = 0.0;
                        for (int b = 0; b < ro.kn; ++b) {
                            const double dx = xa[0] - (E0[0] + gt[b] * (E1[0] - E0[0]));
                            const double dy = xa[1] - (E0[1] + gt[b] * (E1[1] - E0[1]));
                            acc += gw[b] * A.FLEN[f] * (A.FN[2 * f] * dx + A.FN[2 * f + 1] * dy) *
                                   facet_pow<PW>(dx * dx + dy * dy, -(1.0 + s), A.rule32 != nullptr);
                        }
                        Bn += acc;
                    }
                }
            }
            const double f = jk * w[a] * (C * Dk + A.C2s * Bn);
#pragma unroll
            for (int i = 0; i < NV; ++i)
#pragma unroll
                for (int j = i; j < NV; ++j) blk[tri_index(i, j, NV)] += f * phi[a * NV + i] * phi[a * NV + j];
        }
    }
    // identical pair
    if (D == 1) {
        if (lane == 0) {
            const double val = C * pow(jk, 1.0 - 2.0 * s) / ((2.0 - 2.0 * s) * (3.0 - 2.0 * s));
            blk[0] += val;
            blk[1] -= val;
            blk[2] += val;
        }
    } else if (A.rule32) {
        // mixed mode: the same sum in float32 (float64 pow is the slow pipe's work here)
        constexpr int PWF = (PW == 4 || PW == 6) ? PW : 0;
        const float J00 = (float)(v[2] - v[0]), J10 = (float)(v[3] - v[1]);
        const float J01 = (float)(v[4] - v[0]), J11 = (float)(v[5] - v[1]);
        const float* tb = A.rule32 + ro.t_ident;
        const float e2 = (float)(-(1.0 + s));
        float bf[6] = {};
        for (int m = lane; m < ro.n_ident; m += 32) {
            const float u0 = tb[3 * m], u1 = tb[3 * m + 1], f0 = tb[3 * m + 2];
            const float jx = J00 * u0 + J01 * u1, jy = J10 * u0 + J11 * u1;
            const float f = f0 * kpow<PWF>(jx * jx + jy * jy, e2);
            const float g[3] = {-u0 - u1, u0, u1};
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) bf[tri_index(i, j, 3)] += f * g[i] * g[j];
        }
        const double beta = 2.0 * A.r2s * A.r3s * A.r4s;
        const double sc = 0.5 * C * jk * jk * beta;
        for (int q = 0; q < 6; ++q) blk[q] += sc * (double)bf[q];
    } else {
        const double J00 = v[2] - v[0], J10 = v[3] - v[1], J01 = v[4] - v[0], J11 = v[5] - v[1];
        const double* tb = rule + ro.t_ident;
        const double beta = 2.0 / ((2.0 - 2.0 * s) * (3.0 - 2.0 * s) * (4.0 - 2.0 * s));
        const double sc = 0.5 * C * jk * jk * beta;
        for (int m = lane; m < ro.n_ident; m += 32) {
            const double u0 = tb[3 * m], u1 = tb[3 * m + 1], f0 = tb[3 * m + 2];
            const double jx = J00 * u0 + J01 * u1, jy = J10 * u0 + J11 * u1;
            const double f = sc * f0 * kpow<PW>(jx * jx + jy * jy, -(1.0 + s));
            const double g[3] = {-u0 - u1, u0, u1};
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) blk[tri_index(i, j, 3)] += f * g[i] * g[j];
        }
    }
    // boundary facets: touching ones (and, in 1D, far ones)
    if (!A.regional) {
        const int* cv = A.corner + k * NV;
        if (D == 1) {
            int ep = A.ef_ptr[k], ee = A.ef_ptr[k + 1];
            const double* w = rule + ro.far_w;
            const double* lam = rule + ro.far_lam;
            const double* phi = rule + ro.far_phi;
            // dense: every boundary facet of Omega, classes from the list; cluster: the list itself
            const int64_t nloop = A.cluster ? (int64_t)(ee - ep) : A.nf;
            for (int64_t it = 0; it < nloop; ++it) {
                int64_t f = it;
                int cls = 0;
                if (A.cluster) {
                    f = A.ef_fac[ep + it];
                    cls = A.ef_cls[ep + it];
                } else {
                    while (ep < ee && A.ef_fac[ep] < f) ++ep;
                    if (ep < ee && A.ef_fac[ep] == f) cls = A.ef_cls[ep];
                }
                if (cls == 1) continue;  // near: done above
                const int e = A.F[f];
                if (cls == 2) {
                    if (lane == 0) {
                        // e is an end of K: exact ∫ phi_i phi_j |x-e|^{-2s}
                        const int me = (cv[0] == e) ? 0 : 1;
                        const double a_[2] = {me == 0 ? 1.0 : 0.0, me == 1 ? 1.0 : 0.0};
                        const double b_[2] = {me == 0 ? -1.0 : 1.0, me == 1 ? -1.0 : 1.0};
                        const double sc = C / (2.0 * s) * pow(jk, 1.0 - 2.0 * s);
                        for (int i = 0; i < 2; ++i)
                            for (int j = i; j < 2; ++j) {
                                double val = (a_[i] * b_[j] + a_[j] * b_[i]) / (2.0 - 2.0 * s) + b_[i] * b_[j] / (3.0 - 2.0 * s);
                                if (a_[i] * a_[j] != 0.0) val += a_[i] * a_[j] / (1.0 - 2.0 * s);
                                blk[tri_index(i, j, 2)] += sc * val;
                            }
                    }
                } else {
                    const double y = A.V[e];
                    for (int a = lane; a < qf; a += 32) {
                        const double dx = v[0] + lam[a] * (v[1] - v[0]) - y;
                        const double g = A.FN[f] * dx * pow(dx * dx, -(1.0 + 2.0 * s) / 2.0);
                        const double fw = C / (2.0 * s) * jk * w[a] * g;
                        for (int i = 0; i < 2; ++i)
                            for (int j = i; j < 2; ++j) blk[tri_index(i, j, 2)] += fw * phi[a * 2 + i] * phi[a * 2 + j];
                    }
                }
            }
        } else {
            for (int q = A.ef_ptr[k]; q < A.ef_ptr[k + 1]; ++q) {
                const int cls = A.ef_cls[q];
                const int f = A.ef_fac[q];
                if (cls == 2) {
                    // facet is an edge of K; only the opposite vertex R can carry a DOF
                    const int E0 = A.F[2 * f], E1 = A.F[2 * f + 1];
                    int r = 0;
                    for (int i = 0; i < 3; ++i)
                        if (cv[i] != E0 && cv[i] != E1) r = i;
                    const double* pE0 = A.V + 2 * E0;
                    const double* pE1 = A.V + 2 * E1;
                    const double* pR = A.V + 2 * cv[r];
                    const double nx = A.FN[2 * f], ny = A.FN[2 * f + 1];
                    const double H = nx * (pR[0] - pE1[0]) + ny * (pR[1] - pE1[1]);
                    const double ax = pE1[0] - pE0[0], ay = pE1[1] - pE0[1];
                    const double bx = pR[0] - pE1[0], by = pR[1] - pE1[1];
                    const double* tb = rule + ro.b_own;
                    const double sc = A.C2s * jk * A.FLEN[f] * A.r3s * A.r4s;
                    double own = 0.0;
                    for (int m = lane; m < ro.n_own; m += 32) {
                        const double o1 = tb[3 * m], o2 = tb[3 * m + 1], wt = tb[3 * m + 2];
                        const double x = ax * o1 + bx * o2, y = ay * o1 + by * o2;
                        own += sc * wt * H * o2 * facet_pow<PW>(x * x + y * y, -(1.0 + s), A.rule32 != nullptr) * o2 * o2;
                    }
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (q == r) blk[tri_index(q, q, 3)] += own;
                } else if (cls == 3) {
                    // facet and K share one vertex P
                    const int fa = A.F[2 * f], fb = A.F[2 * f + 1];
                    int ip = 0;
                    for (int i = 0; i < 3; ++i)
                        if (cv[i] == fa || cv[i] == fb) ip = i;
                    const int P = cv[ip], E1 = (P == fa) ? fb : fa;
                    const int iq = (ip + 1) % 3, ir = (ip + 2) % 3;
                    const double* pP = A.V + 2 * P;
                    const double* pQ = A.V + 2 * cv[iq];
                    const double* pR = A.V + 2 * cv[ir];
                    const double* pE = A.V + 2 * E1;
                    const double nx = A.FN[2 * f], ny = A.FN[2 * f + 1];
                    const double gq[2] = {pQ[0] - pP[0], pQ[1] - pP[1]};
                    const double gr[2] = {pR[0] - pQ[0], pR[1] - pQ[1]};
                    const double ge[2] = {pE[0] - pP[0], pE[1] - pP[1]};
                    const double* tb = rule + ro.b_vert;
                    const double sc = A.C2s * jk * A.FLEN[f];
                    const int idx[3] = {ip, iq, ir};
                    // local order (P, Q, R): a = e_P, bh = (e_Q - e_P) x1 + (e_R - e_Q) x2; the
                    // local block is summed first, then placed by the cell's vertex order
                    double lb[6] = {};
                    for (int m = lane; m < ro.n_bvert; m += 32) {
                        const double x1 = tb[4 * m], x2 = tb[4 * m + 1], t = tb[4 * m + 2], wt = tb[4 * m + 3];
                        const double xpx = gq[0] * x1 + gr[0] * x2, xpy = gq[1] * x1 + gr[1] * x2;
                        const double N = xpx * nx + xpy * ny;
                        const double dx = xpx - t * ge[0], dy = xpy - t * ge[1];
                        const double g = sc * wt * N * facet_pow<PW>(dx * dx + dy * dy, -(1.0 + s), A.rule32 != nullptr);
                        const double bh[3] = {-x1, x1 - x2, x2};
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int j = i; j < 3; ++j) {
                                const double ai = (i == 0) ? 1.0 : 0.0, aj = (j == 0) ? 1.0 : 0.0;
                                double val = g * bh[i] * bh[j] * A.r4s + g * (ai * bh[j] + aj * bh[i]) * A.r3s;
                                if (i == 0 && j == 0) val += g * A.r2s;
                                lb[tri_index(i, j, 3)] += val;
                            }
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = i; j < 3; ++j) {
#pragma unroll
                            for (int I_ = 0; I_ < 3; ++I_)
#pragma unroll
                                for (int J_ = I_; J_ < 3; ++J_)
                                    if ((idx[i] == I_ && idx[j] == J_) || (idx[i] == J_ && idx[j] == I_))
                                        blk[tri_index(I_, J_, 3)] += lb[tri_index(i, j, 3)];
                        }
                }
            }
        }
    }
    }  // PART == 1
#pragma unroll
    for (int q = 0; q < NV * (NV + 1) / 2; ++q) blk[q] = warp_sum(blk[q]);
    if constexpr (PART == 1) {
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NV * (NV + 1) / 2; ++q) A.eblk[k * 6 + q] = blk[q];
        return;
    }
#pragma unroll
    for (int q = 0; q < NV * (NV + 1) / 2; ++q) blk[q] += A.eblk[k * 6 + q];
    if (lane == 0) {
        double* out = A.contrib + A.slot0 + k * NV * NV;
#pragma unroll
        for (int i = 0; i < NV; ++i)
#pragma unroll
            for (int j = i; j < NV; ++j) out[i * NV + j] = out[j * NV + i] = blk[tri_index(i, j, NV)];
    }
}

// ---------------------------------------------------- gather and compose --
__global__ void gather_csr_kernel(int64_t nnz, const int* csr_row, const int* csr_col, const int64_t* g_ptr,
                                  const int64_t* g_slot, const double* contrib, double* val) {
    const int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (z >= nnz) return;
    if (csr_col[z] < csr_row[z]) return;  // the upper entry serves both
    double acc = 0.0;
    for (int64_t q = g_ptr[z]; q < g_ptr[z + 1]; ++q) acc += contrib[g_slot[q]];
    val[z] = acc;
}

// Full symmetric values of the near-field CSR: an upper entry (col >= row) as gathered; a
// lower entry (i, j), j < i, takes the value of (j, i), found by bisection among row j's
// ascending columns (the pattern is symmetric, so it is there; NaN marks a broken pattern).
__global__ void csr_full_values_kernel(int64_t nnz, const int* csr_ptr, const int* csr_row, const int* csr_col,
                                       const double* val, double* out) {
    const int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (z >= nnz) return;
    const int i = csr_row[z], j = csr_col[z];
    if (j >= i) {
        out[z] = val[z];
        return;
    }
    int lo = csr_ptr[j], hi = csr_ptr[j + 1] - 1;
    if (lo > hi) {
        out[z] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        if (csr_col[mid] < i) lo = mid + 1;
        else hi = mid;
    }
    out[z] = csr_col[lo] == i ? val[lo] : __longlong_as_double(0x7ff8000000000000LL);
}

// A_ij = -C sum over the block occurrences (Ba, la) of DOF min(i, j) and (Bb, lb) of DOF
// max(i, j) of the tile partial blocks, in occurrence order (a major, b minor), so A_ij and
// A_ji are the same sum.  One block per 32 x 32 tile of the upper triangle (tile row
// IB <= tile column JB): 8 warps, each thread four rows of one column; the tile is written
// as is and, through shared memory, transposed, both with coalesced stores.
template <typename T>
__global__ void __launch_bounds__(256) compose_far_kernel(int64_t n, int64_t nblk, const int* occ_ptr,
                                                          const int* occ_blk, const int* occ_loc, const int* L_ptr,
                                                          const int64_t* toff, const T* P, double negC, double* A,
                                                          int64_t lda) {
    __shared__ double tile[32][33];
    // tile index -> (IB, JB), IB <= JB, in row order of the upper triangle
    const int64_t nt = (n + 31) / 32;
    int64_t rem = blockIdx.x, IB = 0;
    while (rem >= nt - IB) {
        rem -= nt - IB;
        ++IB;
    }
    const int64_t JB = IB + rem;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j = JB * 32 + tx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = IB * 32 + ty + 8 * k;
        double acc = 0.0;
        if (i < n && j < n) {
            const int64_t lo = min(i, j), hi = max(i, j);
            // float32 partials: a compensated float32 sum (s, c) holds the total to about
            // float64 accuracy for these few same-signed terms and keeps the float64 pipe
            // (1/64 of the float32 rate here) out of the loop; float64 partials: a float64 sum
            float ks = 0.f, kc = 0.f;
            auto add = [&](T x) {
                if constexpr (sizeof(T) == 4) kahan_add(ks, kc, x);
                else acc += x;
            };
            for (int a = occ_ptr[lo]; a < occ_ptr[lo + 1]; ++a) {
                const int64_t Ba = occ_blk[a];
                const int la = occ_loc[a];
                for (int b = occ_ptr[hi]; b < occ_ptr[hi + 1]; ++b) {
                    const int64_t Bb = occ_blk[b];
                    const int lb = occ_loc[b];
                    if (Ba < Bb) {
                        const int64_t t = Ba * nblk - Ba * (Ba - 1) / 2 + (Bb - Ba);
                        add(P[toff[t] + (int64_t)la * (L_ptr[Bb + 1] - L_ptr[Bb]) + lb]);
                    } else if (Ba > Bb) {
                        const int64_t t = Bb * nblk - Bb * (Bb - 1) / 2 + (Ba - Bb);
                        add(P[toff[t] + (int64_t)lb * (L_ptr[Ba + 1] - L_ptr[Ba]) + la]);
                    } else {
                        const int64_t t = Ba * nblk - Ba * (Ba - 1) / 2;
                        const int64_t nL = L_ptr[Ba + 1] - L_ptr[Ba];
                        add(P[toff[t] + (int64_t)la * nL + lb]);
                        add(P[toff[t] + (int64_t)lb * nL + la]);
                    }
                }
            }
            if constexpr (sizeof(T) == 4) acc = (double)ks - (double)kc;
            A[i * lda + j] = negC * acc;
        }
        tile[ty + 8 * k][tx] = negC * acc;
    }
    if (IB == JB) return;
    __syncthreads();
    // transposed tile: rows JB*32 + ..., columns IB*32 + tx
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t r = JB * 32 + ty + 8 * k, c = IB * 32 + tx;
        if (r < n && c < n) A[r * lda + c] = tile[tx][ty + 8 * k];
    }
}

__global__ void add_csr_kernel(int64_t nnz, const int* csr_row, const int* csr_col, const double* val, double* A,
                               int64_t lda) {
    const int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (z >= nnz) return;
    const int64_t i = csr_row[z], j = csr_col[z];
    if (j < i) return;
    const double v = val[z];
    A[i * lda + j] += v;
    if (j != i) A[j * lda + i] += v;
}

// Near-field entries of the cluster method (Section 6).  Entry z = (i, j): the contribution slots
// of the mesh plan's sparse entry (min, max), if that entry exists, summed in its gather order,
// plus -C times the tile partials over the block occurrences of min(i, j) (major) and max(i, j),
// summed as compose_far_kernel sums them; the product and the sum are not fused, so an entry
// whose slots hold no diagonal block is bitwise the dense matrix's.  Tiles are found by
// bisection in their row of the tile list; a tile missing from it (a broken plan) gives NaN.
template <typename T>
__global__ void hnear_compose_kernel(int64_t nnz, const int* __restrict__ nz_row, const int* __restrict__ nz_col,
                                     const int* __restrict__ csr_ptr, const int* __restrict__ csr_col,
                                     const int64_t* __restrict__ g_ptr, const int64_t* __restrict__ g_slot,
                                     const double* __restrict__ contrib, const int* __restrict__ occ_ptr,
                                     const int* __restrict__ occ_blk, const int* __restrict__ occ_loc,
                                     const int* __restrict__ L_ptr, const int* __restrict__ trow_ptr,
                                     const int* __restrict__ tiles, const int64_t* __restrict__ toff,
                                     const T* __restrict__ Pt, double negC, double* __restrict__ val) {
    const int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (z >= nnz) return;
    const int i = nz_row[z], j = nz_col[z];
    const int lo = min(i, j), hi = max(i, j);
    double acc = 0.0;
    {
        int a = csr_ptr[lo], b = csr_ptr[lo + 1] - 1;
        if (a <= b) {
            while (a < b) {
                const int mid = a + (b - a) / 2;
                if (csr_col[mid] < hi) a = mid + 1;
                else b = mid;
            }
            if (csr_col[a] == hi)
                for (int64_t q = g_ptr[a]; q < g_ptr[a + 1]; ++q) acc += contrib[g_slot[q]];
        }
    }
    double far = 0.0;
    // float32 partials: a compensated float32 sum, as in compose_far_kernel
    float ks = 0.f, kc = 0.f;
    auto add = [&](T x) {
        if constexpr (sizeof(T) == 4) kahan_add(ks, kc, x);
        else far += x;
    };
    bool missing = false;
    for (int oa = occ_ptr[lo]; oa < occ_ptr[lo + 1]; ++oa) {
        const int Ba = occ_blk[oa], la = occ_loc[oa];
        for (int ob = occ_ptr[hi]; ob < occ_ptr[hi + 1]; ++ob) {
            const int Bb = occ_blk[ob], lb = occ_loc[ob];
            const int B0 = min(Ba, Bb), B1 = max(Ba, Bb);
            int a = trow_ptr[B0], b = trow_ptr[B0 + 1] - 1;
            if (a > b) {
                missing = true;
                continue;
            }
            while (a < b) {
                const int mid = a + (b - a) / 2;
                if (tiles[2 * mid + 1] < B1) a = mid + 1;
                else b = mid;
            }
            if (tiles[2 * a + 1] != B1) {
                missing = true;
                continue;
            }
            const int64_t base = toff[a];
            if (Ba < Bb) {
                add(Pt[base + (int64_t)la * (L_ptr[Bb + 1] - L_ptr[Bb]) + lb]);
            } else if (Ba > Bb) {
                add(Pt[base + (int64_t)lb * (L_ptr[Ba + 1] - L_ptr[Ba]) + la]);
            } else {
                const int64_t nL = L_ptr[Ba + 1] - L_ptr[Ba];
                add(Pt[base + (int64_t)la * nL + lb]);
                add(Pt[base + (int64_t)lb * nL + la]);
            }
        }
    }
    if constexpr (sizeof(T) == 4) far = (double)ks - (double)kc;
    val[z] = missing ? __longlong_as_double(0x7ff8000000000000LL) : __dadd_rn(__dmul_rn(negC, far), acc);
}

// ------------------------------------------------- symmetry reduction --
// Rows of the orbit representatives (Section 7, "Exploiting Symmetry"): R[r][j] is the far-field
// part of the whole matrix's entry (rep_r, j), summed from the tile partials exactly as
// compose_far_kernel sums them (occurrences of min(i, j) major), so R[r][j] equals that entry.
// Every tile read holds a representative's cell and is in the list; a missing one (a broken
// plan) shows as NaN.  Grid: x over columns, y over representatives (strided).
template <typename T>
__global__ void compose_rows_kernel(int64_t n, int64_t nred, int64_t nblk, const int* red_rep, const int* occ_ptr,
                                    const int* occ_blk, const int* occ_loc, const int* L_ptr, const int64_t* tri_list,
                                    const int64_t* toff, const T* P, double negC, double* R, int64_t ldr) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int64_t r = blockIdx.y; r < nred; r += gridDim.y) {
        const int64_t i = red_rep[r];
        const int64_t lo = min(i, j), hi = max(i, j);
        double acc = 0.0;
        float ks = 0.f, kc = 0.f;
        bool missing = false;
        auto add = [&](T x) {
            if constexpr (sizeof(T) == 4) kahan_add(ks, kc, x);
            else acc += x;
        };
        for (int a = occ_ptr[lo]; a < occ_ptr[lo + 1]; ++a) {
            const int64_t Ba = occ_blk[a];
            const int la = occ_loc[a];
            for (int b = occ_ptr[hi]; b < occ_ptr[hi + 1]; ++b) {
                const int64_t Bb = occ_blk[b];
                const int lb = occ_loc[b];
                const int64_t B0 = min(Ba, Bb), B1 = max(Ba, Bb);
                const int64_t pos = tri_list[B0 * nblk - B0 * (B0 - 1) / 2 + (B1 - B0)];
                if (pos < 0) {
                    missing = true;
                    continue;
                }
                if (Ba < Bb) {
                    add(P[toff[pos] + (int64_t)la * (L_ptr[Bb + 1] - L_ptr[Bb]) + lb]);
                } else if (Ba > Bb) {
                    add(P[toff[pos] + (int64_t)lb * (L_ptr[Ba + 1] - L_ptr[Ba]) + la]);
                } else {
                    const int64_t nL = L_ptr[Ba + 1] - L_ptr[Ba];
                    add(P[toff[pos] + (int64_t)la * nL + lb]);
                    add(P[toff[pos] + (int64_t)lb * nL + la]);
                }
            }
        }
        if constexpr (sizeof(T) == 4) acc = (double)ks - (double)kc;
        R[r * ldr + j] = missing ? __longlong_as_double(0x7ff8000000000000LL) : negC * acc;
    }
}

// the sparse near-field part added to the representatives' rows (upper entries serve both)
__global__ void add_csr_rows_kernel(int64_t nnz, const int* csr_row, const int* csr_col, const double* val,
                                    const int* red_row, double* R, int64_t ldr) {
    const int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (z >= nnz) return;
    const int64_t i = csr_row[z], j = csr_col[z];
    if (j < i) return;
    const double v = val[z];
    const int ri = red_row[i];
    if (ri >= 0) R[ri * ldr + j] += v;
    if (j != i) {
        const int rj = red_row[j];
        if (rj >= 0) R[rj * ldr + i] += v;
    }
}

// A[r][c] = ((|O_r| / K) sum_{j in O_c} R[r][j] + (|O_c| / K) sum_{i in O_r} R[c][i]) / 2: the
// symmetric part of the row formula for P^T A P / K (bitwise symmetric: both entries add the
// same two terms)
__global__ void fold_sym_kernel(int64_t nred, int K, const int* red_ptr, const int* red_mem, const double* R,
                                int64_t ldr, double* A, int64_t lda) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nred) return;
    for (int64_t r = blockIdx.y; r < nred; r += gridDim.y) {
        double x = 0.0, y = 0.0;
        for (int q = red_ptr[c]; q < red_ptr[c + 1]; ++q) x += R[r * ldr + red_mem[q]];
        for (int q = red_ptr[r]; q < red_ptr[r + 1]; ++q) y += R[c * ldr + red_mem[q]];
        const double sr = (double)(red_ptr[r + 1] - red_ptr[r]) / K, sc = (double)(red_ptr[c + 1] - red_ptr[c]) / K;
        // unfused products and sum, so that (r, c) and (c, r) round alike
        A[r * lda + c] = 0.5 * __dadd_rn(__dmul_rn(sr, x), __dmul_rn(sc, y));
    }
}

// nodal values of a periodic f on the whole mesh from those on the sector
__global__ void expand_nodal_kernel(int64_t nv, int nrhs, const int* sector_of, const double* f, double* fw) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv * nrhs) return;
    const int64_t w = i / nrhs;
    const int c = (int)(i - w * nrhs);
    fw[i] = f[(int64_t)sector_of[w] * nrhs + c];
}

// b[r][c] = (1/K) sum_{i in O_r} bw[i][c]
__global__ void fold_vec_kernel(int64_t nred, int K, int nrhs, const int* red_ptr, const int* red_mem,
                                const double* bw, double* b, int64_t ldb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nred * nrhs) return;
    const int64_t r = i / nrhs;
    const int c = (int)(i - r * nrhs);
    double acc = 0.0;
    for (int q = red_ptr[r]; q < red_ptr[r + 1]; ++q) acc += bw[(int64_t)red_mem[q] * nrhs + c];
    b[r * ldb + c] = acc / K;
}

// ---------------------------------------------------------------- host side --
namespace {

// Host tables bound for one device block: each gets a 256-byte aligned range of it.
struct Uploads {
    struct Item {
        void** dst;
        const void* src;
        size_t bytes;
    };
    std::vector<Item> items;
    template <typename X>
    void add(X*& dst, const std::vector<X>& src) {
        items.push_back({(void**)&dst, src.data(), src.size() * sizeof(X)});
    }
};

// One pooled device block for all tables, filled from one pinned staging buffer by one copy.
int upload_all(fl_ctx* h, const Uploads& U, cudaStream_t st) {
    size_t total = 0;
    for (const auto& it : U.items) total += (std::max<size_t>(it.bytes, 1) + 255) / 256 * 256;
    void* base = nullptr;
    cudaError_t e = pool_dev_alloc(&base, total);
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("device tables: ") + cudaGetErrorString(e));
    h->bufs.push_back({base, total});
    h->ws_bytes += (int64_t)total;
    void* stage = nullptr;
    e = pool_host_alloc(&stage, total);
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("pinned staging: ") + cudaGetErrorString(e));
    size_t off = 0;
    for (const auto& it : U.items) {
        if (it.bytes) std::memcpy((char*)stage + off, it.src, it.bytes);
        *it.dst = (char*)base + off;
        h->h2d_bytes += (int64_t)it.bytes;
        off += (std::max<size_t>(it.bytes, 1) + 255) / 256 * 256;
    }
    e = cudaMemcpyAsync(base, stage, total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    pool_host_free(stage);
    if (e != cudaSuccess) return set_err(h, FL_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
    return FL_OK;
}

int alloc(fl_ctx* h, void** dst, size_t bytes) {
    *dst = nullptr;
    cudaError_t e = pool_dev_alloc(dst, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return set_err(h, FL_ENOMEM, std::string("device workspace: ") + cudaGetErrorString(e));
    h->bufs.push_back({*dst, bytes});
    h->ws_bytes += (int64_t)bytes;
    return FL_OK;
}

// CUDA event pair around stage i when profiling is on
void stage_mark(fl_ctx* h, cudaStream_t st, int i, int end) {
    if (!h->profiling) return;
    if (h->profiling == 2 && i != FL_STAGE_FAR) return;  // the far stage alone, schedule unchanged
    if (!h->ev_made) {
        for (int k = 0; k < 2 * FL_NSTAGES; ++k) cudaEventCreate(&h->ev[k]);
        h->ev_made = true;
    }
    cudaEventRecord(h->ev[2 * i + end], st);
    h->ev_recorded = true;
}

#define FL_TRY(...)                 \
    do {                            \
        int r_ = (__VA_ARGS__);     \
        if (r_ != FL_OK) return r_; \
    } while (0)

int qf_of(const fl_ctx* h) { return h->dim == 1 ? h->opt.k_far : h->opt.k_far * h->opt.k_far; }
int qn_of(const fl_ctx* h) { return h->dim == 1 ? h->opt.k_near : h->opt.k_near * h->opt.k_near; }

int ensure_device(fl_ctx* h, int pi, cudaStream_t st) {
    DevTables& t = h->dev[pi];
    if (t.ready) return FL_OK;
    const Plan& P = h->plan[pi];
    const int D = P.dim, NV = P.nvpc;
    const int64_t nc = P.nc;
    // internal-order geometry
    std::vector<double> cvx(nc * NV * D), cen(nc * D), jac(nc);
    std::vector<int> corner(nc * NV);
    for (int64_t k = 0; k < nc; ++k) {
        const int K = P.perm[k];
        for (int a = 0; a < NV; ++a) {
            const int vtx = P.C[(int64_t)K * NV + a];
            corner[k * NV + a] = vtx;
            for (int d = 0; d < D; ++d) cvx[(k * NV + a) * D + d] = P.V[(int64_t)vtx * D + d];
        }
        for (int d = 0; d < D; ++d) {
            double sacc = 0;
            for (int a = 0; a < NV; ++a) sacc += cvx[(k * NV + a) * D + d];
            cen[k * D + d] = sacc / NV;
        }
        jac[k] = P.jac[K];
    }
    std::vector<int> csr_row(P.csr_col.size());
    for (int64_t i = 0; i < P.n; ++i)
        for (int z = P.csr_ptr[i]; z < P.csr_ptr[i + 1]; ++z) csr_row[z] = (int)i;
    Uploads U;
    U.add(t.V, P.V);
    U.add(t.jac_orig, P.jac);
    U.add(t.F, P.F);
    U.add(t.FN, P.FN);
    U.add(t.FLEN, P.FLEN);
    U.add(t.cvx, cvx);
    U.add(t.cen, cen);
    U.add(t.jac, jac);
    U.add(t.hasdof, P.hasdof);
    U.add(t.loc, P.loc);
    U.add(t.cdof, P.cdof);
    U.add(t.L_ptr, P.L_ptr);
    U.add(t.inc_ptr, P.inc_ptr);
    U.add(t.inc_ent, P.inc_ent);
    U.add(t.occ_ptr, P.occ_ptr);
    U.add(t.occ_blk, P.occ_blk);
    U.add(t.occ_loc, P.occ_loc);
    U.add(t.ex_ptr, P.ex_ptr);
    U.add(t.ex_idx, P.ex_idx);
    U.add(t.np_a, P.np_a);
    U.add(t.np_b, P.np_b);
    U.add(t.enp_ptr, P.enp_ptr);
    U.add(t.enp_ent, P.enp_ent);
    U.add(t.tp_type, P.tp_type);
    U.add(t.tp_vert, P.tp_vert);
    U.add(t.tp_cell, P.tp_cell);
    U.add(t.tp_slot, P.tp_slot);
    U.add(t.ef_ptr, P.ef_ptr);
    U.add(t.ef_fac, P.ef_fac);
    U.add(t.ef_cls, P.ef_cls);
    U.add(t.csr_ptr, P.csr_ptr);
    U.add(t.csr_col, P.csr_col);
    U.add(t.csr_row, csr_row);
    U.add(t.g_ptr, P.g_ptr);
    U.add(t.g_slot, P.g_slot);
    U.add(t.vod, P.vod);
    U.add(t.dov, P.dov);
    U.add(t.corig, corner);
    U.add(t.cells, P.C);
    std::vector<int64_t> v2cp(P.v2c_ptr.begin(), P.v2c_ptr.end());
    U.add(t.v2c_ptr, v2cp);
    U.add(t.v2c, P.v2c);
    std::vector<int> sector_of;
    if (P.sym_K) {
        U.add(t.red_rep, P.red_rep);
        U.add(t.red_ptr, P.red_ptr);
        U.add(t.red_mem, P.red_mem);
        U.add(t.red_row, P.red_row);
        sector_of.assign(P.nv, 0);
        for (int l = 0; l < h->sym_K; ++l)
            for (int64_t v = 0; v < h->sym_nvs; ++v) sector_of[h->sym_vmap[(size_t)l * h->sym_nvs + v]] = (int)v;
        U.add(t.sector_of, sector_of);
    }
    FL_TRY(upload_all(h, U, st));
    const int qf = qf_of(h), qn = qn_of(h);
    FL_TRY(alloc(h, &t.pts, (size_t)nc * qf * D * sizeof(double)));
    if (D == 2 && qn == 36) FL_TRY(alloc(h, &t.pts_near_dw, (size_t)nc * 36 * sizeof(float4)));
    if (D == 2 && qf == 16) {
        FL_TRY(alloc(h, &t.pts_dw, (size_t)nc * 16 * sizeof(float4)));
        const int nch = bnd_dw_chunks(nc);
        if (nch > 1) FL_TRY(alloc(h, (void**)&t.Bfp, (size_t)nch * nc * 16 * sizeof(double)));
    }
    FL_TRY(alloc(h, (void**)&t.Dn, (size_t)P.np_a.size() * 2 * qn * sizeof(double)));
    FL_TRY(alloc(h, (void**)&t.Bf, (size_t)nc * qf * sizeof(double)));
    FL_TRY(alloc(h, (void**)&t.eblk, (size_t)nc * 6 * sizeof(double)));
    FL_TRY(alloc(h, (void**)&t.contrib, (size_t)P.nslots * sizeof(double)));
    FL_TRY(alloc(h, (void**)&t.csr_val, P.csr_col.size() * sizeof(double)));
    FL_TRY(alloc(h, &t.facet_rec, (size_t)std::max<int64_t>(P.nf, 1) * sizeof(FacetRec)));
    if (P.dim == 2 && P.nf > 0) {
        facet_records_kernel<<<(unsigned)((P.nf + 127) / 128), 128, 0, st>>>(P.nf, t.F, t.FN, t.FLEN, t.V,
                                                                             (FacetRec*)t.facet_rec);
        fl::count_launch();
        FL_CUDA_TRY(h, cudaGetLastError());
    }
    t.ready = true;
    return FL_OK;
}

// The dense assembly's tile tables and far-field workspace (every upper-triangle tile of the
// block pairs, its partial blocks and the per-point row sums: O(n^2) memory), separate from
// ensure_device so that the calls that need none of it (the cluster method, the strong form,
// the mass matrix) never allocate it.
int ensure_dense(fl_ctx* h, int pi, cudaStream_t st) {
    DevTables& t = h->dev[pi];
    FL_TRY(ensure_device(h, pi, st));
    if (t.dense_ready) return FL_OK;
    try {
        ensure_plan_tiles(h->plan[pi]);
    } catch (const std::bad_alloc&) {
        return set_err(h, FL_ENOMEM, "out of host memory for the tile list");
    }
    const Plan& P = h->plan[pi];
    Uploads U;
    U.add(t.tiles, P.tiles);
    U.add(t.toff, P.toff);
    if (P.sym_K) U.add(t.tri_list, P.tri_list);
    FL_TRY(upload_all(h, U, st));
    FL_TRY(alloc(h, &t.P, (size_t)P.toff.back() * sizeof(double)));
    FL_TRY(alloc(h, &t.Pd, (size_t)P.nblk * P.nc * qf_of(h) * sizeof(double)));
    t.dense_ready = true;
    return FL_OK;
}

// per-s rule tables, see RuleOffsets
void build_rules(const fl_ctx* h, double s, std::vector<double>& buf, RuleOffsets& ro) {
    const int D = h->dim;
    const fl_options& o = h->opt;
    buf.clear();
    auto put = [&](const std::vector<double>& v) {
        int64_t off = (int64_t)buf.size();
        buf.insert(buf.end(), v.begin(), v.end());
        return off;
    };
    Rule rf = make_rule(D, o.k_far), rn = make_rule(D, o.k_near);
    ro.qf = rf.q;
    ro.qn = rn.q;
    ro.kf = o.k_far;
    ro.kn = o.k_near;
    ro.kt = o.k_touch;
    ro.kb = o.k_bnd;
    ro.far_lam = put(rf.lam);
    ro.far_w = put(rf.w);
    ro.far_phi = put(rf.phi);
    ro.near_lam = put(rn.lam);
    ro.near_w = put(rn.w);
    ro.near_phi = put(rn.phi);
    std::vector<double> t, w;
    gauss01(o.k_far, t, w);
    ro.glf_t = put(t);
    ro.glf_w = put(w);
    gauss01(o.k_near, t, w);
    ro.gln_t = put(t);
    ro.gln_w = put(w);
    std::vector<double> tt, tw;
    gauss01(o.k_touch, tt, tw);
    const int kt = o.k_touch;
    // common edge: four pieces of the l1 directions of (x1-y1, x2, y2)
    {
        std::vector<double> tab;
        for (int piece = 0; piece < 4; ++piece)
            for (int i = 0; i < kt; ++i)
                for (int j = 0; j < kt; ++j) {
                    const double u = tt[i], vv = tt[j], W = tw[i] * tw[j];
                    double w2, w3, jacp, lam, sig;
                    if (piece == 0) { sig = 1; w2 = u / 2; w3 = vv * (1 - w2); jacp = 0.5 * (1 - u / 2); lam = 1 - w2; }
                    else if (piece == 1) { sig = 1; w2 = (1 + u) / 2; w3 = vv * (1 - w2); jacp = 0.25 * (1 - u); lam = w2; }
                    else if (piece == 2) { sig = -1; w3 = u / 2; w2 = vv * (1 - w3); jacp = 0.5 * (1 - u / 2); lam = 1 - w3; }
                    else { sig = -1; w3 = (1 + u) / 2; w2 = vv * (1 - w3); jacp = 0.25 * (1 - u); lam = w3; }
                    const double w1 = sig * (1 - w2 - w3);
                    // dphi over local (P, Q, R, Rt): cz*w1 + cx*w2 + cy*w3
                    tab.push_back(-w1);
                    tab.push_back(w1 - w2 + w3);
                    tab.push_back(w2);
                    tab.push_back(-w3);
                    tab.push_back(w1);
                    tab.push_back(w2);
                    tab.push_back(w3);
                    tab.push_back(W * jacp * std::pow(lam, 2 * s - 3));
                }
        ro.n_edge = 4 * kt * kt;
        ro.t_edge = put(tab);
    }
    // common vertex: two Duffy regions, weight eta2 * w, order k_vertex
    {
        std::vector<double> tab;
        std::vector<double> vt, vw;
        gauss01(o.k_vertex, vt, vw);
        const int kv = o.k_vertex;
        for (int reg = 0; reg < 2; ++reg)
            for (int i = 0; i < kv; ++i)
                for (int j = 0; j < kv; ++j)
                    for (int l = 0; l < kv; ++l) {
                        const double e1 = vt[i], e2 = vt[j], e3 = vt[l], W = vw[i] * vw[j] * vw[l];
                        double x1, x2, y1, y2;
                        if (reg == 0) { x1 = 1; x2 = e1; y1 = e2; y2 = e2 * e3; }
                        else { x1 = e2; x2 = e2 * e3; y1 = 1; y2 = e1; }
                        // local (P, Q, R, Qt, Rt): c1=(eQ-eP), c2=(eR-eQ), c3=-(eQt-eP), c4=-(eRt-eQt)
                        tab.push_back(-x1 + y1);
                        tab.push_back(x1 - x2);
                        tab.push_back(x2);
                        tab.push_back(-y1 + y2);
                        tab.push_back(-y2);
                        tab.push_back(x1);
                        tab.push_back(x2);
                        tab.push_back(y1);
                        tab.push_back(y2);
                        tab.push_back(W * e2);
                    }
        ro.n_vert = 2 * kv * kv * kv;
        ro.t_vert = put(tab);
    }
    // 1D common vertex
    {
        std::vector<double> tab;
        for (int i = 0; i < kt; ++i) {
            tab.push_back(tt[i]);
            tab.push_back(tw[i]);
        }
        ro.n_1d = kt;
        ro.t_1d = put(tab);
    }
    // identical pair: three angular pieces of [0, pi), 2 k_touch points each, weight x rho^{2-2s}
    {
        std::vector<double> tab;
        std::vector<double> it, iw;
        gauss01(2 * kt, it, iw);
        const double pi = 3.14159265358979323846;
        const double lo[3] = {0.0, pi / 2, 3 * pi / 4}, hi[3] = {pi / 2, 3 * pi / 4, pi};
        for (int piece = 0; piece < 3; ++piece)
            for (int i = 0; i < 2 * kt; ++i) {
                const double th = lo[piece] + (hi[piece] - lo[piece]) * it[i];
                const double wt = (hi[piece] - lo[piece]) * iw[i];
                const double u0 = std::cos(th), u1 = std::sin(th);
                const double rho = 2.0 / (std::fabs(u0 + u1) + std::fabs(u0) + std::fabs(u1));
                tab.push_back(u0);
                tab.push_back(u1);
                tab.push_back(wt * std::pow(rho, 2 - 2 * s));
            }
        ro.n_ident = 3 * 2 * kt;
        ro.t_ident = put(tab);
    }
    std::vector<double> bt, bw;
    gauss01(o.k_bnd, bt, bw);
    const int kb = o.k_bnd;
    // boundary, facet is an edge of K: three pieces, weight x lambda^{2s-3}
    {
        std::vector<double> tab;
        const double lo[3] = {0.0, 0.5, 0.0}, hi[3] = {0.5, 1.0, 1.0};
        for (int piece = 0; piece < 3; ++piece)
            for (int i = 0; i < kb; ++i) {
                const double om = lo[piece] + (hi[piece] - lo[piece]) * bt[i];
                const double wt = (hi[piece] - lo[piece]) * bw[i];
                const double sig = (piece == 2) ? -1.0 : 1.0;
                const double lam = (piece == 0) ? 1 - om : (piece == 1 ? om : 1.0);
                tab.push_back(sig * (1 - om));
                tab.push_back(om);
                tab.push_back(wt * std::pow(lam, 2 * s - 3));
            }
        ro.n_own = 3 * kb;
        ro.b_own = put(tab);
    }
    // boundary, facet and K share a vertex: two Duffy regions of K x e
    {
        std::vector<double> tab;
        for (int reg = 0; reg < 2; ++reg)
            for (int i = 0; i < kb; ++i)
                for (int j = 0; j < kb; ++j) {
                    const double u = bt[i], vv = bt[j], W = bw[i] * bw[j];
                    if (reg == 0) { tab.push_back(1.0); tab.push_back(u); tab.push_back(vv); tab.push_back(W); }
                    else { tab.push_back(u); tab.push_back(u * vv); tab.push_back(1.0); tab.push_back(W * u); }
                }
        ro.n_bvert = 2 * kb * kb;
        ro.b_vert = put(tab);
    }
}

int pw_mode(int dim, double s) {
    const double e4 = -2.0 * (dim + 2.0 * s);  // 4e
    const double r = std::round(e4);
    if (std::fabs(e4 - r) > 1e-12) return 0;
    const int m = -(int)r;
    return (m >= 3 && m <= 7) ? m : 0;
}

template <int D, typename T, int Q, int PW>
int launch_far_t(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro,
                 double expo, int64_t ntiles, cudaStream_t st) {
    constexpr int NV = D + 1;
    FarRule<T, Q, NV> R;
    for (int a = 0; a < Q; ++a) {
        R.w[a] = (T)rb[ro.far_w + a];
        for (int v = 0; v < NV; ++v) R.wphi[a * NV + v] = (T)(rb[ro.far_w + a] * rb[ro.far_phi + a * NV + v]);
    }
    for (int a = 0; a < Q; ++a)
        for (int v = 0; v < NV; ++v) R.wpair[((a / 2) * NV + v) * 2 + (a % 2)] = R.wphi[a * NV + v];
    FarArgs<T> A;
    A.cen = t.cen;
    A.pts = (const T*)t.pts;
    A.jac = t.jac;
    A.hasdof = t.hasdof;
    A.loc = t.loc;
    A.ex_ptr = t.ex_ptr;
    A.ex_idx = t.ex_idx;
    A.tiles = t.tiles;
    A.toff = t.toff;
    A.L_ptr = t.L_ptr;
    A.inc_ptr = t.inc_ptr;
    A.inc_ent = t.inc_ent;
    A.P = (T*)t.P;
    A.Pd = (T*)t.Pd;
    A.nc = P.nc;
    A.nblk = P.nblk;
    A.expo = (T)expo;
    const int maxL = std::max(1, P.maxL);
    size_t smem = 32 * D * sizeof(double) + 32 * sizeof(double) + 32 * Q * (Q == 16 ? 1 : D) * sizeof(T) + 32 * Q * sizeof(T) +
                  (size_t)NV * maxL * 32 * sizeof(T) + 32 * NV * sizeof(int) + 32 * sizeof(int);
    auto kern = far_tile_kernel<D, T, Q, PW>;
    FL_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ntiles > 0) {
        kern<<<(unsigned)ntiles, 32, smem, st>>>(A, R, maxL);
        fl::count_launch();
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

template <int D, typename T, int Q>
int launch_far_q(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro,
                 double expo, int pw, int64_t nt, cudaStream_t st) {
    // specialised square-root forms only for the default orders (k_far = 4)
    if constexpr (D == 2 && Q == 16) {
        switch (pw) {
            case 5: return launch_far_t<D, T, Q, 5>(h, P, t, rb, ro, expo, nt, st);
            case 6: return launch_far_t<D, T, Q, 6>(h, P, t, rb, ro, expo, nt, st);
            case 7: return launch_far_t<D, T, Q, 7>(h, P, t, rb, ro, expo, nt, st);
            default: break;
        }
    } else if constexpr (D == 1 && Q == 4) {
        switch (pw) {
            case 3: return launch_far_t<D, T, Q, 3>(h, P, t, rb, ro, expo, nt, st);
            case 4: return launch_far_t<D, T, Q, 4>(h, P, t, rb, ro, expo, nt, st);
            case 5: return launch_far_t<D, T, Q, 5>(h, P, t, rb, ro, expo, nt, st);
            default: break;
        }
    }
    return launch_far_t<D, T, Q, 0>(h, P, t, rb, ro, expo, nt, st);
}

template <typename T>
int launch_far(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro,
               double expo, int pw, cudaStream_t st, int64_t ntiles = -1) {
    const int k = h->opt.k_far;
    const int64_t nt = ntiles >= 0 ? ntiles : (int64_t)P.tiles.size() / 2;
    if (P.dim == 2) {
        switch (k) {
            case 3: return launch_far_q<2, T, 9>(h, P, t, rb, ro, expo, pw, nt, st);
            case 4: return launch_far_q<2, T, 16>(h, P, t, rb, ro, expo, pw, nt, st);
            case 5: return launch_far_q<2, T, 25>(h, P, t, rb, ro, expo, pw, nt, st);
            case 6: return launch_far_q<2, T, 36>(h, P, t, rb, ro, expo, pw, nt, st);
            default: break;
        }
    } else {
        switch (k) {
            case 2: return launch_far_q<1, T, 2>(h, P, t, rb, ro, expo, pw, nt, st);
            case 3: return launch_far_q<1, T, 3>(h, P, t, rb, ro, expo, pw, nt, st);
            case 4: return launch_far_q<1, T, 4>(h, P, t, rb, ro, expo, pw, nt, st);
            case 5: return launch_far_q<1, T, 5>(h, P, t, rb, ro, expo, pw, nt, st);
            case 6: return launch_far_q<1, T, 6>(h, P, t, rb, ro, expo, pw, nt, st);
            case 8: return launch_far_q<1, T, 8>(h, P, t, rb, ro, expo, pw, nt, st);
            default: break;
        }
    }
    return set_err(h, FL_ENOTIMPL, "k_far not compiled for this dimension (2D: 3-6, 1D: 2-6, 8)");
}

template <typename T, int Q>
int launch_bnd_q(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, double expo, int pw, cudaStream_t st) {
    const unsigned nb = (unsigned)((P.nc + 31) / 32);
    const FacetRec* FR = (const FacetRec*)t.facet_rec;
#define FL_BND(PWV)                                                                                                  \
    bnd_far_kernel<T, Q, PWV><<<nb, 32 * BND_WARPS, 0, st>>>(P.nc, P.nf, t.cen, (const T*)t.pts, t.hasdof, t.ef_ptr, \
                                                              t.ef_fac, FR, nullptr, t.rule, ro, (T)expo, t.Bf)
    if (Q == 16 && pw == 6) FL_BND(6);
    else if (Q == 16 && pw == 5) FL_BND(5);
    else if (Q == 16 && pw == 7) FL_BND(7);
    else FL_BND(0);
#undef FL_BND
    fl::count_launch();
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

template <typename T>
int launch_bnd(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, double expo, int pw, cudaStream_t st) {
    switch (h->opt.k_far) {
        case 3: return launch_bnd_q<T, 9>(h, P, t, ro, expo, pw, st);
        case 4: return launch_bnd_q<T, 16>(h, P, t, ro, expo, pw, st);
        case 5: return launch_bnd_q<T, 25>(h, P, t, ro, expo, pw, st);
        case 6: return launch_bnd_q<T, 36>(h, P, t, ro, expo, pw, st);
        default: return set_err(h, FL_ENOTIMPL, "k_far not compiled");
    }
}

template <int D, typename T, int QN, int PW>
int launch_near_fast_t(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro,
                       double expo, double C, cudaStream_t st) {
    constexpr int NV = D + 1;
    NearRule<T, QN, D> R;
    for (int a = 0; a < QN; ++a) {
        for (int d = 0; d < D; ++d) R.lam[a * D + d] = (T)rb[ro.near_lam + a * D + d];
        R.w[a] = (T)rb[ro.near_w + a];
        for (int v = 0; v < NV; ++v) R.wphi[a * NV + v] = (T)(rb[ro.near_w + a] * rb[ro.near_phi + a * NV + v]);
    }
    const int nnear = (int)P.np_a.size();
    near_pair_fast<D, T, PW, QN><<<(unsigned)((nnear + 63) / 64), 64, 0, st>>>(nnear, t.np_a, t.np_b, t.cvx, t.cen,
                                                                                t.jac, R, (T)expo, C, t.contrib,
                                                                                P.np_slot0, t.Dn);
    fl::count_launch();
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

template <int D, typename T, int QN>
int launch_near_fast(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro,
                     double expo, int pw, double C, cudaStream_t st) {
    if constexpr (D == 2) {
        if (pw == 6) return launch_near_fast_t<D, T, QN, 6>(h, P, t, rb, ro, expo, C, st);
        if constexpr (sizeof(T) == 8) {
            if (pw == 5) return launch_near_fast_t<D, T, QN, 5>(h, P, t, rb, ro, expo, C, st);
            if (pw == 7) return launch_near_fast_t<D, T, QN, 7>(h, P, t, rb, ro, expo, C, st);
        }
    } else {
        if (pw == 4) return launch_near_fast_t<D, T, QN, 4>(h, P, t, rb, ro, expo, C, st);
        if constexpr (sizeof(T) == 8) {
            if (pw == 3) return launch_near_fast_t<D, T, QN, 3>(h, P, t, rb, ro, expo, C, st);
            if (pw == 5) return launch_near_fast_t<D, T, QN, 5>(h, P, t, rb, ro, expo, C, st);
        }
    }
    return launch_near_fast_t<D, T, QN, 0>(h, P, t, rb, ro, expo, C, st);
}

}  // namespace

// C(d,s) = 2^{2s} s Γ(s + d/2) / (π^{d/2} Γ(1 - s)), Section 2.
static double frac_constant(int d, double s) {
    const double pi = 3.14159265358979323846;
    return std::pow(2.0, 2 * s) * s * std::tgamma(s + d / 2.0) / (std::pow(pi, d / 2.0) * std::tgamma(1.0 - s));
}

// Output of the near-field CSR route (caller's device arrays).
struct CsrOut {
    int32_t* rowptr;
    int32_t* col;
    double* val;
};

// Near separated pairs (vertex-graph distance 1): off-diagonal blocks (times -C) into the
// contribution slots, per-point row sums of both cells into Dn.
static int launch_near_pairs(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb,
                             const RuleOffsets& ro, double expo, int pw, bool f32, double C, cudaStream_t st) {
    const int D = P.dim;
    const int pw32 = (pw == 4 || pw == 6) ? pw : 0;
    const int nnear = (int)P.np_a.size();
    const bool near_fast = (D == 2 && ro.qn == 36) || (D == 1 && ro.qn == 6);
    if (nnear > 0 && !f32 && near_dw_applies(h, P, pw)) {
        FL_TRY(launch_near_dw(h, P, t, rb, ro, pw, C, st));
    } else if (nnear > 0 && near_fast) {
        if (D == 2) {
            if (f32) FL_TRY(launch_near_fast<2, float, 36>(h, P, t, rb, ro, expo, pw32, C, st));
            else FL_TRY(launch_near_fast<2, double, 36>(h, P, t, rb, ro, expo, pw, C, st));
        } else {
            if (f32) FL_TRY(launch_near_fast<1, float, 6>(h, P, t, rb, ro, expo, pw32, C, st));
            else FL_TRY(launch_near_fast<1, double, 6>(h, P, t, rb, ro, expo, pw, C, st));
        }
    } else if (nnear > 0) {
        const unsigned g = (unsigned)((nnear + 63) / 64);
#define FL_NEAR(DD, TT, PWV)                                                                                    \
    near_pair_kernel<DD, TT, PWV><<<g, 64, 0, st>>>(nnear, t.np_a, t.np_b, t.cvx, t.cen, t.jac, t.rule, ro, (TT)expo, \
                                                    C, t.contrib, P.np_slot0, t.Dn)
        if (D == 2) {
            if (f32) { if (pw == 6) FL_NEAR(2, float, 6); else FL_NEAR(2, float, 0); }
            else { if (pw == 5) FL_NEAR(2, double, 5); else if (pw == 6) FL_NEAR(2, double, 6); else if (pw == 7) FL_NEAR(2, double, 7); else FL_NEAR(2, double, 0); }
        } else {
            if (f32) { if (pw == 4) FL_NEAR(1, float, 4); else FL_NEAR(1, float, 0); }
            else { if (pw == 3) FL_NEAR(1, double, 3); else if (pw == 4) FL_NEAR(1, double, 4); else if (pw == 5) FL_NEAR(1, double, 5); else FL_NEAR(1, double, 0); }
        }
#undef FL_NEAR
        fl::count_launch();
        FL_CUDA_TRY(h, cudaGetLastError());
    }
    return FL_OK;
}

// Touching pairs (common edge / common vertex), one warp each, full blocks into their slots.
static int launch_touch_pairs(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, double s, double C,
                              int pw, bool f32, cudaStream_t st) {
    const int D = P.dim;
    const int ntp = (int)P.tp_type.size();
    if (ntp == 0) return FL_OK;
    if (!f32 && touch_dw_applies(h, P, pw)) return launch_touch_dw(h, P, t, ro, s, C, pw, st);
    const unsigned g = (unsigned)(((int64_t)ntp * 32 + 127) / 128);  // one warp per pair
#define FL_TOUCH(TT, RULE, PWV) \
    touch_pair_kernel<TT, PWV><<<g, 128, 0, st>>>(ntp, D, t.tp_type, t.tp_vert, t.tp_cell, t.tp_slot, t.V, t.jac_orig, RULE, ro, s, C, t.contrib)
    if (f32) {
        if (D == 2 && pw == 6) FL_TOUCH(float, t.rule32, 6);
        else FL_TOUCH(float, t.rule32, 0);
    } else if (D == 2 && pw == 5) FL_TOUCH(double, t.rule, 5);
    else if (D == 2 && pw == 6) FL_TOUCH(double, t.rule, 6);
    else if (D == 2 && pw == 7) FL_TOUCH(double, t.rule, 7);
    else FL_TOUCH(double, t.rule, 0);
#undef FL_TOUCH
    fl::count_launch();
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

static ElemArgs elem_args(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, double s, double C, bool f32) {
    ElemArgs E;
    E.dim = P.dim;
    E.nc = P.nc;
    E.nblk = P.nblk;
    E.nf = P.nf;
    E.nnear = (int64_t)P.np_a.size();
    E.cvx = t.cvx;
    E.cen = t.cen;
    E.jac = t.jac;
    E.hasdof = t.hasdof;
    E.Pd = t.Pd;
    E.pd_is_float = f32 ? 1 : 0;
    E.Dn = t.Dn;
    E.enp_ptr = t.enp_ptr;
    E.enp_ent = t.enp_ent;
    E.Bf = t.Bf;
    E.ef_ptr = t.ef_ptr;
    E.ef_fac = t.ef_fac;
    E.ef_cls = t.ef_cls;
    E.F = t.F;
    E.FN = t.FN;
    E.FLEN = t.FLEN;
    E.V = t.V;
    E.corner = t.corig;
    E.rule = t.rule;
    E.C2s = C / (2.0 * s);
    E.r2s = 1.0 / (2.0 - 2.0 * s);
    E.r3s = 1.0 / (3.0 - 2.0 * s);
    E.r4s = 1.0 / (4.0 - 2.0 * s);
    E.rule32 = f32 ? t.rule32 : nullptr;
    E.ro = ro;
    E.s = s;
    E.C = C;
    E.regional = h->opt.regional;
    E.contrib = t.contrib;
    E.slot0 = P.el_slot0;
    E.eblk = t.eblk;
    E.cluster = 0;
    return E;
}

// One warp per cell; part 1 (far-independent) or part 2 (the diagonal block into its slots).
static int launch_element(fl_ctx* h, const ElemArgs& E, int pw, int part, cudaStream_t st) {
    const int D = E.dim;
    const unsigned ge = (unsigned)((E.nc * 32 + 127) / 128);
    auto go = [&](auto pt) {
        constexpr int PT = decltype(pt)::value;
        if (D == 2 && pw == 5) element_kernel<5, 2, PT><<<ge, 128, 0, st>>>(E);
        else if (D == 2 && pw == 6) element_kernel<6, 2, PT><<<ge, 128, 0, st>>>(E);
        else if (D == 2 && pw == 7) element_kernel<7, 2, PT><<<ge, 128, 0, st>>>(E);
        else if (D == 2) element_kernel<0, 2, PT><<<ge, 128, 0, st>>>(E);
        else element_kernel<0, 1, PT><<<ge, 128, 0, st>>>(E);
    };
    if (E.nc > 0) {
        if (part == 1) go(std::integral_constant<int, 1>{});
        else go(std::integral_constant<int, 2>{});
        fl::count_launch();
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

// The handle's second stream and its fork / join / far events, created on first use; false
// when they cannot be had (the stages then run in sequence on the caller's stream).
static bool side_stream(fl_ctx* h) {
    if (!h->side && cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->side = nullptr;
    }
    if (h->side && !h->ev_fork) {
        if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_far, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (h->ev_fork) cudaEventDestroy(h->ev_fork);
            if (h->ev_join) cudaEventDestroy(h->ev_join);
            h->ev_fork = h->ev_join = h->ev_far = nullptr;
        }
    }
    return h->side && h->ev_fork && h->ev_join && h->ev_far;
}

// Per-s rule tables on the device, built and uploaded once per (handle, plan, s): repeated
// calls at the same s do no host work and no host-synchronising copy.  f32: also the float32
// copy (mixed-mode touching pairs and identical pair).
static int ensure_rules(fl_ctx* h, DevTables& t, double s, bool f32, cudaStream_t st) {
    if (!(t.rule_s == s)) {
        t.rule_s = std::nan("");
        t.rule32_ready = false;
        build_rules(h, s, t.rule_host, t.rule_ro);
        if (t.rule_ro.qn > MAXQ_NEAR) return set_err(h, FL_ENOTIMPL, "k_near too large");
        const std::vector<double>& rb = t.rule_host;
        if (t.rule_len < rb.size()) {
            void* p = nullptr;
            FL_TRY(alloc(h, &p, rb.size() * sizeof(double)));
            t.rule = (double*)p;
            t.rule_len = rb.size();
        }
        FL_CUDA_TRY(h, cudaMemcpyAsync(t.rule, rb.data(), rb.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        // double-word copy (high float, float of the remainder)
        if (t.rule_dw_len < rb.size()) {
            void* p = nullptr;
            FL_TRY(alloc(h, &p, rb.size() * sizeof(float2)));
            t.rule_dw = p;
            t.rule_dw_len = rb.size();
        }
        std::vector<float2> rdw(rb.size());
        for (size_t i = 0; i < rb.size(); ++i) {
            const float hi = (float)rb[i];
            rdw[i] = make_float2(hi, (float)(rb[i] - (double)hi));
        }
        FL_CUDA_TRY(h, cudaMemcpyAsync(t.rule_dw, rdw.data(), rdw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        FL_CUDA_TRY(h, cudaStreamSynchronize(st));  // the staging vector is freed on return
        t.rule_s = s;
    }
    if (f32 && !t.rule32_ready) {
        const std::vector<double>& rb = t.rule_host;
        if (t.rule32_len < rb.size()) {
            void* p = nullptr;
            FL_TRY(alloc(h, &p, rb.size() * sizeof(float)));
            t.rule32 = (float*)p;
            t.rule32_len = rb.size();
        }
        const std::vector<float> rb32(rb.begin(), rb.end());
        FL_CUDA_TRY(h, cudaMemcpyAsync(t.rule32, rb32.data(), rb32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        t.rule32_ready = true;
    }
    return FL_OK;
}

static int assemble_impl(fl_ctx* h, double s, int precision, double* A, int64_t lda, const CsrOut* csr,
                         cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    const bool sym = P.sym_K > 0;
    if (!csr) {
        if (lda < (sym ? P.n_red : P.n)) return set_err(h, FL_EINVAL, "lda < n");
        if (!A) return set_err(h, FL_EINVAL, "A is NULL");
    }
    if (precision != FL_FP64 && precision != FL_MIXED) return set_err(h, FL_EINVAL, "unknown precision");
    if (P.dim == 2 && P.paper_all && !h->opt.regional)
        return set_err(h, FL_ENOTIMPL, "2D boundary DOFs (FL_DOF_PAPER with s < 1/2) are not implemented");
    FL_CUDA_TRY(h, cudaSetDevice(h->device));
    FL_TRY(ensure_dense(h, pi, st));
    DevTables& t = h->dev[pi];
    const int D = P.dim;
    const bool f32 = precision == FL_MIXED;
    FL_TRY(ensure_rules(h, t, s, f32, st));
    const std::vector<double>& rb = t.rule_host;
    const RuleOffsets& ro = t.rule_ro;
    const double C = frac_constant(D, s);
    const double expo = -(D + 2.0 * s) / 2.0;
    const int pw = pw_mode(D, s);
    const int64_t nc = P.nc;
    const unsigned gb = (unsigned)((nc + 127) / 128);
    // symmetry reduction: the representatives' rows R (n_red x n) in the handle's workspace; the
    // row sums of tiles left out stay zero (they belong to cells of no representative)
    double* R = nullptr;
    const int64_t ldr = (P.n + 3) / 4 * 4;
    if (sym) {
        const size_t need = (size_t)std::max<int64_t>(P.n_red, 1) * ldr * sizeof(double);
        if (need > h->sym_ws_bytes) {
            if (h->sym_ws) {
                FL_CUDA_TRY(h, cudaStreamSynchronize(st));
                pool_dev_free(h->sym_ws);
                h->sym_ws = nullptr;
                h->sym_ws_bytes = 0;
            }
            if (pool_dev_alloc(&h->sym_ws, need) != cudaSuccess) {
                cudaGetLastError();
                return set_err(h, FL_ENOMEM, "reduced-assembly workspace");
            }
            h->sym_ws_bytes = need;
        }
        R = (double*)h->sym_ws;
        FL_CUDA_TRY(h, cudaMemsetAsync(t.Pd, 0, (size_t)P.nblk * nc * qf_of(h) * sizeof(double), st));
    }
    // far rule offsets
    stage_mark(h, st, FL_STAGE_PREP, 0);
    if (D == 2) {
        if (f32) { prep_points<float, 2><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (float*)t.pts); fl::count_launch(); }
        else { prep_points<double, 2><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (double*)t.pts); fl::count_launch(); }
        if (!f32 && far_dw_applies(h, P, pw)) FL_TRY(prep_far_dw(h, P, t, ro, st));
    } else {
        if (f32) { prep_points<float, 1><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (float*)t.pts); fl::count_launch(); }
        else { prep_points<double, 1><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (double*)t.pts); fl::count_launch(); }
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    stage_mark(h, st, FL_STAGE_PREP, 1);
    // Two streams: the near, touching and boundary stages read only the tables and the far rule
    // offsets and write their own buffers (contribution slots, Dn, Bf), so they run on the
    // handle's second stream while the far-field stage runs here; their blocks fill the SMs the
    // far kernel leaves idle (its last wave, spare registers).  The element kernel (which adds
    // the far row sums) and the sparse gather follow on the second stream once the far stage is
    // done, while the dense far-field compose runs here; the streams join before the sparse part
    // is added.  With profiling on every stage runs on the caller's stream, one after another,
    // so that each event pair brackets one stage alone.
    cudaStream_t sst = st;
    if (h->profiling != 1 && side_stream(h)) {
        FL_CUDA_TRY(h, cudaEventRecord(h->ev_fork, st));
        FL_CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        sst = h->side;
    }
    // far field (launched first: it takes the SMs, the second stream's blocks fill in behind it)
    stage_mark(h, st, FL_STAGE_FAR, 0);
    // float32: keep only the one-MUFU forms (t^2, t^3); lg2 + ex2 beats rsqrt + sqrt here
    const int pw32 = (pw == 4 || pw == 6) ? pw : 0;
    if (f32) FL_TRY(launch_far<float>(h, P, t, rb, ro, expo, pw32, st));
    else if (far_dw_applies(h, P, pw)) FL_TRY(launch_far_dw(h, P, t, rb, ro, pw, st));
    else FL_TRY(launch_far<double>(h, P, t, rb, ro, expo, pw, st));
    stage_mark(h, st, FL_STAGE_FAR, 1);
    int side_rc = FL_OK;
    const int64_t nnz = (int64_t)P.csr_col.size();
    {
        // the stages of the second stream; on an error the join below still runs, so that the
        // caller's stream never runs ahead of work left on the second stream
        const cudaStream_t h_st = st;
        auto run_side = [&]() -> int {
            const cudaStream_t st = sst;
            stage_mark(h, st, FL_STAGE_NEAR, 0);
            FL_TRY(launch_near_pairs(h, P, t, rb, ro, expo, pw, f32, C, st));
            stage_mark(h, st, FL_STAGE_NEAR, 1);
            // touching pairs (float64; float32 in the mixed mode)
            stage_mark(h, st, FL_STAGE_TOUCH, 0);
            FL_TRY(launch_touch_pairs(h, P, t, ro, s, C, pw, f32, st));
            stage_mark(h, st, FL_STAGE_TOUCH, 1);
            // boundary term over far facets (2D)
            stage_mark(h, st, FL_STAGE_BND, 0);
            if (D == 2 && !h->opt.regional && P.nf > 0) {
                if (f32) FL_TRY(launch_bnd<float>(h, P, t, ro, expo, pw32, st));
                else if (far_dw_applies(h, P, pw)) FL_TRY(launch_bnd_dw(h, P, t, rb, ro, pw, st));
                else FL_TRY(launch_bnd<double>(h, P, t, ro, expo, pw, st));
            }
            stage_mark(h, st, FL_STAGE_BND, 1);
            // per element: the far-independent part now (beside the far tile kernel), the part
            // that adds the far field's per-point row sums once the far stage is done
            stage_mark(h, st, FL_STAGE_ELEMENT, 0);
            {
                const ElemArgs E = elem_args(h, P, t, ro, s, C, f32);
                FL_TRY(launch_element(h, E, pw, 1, st));
                if (sst != h_st) {
                    FL_CUDA_TRY(h, cudaEventRecord(h->ev_far, h_st));
                    FL_CUDA_TRY(h, cudaStreamWaitEvent(sst, h->ev_far, 0));
                }
                FL_TRY(launch_element(h, E, pw, 2, st));
            }
            stage_mark(h, st, FL_STAGE_ELEMENT, 1);
            // sparse near-field values
            stage_mark(h, st, FL_STAGE_COMPOSE, 0);
            if (nnz > 0) {
                gather_csr_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, t.csr_row, t.csr_col, t.g_ptr,
                                                                                 t.g_slot, t.contrib, t.csr_val);
                fl::count_launch();
                FL_CUDA_TRY(h, cudaGetLastError());
            }
            return FL_OK;
        };
        // the dense far-field part reads only the far stage's partial tiles: it runs here while the
        // element and gather kernels run on the second stream
        auto run_compose = [&]() -> int {
            if (sym) {
                const dim3 grid((unsigned)((P.n + 255) / 256), (unsigned)std::min<int64_t>(std::max<int64_t>(P.n_red, 1), 65535));
                if (f32)
                    compose_rows_kernel<float><<<grid, 256, 0, st>>>(P.n, P.n_red, P.nblk, t.red_rep, t.occ_ptr,
                                                                     t.occ_blk, t.occ_loc, t.L_ptr, t.tri_list, t.toff,
                                                                     (const float*)t.P, -C, R, ldr);
                else
                    compose_rows_kernel<double><<<grid, 256, 0, st>>>(P.n, P.n_red, P.nblk, t.red_rep, t.occ_ptr,
                                                                      t.occ_blk, t.occ_loc, t.L_ptr, t.tri_list, t.toff,
                                                                      (const double*)t.P, -C, R, ldr);
                fl::count_launch();
                FL_CUDA_TRY(h, cudaGetLastError());
                return FL_OK;
            }
            const int64_t nt = (P.n + 31) / 32;
            const unsigned grid = (unsigned)(nt * (nt + 1) / 2);  // upper-triangle 32 x 32 tiles
            if (f32)
                compose_far_kernel<float><<<grid, 256, 0, st>>>(P.n, P.nblk, t.occ_ptr, t.occ_blk, t.occ_loc, t.L_ptr,
                                                                t.toff, (const float*)t.P, -C, A, lda);
            else
                compose_far_kernel<double><<<grid, 256, 0, st>>>(P.n, P.nblk, t.occ_ptr, t.occ_blk, t.occ_loc, t.L_ptr,
                                                                 t.toff, (const double*)t.P, -C, A, lda);
            fl::count_launch();
            FL_CUDA_TRY(h, cudaGetLastError());
            return FL_OK;
        };
        side_rc = run_side();
        if (side_rc == FL_OK && !csr) side_rc = run_compose();
        if (sst != st) {
            FL_CUDA_TRY(h, cudaEventRecord(h->ev_join, sst));
            FL_CUDA_TRY(h, cudaStreamWaitEvent(st, h->ev_join, 0));
        }
    }
    if (side_rc != FL_OK) return side_rc;
    if (csr) {  // the near-field part alone: pattern and full symmetric values
        if (nnz > 0) {
            csr_full_values_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, t.csr_ptr, t.csr_row, t.csr_col,
                                                                                t.csr_val, csr->val); fl::count_launch();
            FL_CUDA_TRY(h, cudaGetLastError());
            FL_CUDA_TRY(h, cudaMemcpyAsync(csr->col, t.csr_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        }
        FL_CUDA_TRY(h, cudaMemcpyAsync(csr->rowptr, t.csr_ptr, (P.n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        stage_mark(h, st, FL_STAGE_COMPOSE, 1);
        return FL_OK;
    }
    if (sym) {
        if (nnz > 0) {
            add_csr_rows_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, t.csr_row, t.csr_col, t.csr_val,
                                                                               t.red_row, R, ldr);
            fl::count_launch();
        }
        if (P.n_red > 0) {
            const dim3 grid((unsigned)((P.n_red + 127) / 128), (unsigned)std::min<int64_t>(P.n_red, 65535));
            fold_sym_kernel<<<grid, 128, 0, st>>>(P.n_red, P.sym_K, t.red_ptr, t.red_mem, R, ldr, A, lda);
            fl::count_launch();
        }
        FL_CUDA_TRY(h, cudaGetLastError());
        stage_mark(h, st, FL_STAGE_COMPOSE, 1);
        return FL_OK;
    }
    if (nnz > 0) {
        add_csr_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, t.csr_row, t.csr_col, t.csr_val, A, lda); fl::count_launch();
        FL_CUDA_TRY(h, cudaGetLastError());
    }
    stage_mark(h, st, FL_STAGE_COMPOSE, 1);
    return FL_OK;
}

int ensure_device_tables(fl_ctx* h, int pi, cudaStream_t st) { return ensure_device(h, pi, st); }

int assemble(fl_ctx* h, double s, int precision, double* A, int64_t lda, cudaStream_t st) {
    return assemble_impl(h, s, precision, A, lda, nullptr, st);
}

// Sweep the launch variants of the float64-mode double-word far kernel on this handle's
// mesh at order s: for each, one warm-up assembly and `reps` profiled ones (stages in
// sequence, the far stage timed alone by CUDA events); the median decides.  The winner is
// recorded in the tuning table under (kernel, cell count), which later assemblies consult.
// The near field of the cluster method from local computations (Section 6): the tiles the
// near-field entries touch (separated pairs at distance >= 2, the off-diagonal blocks only),
// near and touching pairs as in the dense assembly, the diagonal blocks with the integral over
// the boundary of N(K) in place of the far pairs' and the boundary facets' part (element
// kernel, cluster mode), and the entries composed from these.  Float64 (double-word far pairs
// where the dense float64 mode takes them).  No O(n^2) table or workspace is touched.
int assemble_hnear(fl_ctx* h, int pi, double s, int precision, const HNearDev& q, int64_t nnz, const int* nz_row,
                   const int* nz_col, double* nz_val, cudaStream_t st) {
    const Plan& P = h->plan[pi];
    if (precision != FL_FP64 && precision != FL_MIXED) return set_err(h, FL_EINVAL, "unknown precision");
    const bool f32 = precision == FL_MIXED;
    if (P.sym_K) return sym_unsupported(h, "the cluster method's near-field assembly");
    if (h->opt.regional) return set_err(h, FL_ENOTIMPL, "the near-field assembly needs the boundary term (not regional)");
    if (P.dim == 2 && P.paper_all) return set_err(h, FL_ENOTIMPL, "2D boundary DOFs are not implemented");
    FL_CUDA_TRY(h, cudaSetDevice(h->device));
    FL_TRY(ensure_device(h, pi, st));
    FL_TRY(ensure_rules(h, h->dev[pi], s, f32, st));
    DevTables t = h->dev[pi];  // the mesh tables, with this assembly's tiles, facets and workspace
    t.tiles = q.tiles;
    t.toff = q.toff;
    t.tile_rowmask = q.rowmask;
    t.P = q.P;
    t.Pd = nullptr;
    t.ef_ptr = q.ef_ptr;
    t.ef_fac = q.ef_fac;
    t.ef_cls = q.ef_cls;
    t.F = q.F;
    t.FN = q.FN;
    t.FLEN = q.FLEN;
    const std::vector<double>& rb = t.rule_host;
    const RuleOffsets& ro = t.rule_ro;
    const int D = P.dim;
    const double C = frac_constant(D, s);
    const double expo = -(D + 2.0 * s) / 2.0;
    const int pw = pw_mode(D, s);
    const int64_t nc = P.nc;
    const unsigned gb = (unsigned)((nc + 127) / 128);
    if (nc > 0) {
        if (f32) {
            if (D == 2) prep_points<float, 2><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (float*)t.pts);
            else prep_points<float, 1><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (float*)t.pts);
        } else {
            if (D == 2) prep_points<double, 2><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (double*)t.pts);
            else prep_points<double, 1><<<gb, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, ro.qf, nc, (double*)t.pts);
        }
        fl::count_launch();
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    const int pw32 = (pw == 4 || pw == 6) ? pw : 0;
    const bool dw = !f32 && D == 2 && far_dw_applies(h, P, pw);
    if (dw) FL_TRY(prep_far_dw(h, P, t, ro, st));
    // the local pairs and the cell blocks on the second stream, beside the tiles (they share no
    // buffer with them); the streams join before the entries are composed
    cudaStream_t sst = st;
    if (h->profiling != 1 && side_stream(h)) {
        FL_CUDA_TRY(h, cudaEventRecord(h->ev_fork, st));
        FL_CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        sst = h->side;
    }
    int rc = FL_OK;
    if (q.ntiles > 0) {
        if (f32) rc = launch_far<float>(h, P, t, rb, ro, expo, pw32, st, q.ntiles);
        else if (dw) rc = launch_far_dw(h, P, t, rb, ro, pw, st, q.ntiles);
        else rc = launch_far<double>(h, P, t, rb, ro, expo, pw, st, q.ntiles);
    }
    ElemArgs E = elem_args(h, P, t, ro, s, C, f32);
    E.cluster = 1;
    E.nblk = 0;
    E.Pd = nullptr;
    E.Bf = nullptr;
    int side_rc = launch_near_pairs(h, P, t, rb, ro, expo, pw, f32, C, sst);
    if (side_rc == FL_OK) side_rc = launch_touch_pairs(h, P, t, ro, s, C, pw, f32, sst);
    if (side_rc == FL_OK) side_rc = launch_element(h, E, pw, 1, sst);
    if (side_rc == FL_OK) side_rc = launch_element(h, E, pw, 2, sst);
    if (sst != st) {  // joined even after an error, so that the caller's stream never runs ahead
        FL_CUDA_TRY(h, cudaEventRecord(h->ev_join, sst));
        FL_CUDA_TRY(h, cudaStreamWaitEvent(st, h->ev_join, 0));
    }
    FL_TRY(rc);
    FL_TRY(side_rc);
    if (nnz > 0) {
        const unsigned g = (unsigned)((nnz + 255) / 256);
        if (f32)
            hnear_compose_kernel<float><<<g, 256, 0, st>>>(nnz, nz_row, nz_col, t.csr_ptr, t.csr_col, t.g_ptr, t.g_slot,
                                                           t.contrib, t.occ_ptr, t.occ_blk, t.occ_loc, t.L_ptr,
                                                           q.trow_ptr, q.tiles, q.toff, (const float*)q.P, -C, nz_val);
        else
            hnear_compose_kernel<double><<<g, 256, 0, st>>>(nnz, nz_row, nz_col, t.csr_ptr, t.csr_col, t.g_ptr,
                                                            t.g_slot, t.contrib, t.occ_ptr, t.occ_blk, t.occ_loc, t.L_ptr,
                                                            q.trow_ptr, q.tiles, q.toff, q.P, -C, nz_val);
        fl::count_launch();
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

int tune_assemble(fl_ctx* h, double s, double* A, int64_t lda, int reps, int* best_variant, double* best_ms,
                  cudaStream_t st) {
    if (reps < 1) return set_err(h, FL_EINVAL, "reps < 1");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    const int pw = pw_mode(P.dim, s);
    if (!far_dw_applies(h, P, pw))
        return set_err(h, FL_ENOTIMPL, "no launch variants to tune (float64 mode, 2D, k_far = 4, s in {1/4, 1/2, 3/4})");
    const int prof0 = h->profiling, var0 = h->far_variant;
    int best = 0, rc = FL_OK;
    double best_t = 0.0;
    h->profiling = 1;
    for (int v = 1; v <= 4 && rc == FL_OK; ++v) {
        h->far_variant = v;
        rc = assemble_impl(h, s, FL_FP64, A, lda, nullptr, st);
        std::vector<float> ts;
        for (int r = 0; r < reps && rc == FL_OK; ++r) {
            rc = assemble_impl(h, s, FL_FP64, A, lda, nullptr, st);
            if (rc != FL_OK) break;
            if (cudaEventSynchronize(h->ev[2 * FL_STAGE_FAR + 1]) != cudaSuccess) {
                rc = set_err(h, FL_ECUDA, "cudaEventSynchronize");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->ev[2 * FL_STAGE_FAR], h->ev[2 * FL_STAGE_FAR + 1]);
            ts.push_back(ms);
        }
        if (rc != FL_OK) break;
        std::sort(ts.begin(), ts.end());
        const double med = ts[ts.size() / 2];
        if (!best || med < best_t) {
            best = v;
            best_t = med;
        }
    }
    h->profiling = prof0;
    h->far_variant = var0;
    if (rc != FL_OK) return rc;
    far_dw_record(P, pw, best, best_t);
    if (best_variant) *best_variant = best;
    if (best_ms) *best_ms = best_t;
    return FL_OK;
}

int assemble_nearfield_csr(fl_ctx* h, double s, int precision, int64_t* nnz, int32_t* rowptr, int32_t* col,
                           double* val, cudaStream_t st) {
    if (!nnz) return set_err(h, FL_EINVAL, "nnz is NULL");
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    const int64_t nz = (int64_t)P.csr_col.size();
    *nnz = nz;
    if (!rowptr) return FL_OK;  // size query
    if (!col || !val) return set_err(h, FL_EINVAL, "col or val is NULL");
    const CsrOut out{rowptr, col, val};
    return assemble_impl(h, s, precision, nullptr, 0, &out, st);
}

// ----------------------------------------------------------- load vector --
// b_i = Σ_{K ∋ i} |K| Σ_b M_ab f_b (P1 mass matrix M_ab = (1 + δ_ab)/((d+1)(d+2))),
// f = 1 when f is NULL; one thread per DOF, cells of its vertex in a fixed order.
__global__ void load_vector_kernel(int64_t n, int dim, const int* vod, const int64_t* v2c_ptr, const int* v2c,
                                   const int* cells, const double* jac_orig, const double* f, int nrhs, int r,
                                   double* b, int64_t ldb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int NV = dim + 1;
    const int vtx = vod[i];
    const double scale = (dim == 2) ? 0.5 : 1.0;  // |K| = jac/2 (2D), jac (1D)
    const double den = 1.0 / ((dim + 1.0) * (dim + 2.0));
    double acc = 0.0;
    for (int64_t q = v2c_ptr[vtx]; q < v2c_ptr[vtx + 1]; ++q) {
        const int K = v2c[q];
        const double vol = scale * jac_orig[K];
        if (!f) {
            acc += vol / NV;
        } else {
            double sacc = 0.0;
            for (int a = 0; a < NV; ++a) {
                const int u = cells[(int64_t)K * NV + a];
                sacc += ((u == vtx) ? 2.0 : 1.0) * f[(int64_t)u * nrhs + r];
            }
            acc += vol * den * sacc;
        }
    }
    b[i * ldb + r] = acc;
}

// ---------------------------------------------------- fractional heat equation --
// Implicit time steps of the fractional heat equation (Section 2) give systems
// (M + dt A^s) u = b with the P1 mass matrix M (Section 5).  M is applied cell by cell from
// the element mass matrix |K| (1 + delta_ab) / ((d + 1)(d + 2)); one thread per DOF row sums
// over the cells around its vertex in a fixed order.

// Y = alpha M X + beta B for column r
__global__ void mass_apply_kernel(int64_t n, int dim, const int* vod, const int* dov, const int64_t* v2c_ptr,
                                  const int* v2c, const int* cells, const double* jac_orig, double alpha,
                                  const double* X, int64_t ldx, double beta, const double* B, int64_t ldb, double* Y,
                                  int64_t ldy, int r) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int NV = dim + 1;
    const int vtx = vod[i];
    const double scale = (dim == 2) ? 0.5 : 1.0;  // |K| = jac/2 (2D), jac (1D)
    const double den = 1.0 / ((dim + 1.0) * (dim + 2.0));
    double acc = 0.0;
    for (int64_t q = v2c_ptr[vtx]; q < v2c_ptr[vtx + 1]; ++q) {
        const int K = v2c[q];
        double sacc = 0.0;
        for (int a = 0; a < NV; ++a) {
            const int u = cells[(int64_t)K * NV + a];
            const int j = dov[u];
            if (j >= 0) sacc += ((u == vtx) ? 2.0 : 1.0) * X[(int64_t)j * ldx + r];
        }
        acc += scale * jac_orig[K] * den * sacc;
    }
    double y = alpha * acc;
    if (beta != 0.0) y += beta * B[i * ldb + r];
    Y[i * ldy + r] = y;
}

// H = dt A, entry by entry (H may be A)
__global__ void scale_matrix_kernel(int64_t n, double dt, const double* A, int64_t lda, double* H, int64_t ldh) {
    for (int64_t row = blockIdx.y; row < n; row += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
            H[row * ldh + j] = dt * A[row * lda + j];
}

// H += M, one thread per row
__global__ void add_mass_kernel(int64_t n, int dim, const int* vod, const int* dov, const int64_t* v2c_ptr,
                                const int* v2c, const int* cells, const double* jac_orig, double* H, int64_t ldh) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int NV = dim + 1;
    const int vtx = vod[i];
    const double scale = (dim == 2) ? 0.5 : 1.0;
    const double den = 1.0 / ((dim + 1.0) * (dim + 2.0));
    double* row = H + i * ldh;
    for (int64_t q = v2c_ptr[vtx]; q < v2c_ptr[vtx + 1]; ++q) {
        const int K = v2c[q];
        const double m = scale * jac_orig[K] * den;
        for (int a = 0; a < NV; ++a) {
            const int u = cells[(int64_t)K * NV + a];
            const int j = dov[u];
            if (j >= 0) row[j] += ((u == vtx) ? 2.0 : 1.0) * m;
        }
    }
}

int heat_matrix(fl_ctx* h, double s, double dt, const double* A, int64_t lda, double* H, int64_t ldh,
                cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!A || !H || lda < P.n || ldh < P.n || !(dt >= 0.0)) return set_err(h, FL_EINVAL, "bad A / H / lda / ldh / dt");
    if (H != A && (H < A + P.n * lda && A < H + P.n * ldh)) return set_err(h, FL_EINVAL, "H overlaps A without being A");
    if (H == A && ldh != lda) return set_err(h, FL_EINVAL, "in place needs ldh = lda");
    FL_CUDA_TRY(h, cudaSetDevice(h->device));
    FL_TRY(ensure_device(h, pi, st));
    DevTables& t = h->dev[pi];
    const unsigned gx = (unsigned)std::min<int64_t>((P.n + 255) / 256, 64);
    const unsigned gy = (unsigned)std::min<int64_t>(P.n, 65535);
    if (P.n > 0) {
        scale_matrix_kernel<<<dim3(gx, gy), 256, 0, st>>>(P.n, dt, A, lda, H, ldh);
        fl::count_launch();
        add_mass_kernel<<<(unsigned)((P.n + 127) / 128), 128, 0, st>>>(P.n, P.dim, t.vod, t.dov, t.v2c_ptr, t.v2c,
                                                                        t.cells, t.jac_orig, H, ldh);
        fl::count_launch();
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

int mass_apply(fl_ctx* h, double s, int nrhs, double alpha, const double* X, int64_t ldx, double beta, const double* B,
               int64_t ldb, double* Y, int64_t ldy, cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!X || !Y || nrhs < 1 || ldx < nrhs || ldy < nrhs || (beta != 0.0 && (!B || ldb < nrhs)))
        return set_err(h, FL_EINVAL, "bad X / B / Y / leading dimensions");
    if (X == Y) return set_err(h, FL_EINVAL, "Y must not be X");
    FL_CUDA_TRY(h, cudaSetDevice(h->device));
    FL_TRY(ensure_device(h, pi, st));
    DevTables& t = h->dev[pi];
    const unsigned g = (unsigned)((P.n + 127) / 128);
    for (int r = 0; r < nrhs && P.n > 0; ++r) {
        mass_apply_kernel<<<g, 128, 0, st>>>(P.n, P.dim, t.vod, t.dov, t.v2c_ptr, t.v2c, t.cells, t.jac_orig, alpha, X,
                                             ldx, beta, B, ldb, Y, ldy, r);
        fl::count_launch();
    }
    FL_CUDA_TRY(h, cudaGetLastError());
    return FL_OK;
}

int load_vector(fl_ctx* h, double s, const double* f, int nrhs, double* b, int64_t ldb, cudaStream_t st) {
    const int pi = plan_for(h, s);
    if (pi < 0) return FL_EINVAL;
    const Plan& P = h->plan[pi];
    if (!b || nrhs < 1 || ldb < nrhs) return set_err(h, FL_EINVAL, "bad b / nrhs / ldb");
    if (!f && nrhs != 1) return set_err(h, FL_EINVAL, "f = 1 needs nrhs = 1");
    FL_CUDA_TRY(h, cudaSetDevice(h->device));
    FL_TRY(ensure_device(h, pi, st));
    DevTables& t = h->dev[pi];
    if (P.sym_K) {
        // whole-mesh load vector of the periodic f (nodal values on the sector's vertices), folded
        void* ws = nullptr;
        const size_t need = ((size_t)P.n + (f ? (size_t)P.nv : 0)) * nrhs * sizeof(double);
        if (pool_dev_alloc(&ws, std::max<size_t>(need, 16)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, FL_ENOMEM, "reduced load-vector workspace");
        }
        double* bw = (double*)ws;
        double* fw = f ? bw + (size_t)P.n * nrhs : nullptr;
        if (f) {
            expand_nodal_kernel<<<(unsigned)((P.nv * nrhs + 127) / 128), 128, 0, st>>>(P.nv, nrhs, t.sector_of, f, fw);
            fl::count_launch();
        }
        const unsigned g = (unsigned)((P.n + 127) / 128);
        for (int r = 0; r < nrhs && P.n > 0; ++r) {
            load_vector_kernel<<<g, 128, 0, st>>>(P.n, P.dim, t.vod, t.v2c_ptr, t.v2c, t.cells, t.jac_orig, fw, nrhs, r,
                                                  bw, nrhs);
            fl::count_launch();
        }
        if (P.n_red > 0) {
            fold_vec_kernel<<<(unsigned)((P.n_red * nrhs + 127) / 128), 128, 0, st>>>(P.n_red, P.sym_K, nrhs, t.red_ptr,
                                                                                      t.red_mem, bw, b, ldb);
            fl::count_launch();
        }
        cudaError_t e = cudaGetLastError();
        cudaError_t e2 = cudaStreamSynchronize(st);
        pool_dev_free(ws);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return set_err(h, FL_ECUDA, std::string("reduced load vector: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return FL_OK;
    }
    const unsigned g = (unsigned)((P.n + 127) / 128);
    for (int r = 0; r < nrhs; ++r) {
        load_vector_kernel<<<g, 128, 0, st>>>(P.n, P.dim, t.vod, t.v2c_ptr, t.v2c, t.cells, t.jac_orig, f, nrhs, r, b, ldb); fl::count_launch();
        FL_CUDA_TRY(h, cudaGetLastError());
    }
    return FL_OK;
}

}  // namespace fl
