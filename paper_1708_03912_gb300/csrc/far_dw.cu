// Separated element pairs of the float64 mode (2D), evaluated in double-word arithmetic.
//
// Section 5 of arXiv:1708.03912 writes the stiffness matrix as a sum over element pairs;
// for pairs with disjoint closures the contribution is a smooth double integral of the
// kernel |x - y|^{-2-2s}, evaluated here by the collapsed Gauss rule of order 4 on both
// cells (16 x 16 points).  These pairs are the N_el^2 part of the assembly.
//
// The float64 pipe of this part retires ~1.7 operations per clock and SM against 128 for
// float32, so the float64 mode does not run these pairs in float64: point offsets and
// centroid differences are float pairs (double-word numbers), |x - y|^2 and the kernel
// power (a float32 estimate with one Newton correction written in double-word terms) are
// double-word values, and every sum is a double-word accumulator.  Each operation is exact
// to a few units of 2^-48 relative, far inside the 1e-12 entry tolerance of this mode.
//
// Work split: DW_WARPS warps per 32 x 32 tile of cells, lane = column cell, warp w takes
// the row points a = w, w + DW_WARPS, ...; per row cell the warps' 3x3 partial blocks and
// row sums are combined in a fixed order, the column sums once per tile, so the result is
// bitwise reproducible.  Outputs are those of the float64 far kernel: the per-tile partial
// blocks over the local DOF lists and the per-point row sums for the diagonal blocks.
// Launch variants (the unroll of the inner point loop, and the minimum resident blocks per
// SM, which bounds the registers a thread may use) are swept by fl_tune_assemble and
// recorded in the tuning table.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "context.h"
#include "device.h"

namespace fl {
namespace {

constexpr int DW_WARPS = 4;
constexpr int DW_Q = 16;  // collapsed Gauss rule of order 4
constexpr int NV = 3;

struct FarRuleDW {
    dw w[DW_Q];
    dw wphi[DW_Q * NV];  // reference weight x shape value
};

struct DwTileArgs {
    const double* cen;
    const double* jac;
    const char* hasdof;
    const int* loc;
    const int* ex_ptr;
    const int* ex_idx;
    const int* tiles;
    const int64_t* toff;
    const uint32_t* rowmask;  // per tile: the row cells to compute (null: all)
    const int* L_ptr;
    const int* inc_ptr;
    const int* inc_ent;
    const float4* pts;  // [cell][16] (x.h, x.l, y.h, y.l)
    double* P;
    double* Pd;  // [cell][block][point] row sums; null: not wanted (the cluster method's near field)
    int64_t nc;
    int64_t nblk;
};

// offsets x_a - c_K of the far rule as double-word pairs, from the same float64 expression
// as the float64 kernel's offsets
__global__ void prep_points_dw(const double* cvx, const double* cen, const double* lam, int64_t nc, float4* pts) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const double* v = cvx + k * 6;
    for (int a = 0; a < DW_Q; ++a) {
        dw o[2];
        for (int d = 0; d < 2; ++d) {
            const double x = v[d] + lam[2 * a] * (v[2 + d] - v[d]) + lam[2 * a + 1] * (v[4 + d] - v[d]);
            o[d] = dw_from(x - cen[k * 2 + d]);
        }
        pts[k * DW_Q + a] = make_float4(o[0].h, o[0].l, o[1].h, o[1].l);
    }
}

__device__ __forceinline__ dw dw_shfl_xor(dw v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.h, m), __shfl_xor_sync(0xffffffffu, v.l, m)};
}

// Sum over the 32 lanes of four double-word values per lane, scattered: afterwards lane l
// holds the total of value 2 ((l >> 4) & 1) + ((l >> 3) & 1); the eight lanes with the
// same bits 4 and 3 hold the same bits.
__device__ __forceinline__ dw reduce_scatter4_dw(const dw (&v)[4], int lane) {
    const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
    dw u[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const dw send = up16 ? v[k] : v[k + 2];
        const dw keep = up16 ? v[k + 2] : v[k];
        u[k] = dw_add(keep, dw_shfl_xor(send, 16));
    }
    dw w = dw_add(up8 ? u[1] : u[0], dw_shfl_xor(up8 ? u[0] : u[1], 8));
#pragma unroll
    for (int m = 4; m >= 1; m >>= 1) w = dw_add(w, dw_shfl_xor(w, m));
    return w;
}

template <int PW, int UB, int MINB>
__global__ void __launch_bounds__(32 * DW_WARPS, MINB)
    far_tile_dw_kernel(const DwTileArgs A, const __grid_constant__ FarRuleDW R, int maxL) {
    constexpr int Q = DW_Q, NA = Q / DW_WARPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tix = blockIdx.x;
    const int I = A.tiles[2 * tix], J = A.tiles[2 * tix + 1];
    const int nLI = A.L_ptr[I + 1] - A.L_ptr[I];
    const int nLJ = A.L_ptr[J + 1] - A.L_ptr[J];
    const int64_t nc = A.nc;
    const int64_t K0 = (int64_t)I * 32, Kt0 = (int64_t)J * 32;
    const int nI = (int)min((int64_t)32, nc - K0);
    const uint32_t rmask = A.rowmask ? A.rowmask[tix] : 0xffffffffu;

    float4* sQ = reinterpret_cast<float4*>(smem_raw);                  // [Q][32] column points
    dw* sS = reinterpret_cast<dw*>(sQ + Q * 32);                        // [DW_WARPS][Q][32] column sums
    dw* sOff = sS + DW_WARPS * Q * 32;                                  // [DW_WARPS][9][32] partial blocks
    dw* sW = sOff + DW_WARPS * 9 * 32;                                  // [Q * NV] weight x shape value
    double* sD = reinterpret_cast<double*>(sW + Q * NV);                // [32][Q] diagonal tile row sums
    double* sCen = sD + 32 * Q;                                         // [32][2]
    double* sJac = sCen + 64;                                           // [32]
    dw* priv = reinterpret_cast<dw*>(sJac + 32);                        // [NV][maxL][32] double-word
    int* sLoc = reinterpret_cast<int*>(priv + NV * maxL * 32);          // [32][NV]
    int* sHas = sLoc + 32 * NV;                                         // [32]

    const int64_t Kt = Kt0 + lane;
    const bool valid = Kt < nc;
    for (int b = warp; b < Q; b += DW_WARPS)
        sQ[b * 32 + lane] = valid ? A.pts[Kt * Q + b] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i < DW_WARPS * Q * 32; i += blockDim.x) sS[i] = {0.f, 0.f};
    for (int i = threadIdx.x; i < Q * NV; i += blockDim.x) sW[i] = R.wphi[i];
    for (int i = threadIdx.x; i < nI * 2; i += blockDim.x) sCen[i] = A.cen[K0 * 2 + i];
    for (int i = threadIdx.x; i < nI * NV; i += blockDim.x) sLoc[i] = A.loc[K0 * NV + i];
    for (int i = threadIdx.x; i < nI; i += blockDim.x) {
        sJac[i] = A.jac[K0 + i];
        sHas[i] = A.hasdof[K0 + i];
    }
    for (int i = threadIdx.x; i < NV * nLI * 32; i += blockDim.x) priv[i] = {0.f, 0.f};
    for (int i = threadIdx.x; i < 32 * Q; i += blockDim.x) sD[i] = 0.0;
    __syncthreads();

    double cj[2] = {0.0, 0.0};
    double wj = 0.0;
    bool hj = false;
    int ep = 0, ee = 0;
    if (valid) {
        cj[0] = A.cen[Kt * 2];
        cj[1] = A.cen[Kt * 2 + 1];
        wj = A.jac[Kt];
        hj = A.hasdof[Kt] != 0;
        ep = A.ex_ptr[Kt];
        ee = A.ex_ptr[Kt + 1];
    }
    const dw wjd = dw_from(wj);
    dw* mS = sS + warp * Q * 32 + lane;  // this thread's column sums, stride 32
    // an inactive lane's row cell is moved far away (every value stays finite) and its
    // kernel values are multiplied by zero
    const double far_away = 1e15;

    for (int kk = 0; kk < nI; ++kk) {
        const int64_t K = K0 + kk;
        bool act = valid && (I != J || kk < lane) && ((rmask >> kk) & 1u);
        if (act) {
            while (ep < ee && A.ex_idx[ep] < K) ++ep;
            if (ep < ee && A.ex_idx[ep] == K) act = false;
        }
        act = act && (hj || sHas[kk] != 0);
        if (!__any_sync(0xffffffffu, act)) {  // the same in every warp of the block
            if (I != J && A.Pd)
                for (int a = threadIdx.x; a < Q; a += blockDim.x) A.Pd[((int64_t)K * A.nblk + J) * Q + a] = 0.0;
            continue;
        }
        const float mask = act ? 1.f : 0.f;
        const dw Dx = dw_from(act ? sCen[kk * 2] - cj[0] : far_away);
        const dw Dy = dw_from(act ? sCen[kk * 2 + 1] - cj[1] : far_away);
        const double wK = sJac[kk];
        const dw wKd = dw_from(wK);
        // this warp's row points a = warp + DW_WARPS m: offsets from c_K', weights; the weights
        // of an inactive lane are zero, so its (finite) kernel values add nothing
        dw X[NA], Y[NA], waK[NA], t[NA][NV];
#pragma unroll
        for (int m = 0; m < NA; ++m) {
            const int a = warp + DW_WARPS * m;
            const float4 pa = __ldg(A.pts + K * Q + a);
            X[m] = dw_add(Dx, dw{pa.x, pa.y});
            Y[m] = dw_add(Dy, dw{pa.z, pa.w});
            waK[m] = dw_mul(R.w[a], wKd);
            waK[m].h = __fmul_rn(waK[m].h, mask);
            waK[m].l = __fmul_rn(waK[m].l, mask);
#pragma unroll
            for (int v = 0; v < NV; ++v) t[m][v] = {0.f, 0.f};
        }
#pragma unroll UB
        for (int b = 0; b < Q; ++b) {
            const float4 q = sQ[b * 32 + lane];
            const dw c0 = sW[b * NV], c1 = sW[b * NV + 1], c2 = sW[b * NV + 2];
            dw sb = mS[b * 32];
#pragma unroll
            for (int m = 0; m < NA; ++m) {
                const dw dx = dw_sub(X[m], dw{q.x, q.y});
                const dw dy = dw_sub(Y[m], dw{q.z, q.w});
                // |x - y|^2 = dx^2 + dy^2: exact squares of the high parts, both non-negative
                const dw px = two_prod(dx.h, dx.h), py = two_prod(dy.h, dy.h);
                dw r2 = fast_two_sum(fmaxf(px.h, py.h), fminf(px.h, py.h));
                const float cr = __fmaf_rn(dx.h, dx.l, __fmul_rn(dy.h, dy.l));
                r2.l = __fadd_rn(r2.l, __fmaf_rn(2.f, cr, __fadd_rn(px.l, py.l)));
                const dw kv = dw_kpow<PW>(r2);
                dw_mac_pos(t[m][0], c0, kv);
                dw_mac_pos(t[m][1], c1, kv);
                dw_mac_pos(t[m][2], c2, kv);
                dw_mac_pos(sb, waK[m], kv);
            }
            mS[b * 32] = sb;
        }
        dw off[NV][NV];
#pragma unroll
        for (int i = 0; i < NV; ++i)
#pragma unroll
            for (int j = 0; j < NV; ++j) off[i][j] = {0.f, 0.f};
        dw ru[NA];  // row sums (times |K'|) of this warp's row points
#pragma unroll
        for (int m = 0; m < NA; ++m) {
            const int a = warp + DW_WARPS * m;
#pragma unroll
            for (int v = 0; v < NV; ++v) t[m][v] = dw_renorm(t[m][v]);
            ru[m] = dw_mul(dw_add(dw_add(t[m][0], t[m][1]), t[m][2]), wjd);
            ru[m].h = __fmul_rn(ru[m].h, mask);
            ru[m].l = __fmul_rn(ru[m].l, mask);
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const dw c = R.wphi[a * NV + i];
#pragma unroll
                for (int j = 0; j < NV; ++j) dw_mac_pos(off[i][j], c, t[m][j]);
            }
        }
        for (int b = 0; b < Q; ++b) mS[b * 32] = dw_renorm(mS[b * 32]);
        // row sums of cell K over this tile's columns: lane l ends with the total of row point
        // warp + DW_WARPS (2 ((l >> 4) & 1) + ((l >> 3) & 1))
        {
            const dw tot = reduce_scatter4_dw(ru, lane);
            if ((lane & 7) == 0) {
                const int a = warp + DW_WARPS * ((((lane >> 4) & 1) << 1) | ((lane >> 3) & 1));
                if (I == J) sD[kk * Q + a] += dw_to(tot);
                else if (A.Pd) A.Pd[((int64_t)K * A.nblk + J) * Q + a] = dw_to(tot);
            }
        }
#pragma unroll
        for (int i = 0; i < NV; ++i)
#pragma unroll
            for (int j = 0; j < NV; ++j) sOff[(warp * 9 + i * NV + j) * 32 + lane] = dw_renorm(off[i][j]);
        __syncthreads();
        // warp j < 3 adds column j of the 3x3 block (the warps' partials in order) to the
        // lane-private partial block
        if (warp < NV && act) {
            const int j = warp;
            // |K| |K'| as a double-word number: the accumulation stays on the float32 pipe
            const dw sc = dw_mul(wKd, wjd);
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int li = sLoc[kk * NV + i];
                if (li >= 0) {
                    dw o = sOff[(i * NV + j) * 32 + lane];
#pragma unroll
                    for (int w = 1; w < DW_WARPS; ++w) o = dw_add(o, sOff[(w * 9 + i * NV + j) * 32 + lane]);
                    dw& pv = priv[(j * nLI + li) * 32 + lane];
                    pv = dw_add(pv, dw_mul(o, sc));
                }
            }
        }
        __syncthreads();
    }
    // column sums of this tile's cells: the warps' parts added in warp order
    if (valid && A.Pd) {
        for (int b = warp; b < Q; b += DW_WARPS) {
            dw acc = sS[b * 32 + lane];
            for (int w = 1; w < DW_WARPS; ++w) acc = dw_add(acc, sS[(w * Q + b) * 32 + lane]);
            double v = dw_to(acc);
            if (I == J) v += sD[lane * Q + b];
            A.Pd[((int64_t)Kt * A.nblk + I) * Q + b] = v;
        }
    }
    // partial block over the local DOF lists of blocks I and J
    double* Pt = A.P + A.toff[tix];
    const int pJ = A.L_ptr[J];
    for (int idx = threadIdx.x; idx < nLI * nLJ; idx += blockDim.x) {
        const int li = idx / nLJ, lj = idx - li * nLJ;
        double acc = 0.0;
        for (int q = A.inc_ptr[pJ + lj]; q < A.inc_ptr[pJ + lj + 1]; ++q) {
            const int e = A.inc_ent[q];
            const int l = e / NV, j = e - l * NV;
            acc += dw_to(priv[(j * nLI + li) * 32 + l]);
        }
        Pt[idx] = acc;
    }
}

// Element x far boundary facet sums of the boundary term (Section 2: the Omega x Omega^c part
// of the form reduced to the boundary), float64 mode, double-word arithmetic.  For cell k
// and its far rule point x_a: Bf[k][a] = sum over far facets e of sum_b w_b |e|
// n_e.(x_a - y_b) |x_a - y_b|^{-2-2s}, y_b the k_far-point Gauss rule on e.  n_e.(x - y)
// is taken as n.(c_k - e0) + n.(x_a - c_k) - t_b n.E (the last term is zero up to the
// rounding of the stored normal and is kept as a float32 correction).  One lane per cell,
// BW_WARPS warps stride over the facets, their partial sums are added in warp order.
constexpr int BW_WARPS = 4;
constexpr int BW_K = 4;  // Gauss points per facet (k_far = 4)

struct BndRuleDW {
    dw t[BW_K];
    dw w[BW_K];
};

template <int PW>
__global__ void __launch_bounds__(32 * BW_WARPS)
    bnd_far_dw_kernel(int64_t nc, int64_t nf, const double* __restrict__ cen, const float4* __restrict__ pts,
                      const char* __restrict__ hasdof, const int* __restrict__ ef_ptr, const int* __restrict__ ef_fac,
                      const FacetRec* __restrict__ FR, const __grid_constant__ BndRuleDW G, double* __restrict__ Bf) {
    constexpr int Q = DW_Q;
    // facet chunk blockIdx.y of gridDim.y: its partial sums go to Bf + blockIdx.y nc Q
    const int64_t f_lo = nf * blockIdx.y / gridDim.y, f_hi = nf * (blockIdx.y + 1) / gridDim.y;
    Bf += (int64_t)blockIdx.y * nc * Q;
    __shared__ float4 sX[Q][32];
    __shared__ dw part[BW_WARPS][Q][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = k < nc && hasdof[k];
    for (int a = wid; a < Q; a += BW_WARPS) sX[a][lane] = valid ? pts[k * Q + a] : make_float4(0.f, 0.f, 0.f, 0.f);
    double c[2] = {0.0, 0.0};
    int ep = 0, ee = 0;
    if (valid) {
        c[0] = cen[2 * k];
        c[1] = cen[2 * k + 1];
        ep = ef_ptr[k];
        ee = ef_ptr[k + 1];
        while (ep < ee && ef_fac[ep] < f_lo) ++ep;
    }
    __syncthreads();
    dw B[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) B[a] = {0.f, 0.f};
    const bool any = __any_sync(0xffffffffu, valid);
    const double far_away = 1e15;
    for (int64_t f = f_lo + wid; any && f < f_hi; f += BW_WARPS) {
        bool act = valid;
        if (act) {
            while (ep < ee && ef_fac[ep] < f) ++ep;
            if (ep < ee && ef_fac[ep] == f) act = false;
        }
        const FacetRec r = FR[f];
        const float mask = act ? 1.f : 0.f;
        const dw Dx = dw_from(act ? c[0] - r.e0x : far_away), Dy = dw_from(act ? c[1] - r.e0y : far_away);
        const dw Ex = dw_from(r.ex), Ey = dw_from(r.ey), nx = dw_from(r.nx), ny = dw_from(r.ny);
        const dw Ld = dw_from(r.len);
        const float nE = (float)(r.nx * r.ex + r.ny * r.ey);
        dw Ux[BW_K], Uy[BW_K], LW[BW_K];
        float c2[BW_K];
#pragma unroll
        for (int b = 0; b < BW_K; ++b) {
            Ux[b] = dw_sub(Dx, dw_mul(G.t[b], Ex));
            Uy[b] = dw_sub(Dy, dw_mul(G.t[b], Ey));
            LW[b] = dw_mul(G.w[b], Ld);
            c2[b] = __fmul_rn(__fmul_rn(G.t[b].h, nE), LW[b].h);
        }
        const dw d0 = dw_add(dw_mul(nx, Dx), dw_mul(ny, Dy));  // n.(c_k - e0)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float4 q = sX[a][lane];
            const dw X = {q.x, q.y}, Y = {q.z, q.w};
            const dw da = dw_add(d0, dw_add(dw_mul(nx, X), dw_mul(ny, Y)));  // n.(x_a - e0)
            dw T = {0.f, 0.f};
            float corr = 0.f;
#pragma unroll
            for (int b = 0; b < BW_K; ++b) {
                dw dx = two_sum(Ux[b].h, X.h);
                dx.l = __fadd_rn(dx.l, __fadd_rn(Ux[b].l, X.l));
                dw dy = two_sum(Uy[b].h, Y.h);
                dy.l = __fadd_rn(dy.l, __fadd_rn(Uy[b].l, Y.l));
                const dw px = two_prod(dx.h, dx.h), py = two_prod(dy.h, dy.h);
                dw r2 = fast_two_sum(fmaxf(px.h, py.h), fminf(px.h, py.h));
                const float cr = __fmaf_rn(dx.h, dx.l, __fmul_rn(dy.h, dy.l));
                r2.l = __fadd_rn(r2.l, __fmaf_rn(2.f, cr, __fadd_rn(px.l, py.l)));
                dw kv = dw_kpow<PW>(r2);
                kv.h = __fmul_rn(kv.h, mask);
                kv.l = __fmul_rn(kv.l, mask);
                dw_mac(T, LW[b], kv);
                corr = __fmaf_rn(c2[b], kv.h, corr);
            }
            dw_mac(B[a], da, dw_renorm(T));
            B[a].l = __fsub_rn(B[a].l, corr);
        }
#pragma unroll
        for (int a = 0; a < Q; ++a) B[a] = dw_renorm(B[a]);
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) part[wid][a][lane] = B[a];
    __syncthreads();
    if (valid)
        for (int a = wid; a < Q; a += BW_WARPS) {
            dw acc = part[0][a][lane];
            for (int w = 1; w < BW_WARPS; ++w) acc = dw_add(acc, part[w][a][lane]);
            Bf[k * Q + a] = dw_to(acc);
        }
}

// Near separated pairs (vertex-graph distance 1) of the float64 mode in double-word arithmetic:
// the order-6 collapsed Gauss rule (36 points) on both cells, one thread per unordered pair,
// the same outputs as the float64 near-pair kernel (off-diagonal block times -C into the
// contribution slots, the per-point row sums of both cells into Dn).  Point offsets from the
// cell centroids come from a per-cell double-word table (prep_near_dw); every sum is a
// double-word accumulator, renormalised after each row point.
constexpr int NQ = 36;  // collapsed Gauss rule of order 6

struct NearRuleDW {
    dw w[NQ];
    dw wphi[NQ * NV];
};

__global__ void prep_near_dw(const double* cvx, const double* cen, const double* lam, int64_t nc, float4* pts) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * NQ) return;
    const int64_t k = t / NQ;
    const int a = (int)(t - k * NQ);
    const double* v = cvx + k * 6;
    dw o[2];
    for (int d = 0; d < 2; ++d) {
        const double x = v[d] + lam[2 * a] * (v[2 + d] - v[d]) + lam[2 * a + 1] * (v[4 + d] - v[d]);
        o[d] = dw_from(x - cen[k * 2 + d]);
    }
    pts[t] = make_float4(o[0].h, o[0].l, o[1].h, o[1].l);
}

template <int PW>
__global__ void __launch_bounds__(128) near_pair_dw_kernel(int nnear, const int* __restrict__ np_a,
                                                           const int* __restrict__ np_b, const double* __restrict__ cen,
                                                           const double* __restrict__ jac,
                                                           const float4* __restrict__ pts,
                                                           const __grid_constant__ NearRuleDW R, double C,
                                                           double* __restrict__ contrib, int64_t slot0,
                                                           double* __restrict__ Dn) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnear) return;
    const int ka = np_a[p], kb = np_b[p];
    const dw Dx = dw_from(cen[2 * (int64_t)ka] - cen[2 * (int64_t)kb]);
    const dw Dy = dw_from(cen[2 * (int64_t)ka + 1] - cen[2 * (int64_t)kb + 1]);
    const float4* pa = pts + (int64_t)ka * NQ;
    const float4* pb = pts + (int64_t)kb * NQ;
    const double ja = jac[ka], jb = jac[kb];
    double* Da = Dn + ((int64_t)p * 2 + 0) * NQ;
    double* Db = Dn + ((int64_t)p * 2 + 1) * NQ;
    dw S[NQ];
#pragma unroll
    for (int b = 0; b < NQ; ++b) S[b] = {0.f, 0.f};
    dw off[NV][NV];
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int j = 0; j < NV; ++j) off[i][j] = {0.f, 0.f};
#pragma unroll 1
    for (int a = 0; a < NQ; ++a) {
        const float4 qa = __ldg(pa + a);
        const dw X = dw_add(Dx, dw{qa.x, qa.y});
        const dw Y = dw_add(Dy, dw{qa.z, qa.w});
        const dw wa = R.w[a];
        dw t[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) t[v] = {0.f, 0.f};
#pragma unroll
        for (int b = 0; b < NQ; ++b) {
            const float4 qb = __ldg(pb + b);
            const dw dx = dw_sub(X, dw{qb.x, qb.y});
            const dw dy = dw_sub(Y, dw{qb.z, qb.w});
            // |x - y|^2 = dx^2 + dy^2: exact squares of the high parts, both non-negative
            const dw px = two_prod(dx.h, dx.h), py = two_prod(dy.h, dy.h);
            dw r2 = fast_two_sum(fmaxf(px.h, py.h), fminf(px.h, py.h));
            const float cr = __fmaf_rn(dx.h, dx.l, __fmul_rn(dy.h, dy.l));
            r2.l = __fadd_rn(r2.l, __fmaf_rn(2.f, cr, __fadd_rn(px.l, py.l)));
            const dw kv = dw_kpow<PW>(r2);
#pragma unroll
            for (int v = 0; v < NV; ++v) dw_mac_pos(t[v], R.wphi[b * NV + v], kv);
            dw_mac_pos(S[b], wa, kv);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) t[v] = dw_renorm(t[v]);
#pragma unroll
        for (int b = 0; b < NQ; ++b) S[b] = dw_renorm(S[b]);
        Da[a] = jb * dw_to(dw_add(dw_add(t[0], t[1]), t[2]));
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const dw c = R.wphi[a * NV + i];
#pragma unroll
            for (int j = 0; j < NV; ++j) dw_mac_pos(off[i][j], c, t[j]);
        }
    }
#pragma unroll
    for (int b = 0; b < NQ; ++b) Db[b] = ja * dw_to(S[b]);
    double* out = contrib + slot0 + (int64_t)p * NV * NV;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int j = 0; j < NV; ++j) out[i * NV + j] = -C * ja * jb * dw_to(dw_renorm(off[i][j]));
}

// Touching pairs of the float64 mode (2D: common edge, common vertex) in double-word arithmetic:
// the singular rules' tables (angular / Duffy points with the exact radial factor in their
// weights) as double-word numbers, one warp per pair, lanes over the points in a strided order,
// then a butterfly sum; the outputs of the float64 touching kernel.  The terms are signed
// (products of shape-function differences), so the sums use the signed accumulation.
__device__ __forceinline__ dw ldw(const float2* t, int i) {
    const float2 v = t[i];
    return {v.x, v.y};
}

template <int NL>
__device__ __forceinline__ void touch_accumulate(dw (&acc)[NL * (NL + 1) / 2], dw f, const float2* r) {
    int q = 0;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        const dw fi = dw_mul(f, ldw(r, i));
#pragma unroll
        for (int j = i; j < NL; ++j) dw_mac(acc[q++], fi, ldw(r, j));
    }
}

template <int PW>
__global__ void __launch_bounds__(128) touch_pair_dw_kernel(int ntp, const int* __restrict__ tp_type,
                                                            const int* __restrict__ tp_vert,
                                                            const int* __restrict__ tp_cell,
                                                            const int64_t* __restrict__ tp_slot,
                                                            const double* __restrict__ V,
                                                            const double* __restrict__ jac_orig,
                                                            const float2* __restrict__ rdw, RuleOffsets ro, double s,
                                                            double C, double* __restrict__ contrib) {
    const int lane = threadIdx.x & 31;
    const int p = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (p >= ntp) return;
    const int type = tp_type[p];
    const int* tv = tp_vert + 5 * p;
    double* out = contrib + tp_slot[p];
    const double jK = jac_orig[tp_cell[2 * p]], jM = jac_orig[tp_cell[2 * p + 1]];
    if (type == 0) {  // common edge [P,Q], thirds R (K) and Rt (M)
        const double *P_ = V + 2 * tv[0], *Q_ = V + 2 * tv[1], *R_ = V + 2 * tv[2], *Rt = V + 2 * tv[3];
        const dw a0 = dw_from(Q_[0] - P_[0]), a1 = dw_from(Q_[1] - P_[1]);
        const dw b0 = dw_from(R_[0] - Q_[0]), b1 = dw_from(R_[1] - Q_[1]);
        const dw c0 = dw_from(-(Rt[0] - Q_[0])), c1 = dw_from(-(Rt[1] - Q_[1]));
        const float2* tb = rdw + ro.t_edge;
        dw acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = {0.f, 0.f};
        for (int m = lane; m < ro.n_edge; m += 32) {
            const float2* r = tb + 8 * m;  // dphi[4], w1, w2, w3, weight
            const dw w1 = ldw(r, 4), w2 = ldw(r, 5), w3 = ldw(r, 6);
            const dw x = dw_add(dw_add(dw_mul(a0, w1), dw_mul(b0, w2)), dw_mul(c0, w3));
            const dw y = dw_add(dw_add(dw_mul(a1, w1), dw_mul(b1, w2)), dw_mul(c1, w3));
            const dw kv = dw_kpow<PW>(dw_add(dw_sqr(x), dw_sqr(y)));
            touch_accumulate<4>(acc, dw_mul(ldw(r, 7), kv), r);
#pragma unroll
            for (int q = 0; q < 10; ++q) acc[q] = dw_renorm(acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 10; ++q)
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) acc[q] = dw_add(acc[q], dw_shfl_xor(acc[q], o));
        if (lane == 0) {
            const double sc = C * jK * jM / ((3.0 - 2.0 * s) * (4.0 - 2.0 * s));
            int q = 0;
            for (int i = 0; i < 4; ++i)
                for (int j = i; j < 4; ++j, ++q) out[i * 4 + j] = out[j * 4 + i] = sc * dw_to(acc[q]);
        }
    } else {  // common vertex P: K = (P,Q,R), M = (P,Qt,Rt)
        const double *P_ = V + 2 * tv[0], *Q_ = V + 2 * tv[1], *R_ = V + 2 * tv[2], *Qt = V + 2 * tv[3], *Rt = V + 2 * tv[4];
        const dw g10 = dw_from(Q_[0] - P_[0]), g11 = dw_from(Q_[1] - P_[1]);
        const dw g20 = dw_from(R_[0] - Q_[0]), g21 = dw_from(R_[1] - Q_[1]);
        const dw g30 = dw_from(-(Qt[0] - P_[0])), g31 = dw_from(-(Qt[1] - P_[1]));
        const dw g40 = dw_from(-(Rt[0] - Qt[0])), g41 = dw_from(-(Rt[1] - Qt[1]));
        const float2* tb = rdw + ro.t_vert;
        dw acc[15];
#pragma unroll
        for (int q = 0; q < 15; ++q) acc[q] = {0.f, 0.f};
        for (int m = lane; m < ro.n_vert; m += 32) {
            const float2* r = tb + 10 * m;  // dphi[5], x1, x2, y1, y2, weight
            const dw u1 = ldw(r, 5), u2 = ldw(r, 6), u3 = ldw(r, 7), u4 = ldw(r, 8);
            const dw x = dw_add(dw_add(dw_mul(g10, u1), dw_mul(g20, u2)), dw_add(dw_mul(g30, u3), dw_mul(g40, u4)));
            const dw y = dw_add(dw_add(dw_mul(g11, u1), dw_mul(g21, u2)), dw_add(dw_mul(g31, u3), dw_mul(g41, u4)));
            const dw kv = dw_kpow<PW>(dw_add(dw_sqr(x), dw_sqr(y)));
            touch_accumulate<5>(acc, dw_mul(ldw(r, 9), kv), r);
#pragma unroll
            for (int q = 0; q < 15; ++q) acc[q] = dw_renorm(acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 15; ++q)
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) acc[q] = dw_add(acc[q], dw_shfl_xor(acc[q], o));
        if (lane == 0) {
            const double sc = C * jK * jM / (4.0 - 2.0 * s);
            int q = 0;
            for (int i = 0; i < 5; ++i)
                for (int j = i; j < 5; ++j, ++q) out[i * 5 + j] = out[j * 5 + i] = sc * dw_to(acc[q]);
        }
    }
}

// partial boundary sums of the facet chunks -> Bf, chunks added in order
__global__ void bnd_chunks_sum(int64_t m, int nch, const double* __restrict__ part, double* __restrict__ Bf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double acc = part[i];
    for (int c = 1; c < nch; ++c) acc += part[(int64_t)c * m + i];
    Bf[i] = acc;
}

size_t dw_smem_bytes(int maxL) {
    return (size_t)DW_Q * 32 * sizeof(float4) + (size_t)DW_WARPS * DW_Q * 32 * sizeof(dw) +
           (size_t)DW_WARPS * 9 * 32 * sizeof(dw) + DW_Q * NV * sizeof(dw) + 32 * DW_Q * sizeof(double) +
           96 * sizeof(double) + (size_t)NV * maxL * 32 * sizeof(double) + 32 * NV * sizeof(int) + 32 * sizeof(int);
}

template <int PW, int UB, int MINB>
int launch_t(fl_ctx* h, const Plan& P, DevTables& t, const FarRuleDW& R, int64_t ntiles, cudaStream_t st) {
    DwTileArgs A;
    A.cen = t.cen;
    A.jac = t.jac;
    A.hasdof = t.hasdof;
    A.loc = t.loc;
    A.ex_ptr = t.ex_ptr;
    A.ex_idx = t.ex_idx;
    A.tiles = t.tiles;
    A.toff = t.toff;
    A.rowmask = t.tile_rowmask;
    A.L_ptr = t.L_ptr;
    A.inc_ptr = t.inc_ptr;
    A.inc_ent = t.inc_ent;
    A.pts = (const float4*)t.pts_dw;
    A.P = (double*)t.P;
    A.Pd = (double*)t.Pd;
    A.nc = P.nc;
    A.nblk = P.nblk;
    const int maxL = std::max(1, P.maxL);
    const size_t smem = dw_smem_bytes(maxL);
    auto kern = far_tile_dw_kernel<PW, UB, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_err(h, FL_ECUDA, std::string("far_tile_dw smem: ") + cudaGetErrorString(e));
    if (ntiles > 0) {
        kern<<<(unsigned)ntiles, 32 * DW_WARPS, smem, st>>>(A, R, maxL);
        count_launch(1);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(h, FL_ECUDA, std::string("far_tile_dw launch: ") + cudaGetErrorString(e));
    return FL_OK;
}

// launch variants: (unroll of the loop over the column cell's points, minimum resident
// blocks per SM)   1: (4, 1)   2: (1, 2)   3: (2, 2)   4: (1, 3)
constexpr int DW_VARIANTS = 4;

template <int PW>
int launch_pw(fl_ctx* h, const Plan& P, DevTables& t, const FarRuleDW& R, int variant, int64_t nt, cudaStream_t st) {
    switch (variant) {
        case 1: return launch_t<PW, 4, 1>(h, P, t, R, nt, st);
        case 2: return launch_t<PW, 1, 2>(h, P, t, R, nt, st);
        case 4: return launch_t<PW, 1, 3>(h, P, t, R, nt, st);
        default: return launch_t<PW, 2, 2>(h, P, t, R, nt, st);
    }
}

std::string kernel_name(int pw) { return "far_tile_dw<" + std::to_string(pw) + ">"; }

}  // namespace

// facet chunks of the double-word boundary kernel: about four waves of 3 blocks per SM
int bnd_dw_chunks(int64_t nc) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    const int64_t nb = std::max<int64_t>(1, (nc + 31) / 32);
    return (int)std::min<int64_t>(8, std::max<int64_t>(1, (12 * (int64_t)sms + nb - 1) / nb));
}

bool far_dw_applies(const fl_ctx* h, const Plan& P, int pw) {
    return P.dim == 2 && h->opt.k_far == 4 && (pw == 5 || pw == 6 || pw == 7) && !h->far_f64_pipe;
}

int prep_far_dw(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, cudaStream_t st) {
    const unsigned g = (unsigned)((P.nc + 127) / 128);
    if (P.nc > 0) {
        prep_points_dw<<<g, 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.far_lam, P.nc, (float4*)t.pts_dw);
        count_launch(1);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FL_OK : set_err(h, FL_ECUDA, std::string("prep_points_dw: ") + cudaGetErrorString(e));
}

// Variant of the launch: the caller's choice if > 0, else the tuning table's entry for this
// kernel and cell count, else 3 (the fastest on the disc workloads measured).
int far_dw_variant(const fl_ctx* h, const Plan& P, int pw) {
    if (h->far_variant > 0) return h->far_variant;
    int p0 = 0, p1 = 0;
    if (tune_lookup(device_name(), kernel_name(pw), P.nc, 1, 1, &p0, &p1) && p0 >= 1 && p0 <= DW_VARIANTS) return p0;
    return 3;
}

int launch_far_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                  cudaStream_t st, int64_t ntiles) {
    const int64_t nt = ntiles >= 0 ? ntiles : (int64_t)P.tiles.size() / 2;
    FarRuleDW R;
    for (int a = 0; a < DW_Q; ++a) {
        const double w = rb[ro.far_w + a];
        R.w[a].h = (float)w;
        R.w[a].l = (float)(w - (double)R.w[a].h);
        for (int v = 0; v < NV; ++v) {
            const double c = w * rb[ro.far_phi + a * NV + v];
            R.wphi[a * NV + v].h = (float)c;
            R.wphi[a * NV + v].l = (float)(c - (double)R.wphi[a * NV + v].h);
        }
    }
    const int variant = far_dw_variant(h, P, pw);
    switch (pw) {
        case 5: return launch_pw<5>(h, P, t, R, variant, nt, st);
        case 6: return launch_pw<6>(h, P, t, R, variant, nt, st);
        default: return launch_pw<7>(h, P, t, R, variant, nt, st);
    }
}

int launch_bnd_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                  cudaStream_t st) {
    BndRuleDW G;
    for (int b = 0; b < BW_K; ++b) {
        const double tb = rb[ro.glf_t + b], wb = rb[ro.glf_w + b];
        G.t[b].h = (float)tb;
        G.t[b].l = (float)(tb - (double)G.t[b].h);
        G.w[b].h = (float)wb;
        G.w[b].l = (float)(wb - (double)G.w[b].h);
    }
    const unsigned nb = (unsigned)((P.nc + 31) / 32);
    const FacetRec* FR = (const FacetRec*)t.facet_rec;
    // facets split into chunks (one grid row each) so that small meshes still fill the GPU
    const int nch = bnd_dw_chunks(P.nc);
    double* out = nch > 1 ? t.Bfp : t.Bf;
    if (nb > 0) {
#define FL_BNDW(PWV)                                                                                             \
    bnd_far_dw_kernel<PWV><<<dim3(nb, nch), 32 * BW_WARPS, 0, st>>>(P.nc, P.nf, t.cen, (const float4*)t.pts_dw, \
                                                                   t.hasdof, t.ef_ptr, t.ef_fac, FR, G, out)
        if (pw == 5) FL_BNDW(5);
        else if (pw == 6) FL_BNDW(6);
        else FL_BNDW(7);
#undef FL_BNDW
        count_launch(1);
        if (nch > 1) {
            const int64_t m = P.nc * DW_Q;
            bnd_chunks_sum<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, nch, t.Bfp, t.Bf);
            count_launch(1);
        }
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FL_OK : set_err(h, FL_ECUDA, std::string("bnd_far_dw: ") + cudaGetErrorString(e));
}

bool near_dw_applies(const fl_ctx* h, const Plan& P, int pw) {
    return P.dim == 2 && h->opt.k_near == 6 && (pw == 5 || pw == 6 || pw == 7) && !h->far_f64_pipe;
}

int launch_near_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                   double C, cudaStream_t st) {
    const int nnear = (int)P.np_a.size();
    if (nnear == 0) return FL_OK;
    if (ro.qn != NQ || !t.pts_near_dw) return set_err(h, FL_EINVAL, "near_pair_dw: order-6 rule and its point table needed");
    NearRuleDW R;
    for (int a = 0; a < NQ; ++a) {
        const double w = rb[ro.near_w + a];
        R.w[a].h = (float)w;
        R.w[a].l = (float)(w - (double)R.w[a].h);
        for (int v = 0; v < NV; ++v) {
            const double c = w * rb[ro.near_phi + a * NV + v];
            R.wphi[a * NV + v].h = (float)c;
            R.wphi[a * NV + v].l = (float)(c - (double)R.wphi[a * NV + v].h);
        }
    }
    const int64_t np = P.nc * NQ;
    prep_near_dw<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(t.cvx, t.cen, t.rule + ro.near_lam, P.nc,
                                                               (float4*)t.pts_near_dw);
    const unsigned g = (unsigned)((nnear + 127) / 128);
    const float4* pts = (const float4*)t.pts_near_dw;
    if (pw == 5) near_pair_dw_kernel<5><<<g, 128, 0, st>>>(nnear, t.np_a, t.np_b, t.cen, t.jac, pts, R, C, t.contrib, P.np_slot0, t.Dn);
    else if (pw == 6) near_pair_dw_kernel<6><<<g, 128, 0, st>>>(nnear, t.np_a, t.np_b, t.cen, t.jac, pts, R, C, t.contrib, P.np_slot0, t.Dn);
    else near_pair_dw_kernel<7><<<g, 128, 0, st>>>(nnear, t.np_a, t.np_b, t.cen, t.jac, pts, R, C, t.contrib, P.np_slot0, t.Dn);
    count_launch(2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FL_OK : set_err(h, FL_ECUDA, std::string("near_pair_dw: ") + cudaGetErrorString(e));
}

bool touch_dw_applies(const fl_ctx* h, const Plan& P, int pw) {
    return P.dim == 2 && (pw == 5 || pw == 6 || pw == 7) && !h->far_f64_pipe;
}

int launch_touch_dw(fl_ctx* h, const Plan& P, DevTables& t, const RuleOffsets& ro, double s, double C, int pw,
                    cudaStream_t st) {
    const int ntp = (int)P.tp_type.size();
    if (ntp == 0) return FL_OK;
    if (!t.rule_dw) return set_err(h, FL_EINVAL, "touch_pair_dw: double-word rule tables missing");
    const unsigned g = (unsigned)(((int64_t)ntp * 32 + 127) / 128);
    if (pw == 5) touch_pair_dw_kernel<5><<<g, 128, 0, st>>>(ntp, t.tp_type, t.tp_vert, t.tp_cell, t.tp_slot, t.V, t.jac_orig, (const float2*)t.rule_dw, ro, s, C, t.contrib);
    else if (pw == 6) touch_pair_dw_kernel<6><<<g, 128, 0, st>>>(ntp, t.tp_type, t.tp_vert, t.tp_cell, t.tp_slot, t.V, t.jac_orig, (const float2*)t.rule_dw, ro, s, C, t.contrib);
    else touch_pair_dw_kernel<7><<<g, 128, 0, st>>>(ntp, t.tp_type, t.tp_vert, t.tp_cell, t.tp_slot, t.V, t.jac_orig, (const float2*)t.rule_dw, ro, s, C, t.contrib);
    count_launch(1);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FL_OK : set_err(h, FL_ECUDA, std::string("touch_pair_dw: ") + cudaGetErrorString(e));
}

void far_dw_record(const Plan& P, int pw, int variant, double ms) {
    tune_record(device_name(), kernel_name(pw), P.nc, 1, 1, variant, 0, ms);
}

}  // namespace fl
