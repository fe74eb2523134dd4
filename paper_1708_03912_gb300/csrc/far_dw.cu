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
// Variants (the launch's minimum resident blocks per SM, which bounds the registers a
// thread may use) are swept by fl_tune_assemble and recorded in the tuning table.
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
    const int* L_ptr;
    const int* inc_ptr;
    const int* inc_ent;
    const float4* pts;  // [cell][16] (x.h, x.l, y.h, y.l)
    double* P;
    double* Pd;  // [cell][block][point] row sums
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

template <int PW, int MINB>
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

    float4* sQ = reinterpret_cast<float4*>(smem_raw);                  // [Q][32] column points
    dw* sOff = reinterpret_cast<dw*>(sQ + Q * 32);                      // [DW_WARPS][9][32] partial blocks
    double* sD = reinterpret_cast<double*>(sOff + DW_WARPS * 9 * 32);  // [32][Q] diagonal tile row sums
    double* sCen = sD + 32 * Q;                                         // [32][2]
    double* sJac = sCen + 64;                                           // [32]
    double* priv = sJac + 32;                                           // [NV][maxL][32]
    int* sLoc = reinterpret_cast<int*>(priv + NV * maxL * 32);          // [32][NV]
    int* sHas = sLoc + 32 * NV;                                         // [32]

    const int64_t Kt = Kt0 + lane;
    const bool valid = Kt < nc;
    for (int b = warp; b < Q; b += DW_WARPS)
        sQ[b * 32 + lane] = valid ? A.pts[Kt * Q + b] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i < nI * 2; i += blockDim.x) sCen[i] = A.cen[K0 * 2 + i];
    for (int i = threadIdx.x; i < nI * NV; i += blockDim.x) sLoc[i] = A.loc[K0 * NV + i];
    for (int i = threadIdx.x; i < nI; i += blockDim.x) {
        sJac[i] = A.jac[K0 + i];
        sHas[i] = A.hasdof[K0 + i];
    }
    for (int i = threadIdx.x; i < NV * nLI * 32; i += blockDim.x) priv[i] = 0.0;
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
    dw S[Q];  // column sums of this lane's cell over this warp's row points
#pragma unroll
    for (int b = 0; b < Q; ++b) S[b] = {0.f, 0.f};
    // an inactive lane's row cell is moved far away (every value stays finite) and its
    // kernel values are multiplied by zero
    const double far_away = 1e15;

    for (int kk = 0; kk < nI; ++kk) {
        const int64_t K = K0 + kk;
        bool act = valid && (I != J || kk < lane);
        if (act) {
            while (ep < ee && A.ex_idx[ep] < K) ++ep;
            if (ep < ee && A.ex_idx[ep] == K) act = false;
        }
        act = act && (hj || sHas[kk] != 0);
        if (!__any_sync(0xffffffffu, act)) {  // the same in every warp of the block
            if (I != J)
                for (int a = threadIdx.x; a < Q; a += blockDim.x) A.Pd[((int64_t)K * A.nblk + J) * Q + a] = 0.0;
            continue;
        }
        const float mask = act ? 1.f : 0.f;
        const dw Dx = dw_from(act ? sCen[kk * 2] - cj[0] : far_away);
        const dw Dy = dw_from(act ? sCen[kk * 2 + 1] - cj[1] : far_away);
        const double wK = sJac[kk];
        const dw wKd = dw_from(wK);
        dw off[NV][NV];
#pragma unroll
        for (int i = 0; i < NV; ++i)
#pragma unroll
            for (int j = 0; j < NV; ++j) off[i][j] = {0.f, 0.f};
        dw ru[NA];  // row sums (times |K'|) of this warp's row points
#pragma unroll
        for (int m = 0; m < NA; ++m) {
            const int a = warp + DW_WARPS * m;
            const float4 pa = __ldg(A.pts + K * Q + a);
            const dw X = dw_add(Dx, dw{pa.x, pa.y});
            const dw Y = dw_add(Dy, dw{pa.z, pa.w});
            const dw waK = dw_mul(R.w[a], wKd);
            dw t[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) t[v] = {0.f, 0.f};
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                const float4 q = sQ[b * 32 + lane];
                const dw dx = dw_sub(X, dw{q.x, q.y});
                const dw dy = dw_sub(Y, dw{q.z, q.w});
                // |x - y|^2 = dx^2 + dy^2: exact squares of the high parts, both non-negative
                const dw px = two_prod(dx.h, dx.h), py = two_prod(dy.h, dy.h);
                dw r2 = fast_two_sum(fmaxf(px.h, py.h), fminf(px.h, py.h));
                const float cr = __fmaf_rn(dx.h, dx.l, __fmul_rn(dy.h, dy.l));
                r2.l = __fadd_rn(r2.l, __fmaf_rn(2.f, cr, __fadd_rn(px.l, py.l)));
                dw kv = dw_kpow<PW>(r2);
                kv.h = __fmul_rn(kv.h, mask);
                kv.l = __fmul_rn(kv.l, mask);
#pragma unroll
                for (int v = 0; v < NV; ++v) dw_mac(t[v], R.wphi[b * NV + v], kv);
                dw_mac(S[b], waK, kv);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) t[v] = dw_renorm(t[v]);
            ru[m] = dw_mul(dw_add(dw_add(t[0], t[1]), t[2]), wjd);
#pragma unroll
            for (int i = 0; i < NV; ++i)
#pragma unroll
                for (int j = 0; j < NV; ++j) dw_mac(off[i][j], R.wphi[a * NV + i], t[j]);
        }
#pragma unroll
        for (int b = 0; b < Q; ++b) S[b] = dw_renorm(S[b]);
        // row sums of cell K over this tile's columns: lane l ends with the total of row point
        // warp + DW_WARPS (2 ((l >> 4) & 1) + ((l >> 3) & 1))
        {
            const dw tot = reduce_scatter4_dw(ru, lane);
            if ((lane & 7) == 0) {
                const int a = warp + DW_WARPS * ((((lane >> 4) & 1) << 1) | ((lane >> 3) & 1));
                if (I == J) sD[kk * Q + a] += dw_to(tot);
                else A.Pd[((int64_t)K * A.nblk + J) * Q + a] = dw_to(tot);
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
            const double sc = wK * wj;
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int li = sLoc[kk * NV + i];
                if (li >= 0) {
                    dw o = sOff[(i * NV + j) * 32 + lane];
#pragma unroll
                    for (int w = 1; w < DW_WARPS; ++w) o = dw_add(o, sOff[(w * 9 + i * NV + j) * 32 + lane]);
                    priv[(j * nLI + li) * 32 + lane] += dw_to(o) * sc;
                }
            }
        }
        __syncthreads();
    }
    // column sums: the warps' parts added in warp order (sOff reused as [Q][32])
    dw* sS = sOff;
    for (int w = 0; w < DW_WARPS; ++w) {
        if (warp == w) {
#pragma unroll
            for (int b = 0; b < Q; ++b) sS[b * 32 + lane] = (w == 0) ? S[b] : dw_add(sS[b * 32 + lane], S[b]);
        }
        __syncthreads();
    }
    if (valid) {
        for (int b = warp; b < Q; b += DW_WARPS) {
            double v = dw_to(sS[b * 32 + lane]);
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
            acc += priv[(j * nLI + li) * 32 + l];
        }
        Pt[idx] = acc;
    }
}

size_t dw_smem_bytes(int maxL) {
    return (size_t)DW_Q * 32 * sizeof(float4) + (size_t)DW_WARPS * 9 * 32 * sizeof(dw) + 32 * DW_Q * sizeof(double) +
           96 * sizeof(double) + (size_t)NV * maxL * 32 * sizeof(double) + 32 * NV * sizeof(int) + 32 * sizeof(int);
}

template <int PW, int MINB>
int launch_t(fl_ctx* h, const Plan& P, DevTables& t, const FarRuleDW& R, cudaStream_t st) {
    DwTileArgs A;
    A.cen = t.cen;
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
    A.pts = (const float4*)t.pts_dw;
    A.P = (double*)t.P;
    A.Pd = (double*)t.Pd;
    A.nc = P.nc;
    A.nblk = P.nblk;
    const int maxL = std::max(1, P.maxL);
    const size_t smem = dw_smem_bytes(maxL);
    const int64_t ntiles = (int64_t)P.tiles.size() / 2;
    auto kern = far_tile_dw_kernel<PW, MINB>;
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

template <int PW>
int launch_pw(fl_ctx* h, const Plan& P, DevTables& t, const FarRuleDW& R, int variant, cudaStream_t st) {
    switch (variant) {
        case 2: return launch_t<PW, 2>(h, P, t, R, st);
        case 4: return launch_t<PW, 4>(h, P, t, R, st);
        default: return launch_t<PW, 3>(h, P, t, R, st);
    }
}

std::string kernel_name(int pw) { return "far_tile_dw<" + std::to_string(pw) + ">"; }

}  // namespace

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

// Variant (minimum resident blocks per SM) of the launch: the caller's choice if > 0, else
// the tuning table's entry for this kernel and cell count, else 3.
int far_dw_variant(const fl_ctx* h, const Plan& P, int pw) {
    if (h->far_variant > 0) return h->far_variant;
    int p0 = 0, p1 = 0;
    if (tune_lookup(device_name(), kernel_name(pw), P.nc, 1, 1, &p0, &p1) && p0 >= 2 && p0 <= 4) return p0;
    return 3;
}

int launch_far_dw(fl_ctx* h, const Plan& P, DevTables& t, const std::vector<double>& rb, const RuleOffsets& ro, int pw,
                  cudaStream_t st) {
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
        case 5: return launch_pw<5>(h, P, t, R, variant, st);
        case 6: return launch_pw<6>(h, P, t, R, variant, st);
        default: return launch_pw<7>(h, P, t, R, variant, st);
    }
}

void far_dw_record(const Plan& P, int pw, int variant, double ms) {
    tune_record(device_name(), kernel_name(pw), P.nc, 1, 1, variant, 0, ms);
}

}  // namespace fl
