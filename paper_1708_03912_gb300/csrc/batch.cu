// Batched solves of A^s U = B for several orders s (several matrices) and many
// right-hand sides at once: conjugate gradients on a Jacobi-scaled bfloat16 copy
// of each matrix, whose block product Ã P is a tensor-core GEMM (tcgen05, bf16
// operands, float32 accumulation in tensor memory, operands staged by TMA), inside
// float64 iterative refinement judged by the float64 residual B - A U.
//
// The paper's solver (Section 5) is diagonally preconditioned CG on one system;
// running many systems together turns the matrix-vector product, whose cost is
// streaming A once (n^2 entries), into a GEMM that streams each matrix once for
// all right-hand sides.  With 64 right-hand sides the GEMM performs 64 flops per
// byte of bf16 matrix, below the tensor-core ridge: the inner iteration is still
// bound by HBM bandwidth, now shared by 64 solves.
//
// Precision: a float32 vector p is carried as p_hi + p_lo (two bf16), the
// scaled matrix Ã as S_0 (+ S_1) (one or two bf16 slices); the product formed is
// S_0 (p_hi + p_lo) + S_1 p_hi with float32 accumulation, relative accuracy about
// 2^-16 with two slices and 2^-8 with one.  The refinement residual and the
// solution update are float64.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "context.h"
#include "device.h"
#include "tc.h"

namespace fl {
namespace bt {

constexpr int BM = 128;            // matrix rows per GEMM tile (MMA M)
constexpr int BK = 64;             // K extent of one chunk: one 128-byte bf16 row
constexpr int THREADS = 256;       // warp 0: TMA producer, warp 1: MMA issuer, warps 4-7: epilogue
constexpr int MAXP = FL_BATCH_MAXPROB;
constexpr int A_TILE = BM * BK * 2;  // bytes of one matrix tile (16 KiB)
constexpr int MAX_STAGES = 8;
constexpr int MAX_TILES = 512;     // n <= 65536
constexpr int UMIN = 8;            // fewest chunks a CTA takes in a GEMM phase

struct ColState {
    double rr, rr0;  // current and initial r.r of the inner iteration
    int done, its, status, pad;
};
struct ColOuter {
    double bb, rel;  // ||b||^2 and the last relative float64 residual
    int odone, status;
};

struct ProbDev {
    int n, nr, nslices, mtiles, chunks, ldv;
    float *r, *z, *p, *q;  // [nr][ldv]
    __nv_bfloat16* P;      // [2 nr][ldv]: p_hi rows then p_lo rows (TMA source)
    ColState* col;         // [nr]
};

struct Params {
    CUtensorMap tmA[MAXP][2];  // bf16 slices S_0, S_1 (box 64 x 128)
    CUtensorMap tmP[MAXP];     // P (box 64 x 2 nr)
    ProbDev prob[MAXP];
    int nprob, stages, rmax, nrmax, maxit, tmem_cols, nsmax;
    double tol2;
    float* slots;    // [G][rmax][nrmax][128] per-run partial products
    unsigned* gbar;  // grid barrier state (2 words)
    int* err;        // bit 0: mbarrier timeout, 1: run-slot overflow, 2: grid barrier timeout
    int* ndone;      // [MAXP] finished columns per problem
    int* active;     // [MAXP] (GEMM-only launches): problem takes part
    int* iters;      // CG steps taken by the last persistent launch
};

struct Ctl {
    uint64_t full[MAX_STAGES], empty[MAX_STAGES];
    uint64_t acc_full, acc_empty, drain;
    uint32_t tmem_base;
    int na, geff;
    int act[MAXP];
    long long ubase[MAXP + 1];
    int tbase[MAXP + 1];
    long long U;
    int own_first[MAX_TILES], own_r[MAX_TILES], own_cnt[MAX_TILES];
    double red[THREADS / 32];
    int flag;
};

struct Unit {
    int k, p, t, c;
};

__device__ __forceinline__ Unit decode(const Ctl& s, const Params& P, long long g) {
    int k = 0;
    while (k + 1 < s.na && g >= s.ubase[k + 1]) ++k;
    const int p = s.act[k];
    const long long l = g - s.ubase[k];
    const int ch = P.prob[p].chunks;
    return {k, p, (int)(l / ch), (int)(l % ch)};
}
__device__ __forceinline__ long long range_start(long long U, int G, int b) { return (U * b) / G; }
__device__ __forceinline__ int owner(long long g, long long U, int G) {
    int b = (int)((g * G) / U);
    while (b + 1 < G && range_start(U, G, b + 1) <= g) ++b;
    while (b > 0 && range_start(U, G, b) > g) --b;
    return b;
}
__device__ __forceinline__ long long tile_ordinal(const Ctl& s, const Params& P, long long g) {
    const Unit u = decode(s, P, g);
    return s.tbase[u.k] + u.t;
}

// Active problems of this phase, the unit (chunk) numbering over them and the
// number of CTAs that take part in the GEMM.  Run by every CTA on data that no
// CTA modifies during the phase, so all CTAs agree.
__device__ void plan_phase(Ctl& s, const Params& P, int G, bool cg_mode) {
    if (threadIdx.x == 0) {
        int na = 0, tt = 0;
        long long u = 0;
        for (int p = 0; p < P.nprob; ++p) {
            const bool on = cg_mode ? (__ldcg(P.ndone + p) < P.prob[p].nr) : (__ldcg(P.active + p) != 0);
            if (!on) continue;
            s.act[na] = p;
            s.ubase[na] = u;
            s.tbase[na] = tt;
            u += (long long)P.prob[p].mtiles * P.prob[p].chunks;
            tt += P.prob[p].mtiles;
            ++na;
        }
        s.ubase[na] = u;
        s.tbase[na] = tt;
        s.na = na;
        s.U = u;
        s.geff = (int)std::max<long long>(1, std::min<long long>(G, u / UMIN));
    }
    __syncthreads();
}

__device__ __forceinline__ uint8_t* stage_base(int stages) {
    extern __shared__ uint8_t dyn_smem[];
    (void)stages;
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
}

// Pipeline counters of the role threads, kept in registers across phases.
struct Roles {
    uint32_t pc = 0;  // chunks issued (producer) / consumed (MMA)
    uint32_t rc = 0;  // runs accumulated (MMA) / drained (epilogue)
    int last_issued = -1;
};

// One GEMM phase: for every active problem, Y = Ã P over its row tiles, the
// chunks (64-wide K slices) of all tiles split into G_eff contiguous ranges, one
// per CTA.  A CTA accumulates consecutive chunks of one tile in tensor memory
// (a "run") and writes each run's 128 x nr product to its slot.
__device__ void gemm_phase(Ctl& s, const Params& P, int b, Roles& ro) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (s.U == 0 || b >= s.geff) return;
    const long long u0 = range_start(s.U, s.geff, b), u1 = range_start(s.U, s.geff, b + 1);
    if (u0 >= u1) return;
    const int S = P.stages;
    const int stage_bytes = A_TILE * P.nsmax + P.nrmax * 2 * BK * 2;
    uint8_t* base = stage_base(S);

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pol_a = tc::policy_evict_first(), pol_b = tc::policy_evict_last();
            tc::fence_proxy_async_global();
            for (long long g = u0; g < u1; ++g) {
                const Unit u = decode(s, P, g);
                const ProbDev& pr = P.prob[u.p];
                const int st = ro.pc % S;
                const uint32_t ph = (ro.pc / S) & 1;
                if (!tc::mbar_wait(&s.empty[st], ph ^ 1)) {
                    atomicOr(P.err, 1);
                    break;
                }
                const uint32_t bytes = A_TILE * pr.nslices + pr.nr * 2 * BK * 2;
                tc::mbar_arrive_expect_tx(&s.full[st], bytes);
                uint8_t* sa = base + (size_t)st * stage_bytes;
                tc::tma_load_2d(sa, &P.tmA[u.p][0], u.c * BK, u.t * BM, &s.full[st], pol_a);
                if (pr.nslices > 1) tc::tma_load_2d(sa + A_TILE, &P.tmA[u.p][1], u.c * BK, u.t * BM, &s.full[st], pol_a);
                tc::tma_load_2d(sa + (size_t)A_TILE * P.nsmax, &P.tmP[u.p], u.c * BK, 0, &s.full[st], pol_b);
                ro.last_issued = (int)ro.pc;
                ++ro.pc;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (long long g = u0; g < u1; ++g) {
                const Unit u = decode(s, P, g);
                const ProbDev& pr = P.prob[u.p];
                const bool first = (g == u0) || (u.c == 0);
                const bool last = (g == u1 - 1) || (u.c == pr.chunks - 1);
                if (first) {
                    if (!tc::mbar_wait(&s.acc_empty, (ro.rc & 1) ^ 1)) {
                        atomicOr(P.err, 1);
                        break;
                    }
                    tc::tc_fence_after();
                }
                const int st = ro.pc % S;
                const uint32_t ph = (ro.pc / S) & 1;
                if (!tc::mbar_wait(&s.full[st], ph)) {
                    atomicOr(P.err, 1);
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_addr(base + (size_t)st * stage_bytes);
                const uint32_t sb = sa + A_TILE * P.nsmax;
                const uint32_t id_all = tc::idesc_bf16_f32(BM, 2 * pr.nr);
                const uint32_t id_hi = tc::idesc_bf16_f32(BM, pr.nr);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    tc::mma_bf16(s.tmem_base, tc::sdesc_sw128(sa + kk * 32), tc::sdesc_sw128(sb + kk * 32), id_all,
                                 (first && kk == 0) ? 0u : 1u);
                    if (pr.nslices > 1)
                        tc::mma_bf16(s.tmem_base + pr.nr, tc::sdesc_sw128(sa + A_TILE + kk * 32),
                                     tc::sdesc_sw128(sb + kk * 32), id_hi, 1u);
                }
                tc::mma_commit(&s.empty[st]);
                if (last) {
                    tc::mma_commit(&s.acc_full);
                    ++ro.rc;
                }
                ++ro.pc;
            }
        }
    } else if (warp >= 4) {
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        long long g = u0;
        int r = 0;
        while (g < u1) {
            const Unit u = decode(s, P, g);
            const ProbDev& pr = P.prob[u.p];
            const long long gend = std::min<long long>(u1, g + (pr.chunks - u.c));
            int ok = 1;
            if (lane == 0) ok = tc::mbar_wait(&s.acc_full, ro.rc & 1) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicOr(P.err, 1);
                break;
            }
            __syncwarp();
            tc::tc_fence_after();
            if (r < P.rmax) {
                float* slot = P.slots + ((size_t)(b * P.rmax + r) * P.nrmax) * BM;
                const uint32_t ta = s.tmem_base + ((uint32_t)(quarter * 32) << 16);
                for (int jc = 0; jc < pr.nr; jc += 16) {
                    float a[16], c[16];
                    tc::tmem_ld16(ta + jc, a);
                    tc::tmem_ld16(ta + pr.nr + jc, c);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) __stcg(slot + (size_t)(jc + i) * BM + row, a[i] + c[i]);
                }
            } else if (lane == 0) {
                atomicOr(P.err, 2);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&s.acc_empty);
            ++ro.rc;
            ++r;
            g = gend;
        }
    }
}

// For every row tile of active problem k: the first CTA whose run covers it, that
// run's index, and the number of CTAs contributing (later ones use run 0).
__device__ void owner_table(Ctl& s, const Params& P, int k) {
    __syncthreads();  // earlier readers of the table are done
    const int p = s.act[k];
    const ProbDev& pr = P.prob[p];
    for (int t = threadIdx.x; t < pr.mtiles; t += blockDim.x) {
        const long long g0 = s.ubase[k] + (long long)t * pr.chunks, g1 = g0 + pr.chunks - 1;
        const int bf = owner(g0, s.U, s.geff), bl = owner(g1, s.U, s.geff);
        s.own_first[t] = bf;
        s.own_cnt[t] = bl - bf + 1;
        s.own_r[t] = (int)(tile_ordinal(s, P, g0) - tile_ordinal(s, P, range_start(s.U, s.geff, bf)));
    }
    __syncthreads();
}

// y[i .. i+3] of column j: the sum of the run slots that cover row tile i / 128
__device__ __forceinline__ float4 gather_q(const Ctl& s, const Params& P, int j, int i) {
    const int t = i >> 7, off = i & 127;
    const int bf = s.own_first[t], cnt = s.own_cnt[t];
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int o = 0; o < cnt; ++o) {
        const int sl = (o == 0) ? ((bf)*P.rmax + s.own_r[t]) : ((bf + o) * P.rmax);
        const float4 v = __ldcg(reinterpret_cast<const float4*>(P.slots + ((size_t)sl * P.nrmax + j) * BM + off));
        q.x += v.x;
        q.y += v.y;
        q.z += v.z;
        q.w += v.w;
    }
    return q;
}

__device__ __forceinline__ double block_sum(double v, Ctl& s) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s.red[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < THREADS / 32; ++i) t += s.red[i];
    return t;
}

__device__ __forceinline__ void split_store(__nv_bfloat16* hi, __nv_bfloat16* lo, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    *hi = h;
    *lo = l;
}

// One CG step for every unfinished column of the active problems, a CTA per column.
__device__ void vector_phase(Ctl& s, const Params& P, int b, int G) {
    int total = 0;
    for (int k = 0; k < s.na; ++k) total += P.prob[s.act[k]].nr;
    int cached_k = -1;
    for (int ci = b; ci < total; ci += G) {
        int k = 0, j = ci;
        while (j >= P.prob[s.act[k]].nr) j -= P.prob[s.act[k++]].nr;
        const int p = s.act[k];
        const ProbDev& pr = P.prob[p];
        ColState* cs = pr.col + j;
        if (__ldcg(&cs->done)) continue;
        // column state, read before any thread of the block can update it
        const double rr = __ldcg(&cs->rr), rr0 = __ldcg(&cs->rr0);
        const int its = __ldcg(&cs->its) + 1;
        if (k != cached_k) {
            owner_table(s, P, k);
            cached_k = k;
        }
        const int rows = pr.mtiles * BM;
        float* pv = pr.p + (size_t)j * pr.ldv;
        float* qv = pr.q + (size_t)j * pr.ldv;
        float* rv = pr.r + (size_t)j * pr.ldv;
        float* zv = pr.z + (size_t)j * pr.ldv;
        // q = Ã p from the run slots; p.q
        double pq = 0.0;
        for (int i = threadIdx.x * 4; i < rows; i += THREADS * 4) {
            const float4 q = gather_q(s, P, j, i);
            const float4 pp = __ldcg(reinterpret_cast<const float4*>(pv + i));
            pq += (double)pp.x * q.x + (double)pp.y * q.y + (double)pp.z * q.z + (double)pp.w * q.w;
            __stcg(reinterpret_cast<float4*>(qv + i), q);
        }
        pq = block_sum(pq, s);
        if (!(pq > 0.0)) {
            if (threadIdx.x == 0) {
                __stcg(&cs->done, 1);
                __stcg(&cs->status, (int)FL_ENOTSPD);
                atomicAdd(P.ndone + p, 1);
            }
            continue;
        }
        const float alpha = (float)(rr / pq);
        double rn = 0.0;
        for (int i = threadIdx.x * 4; i < rows; i += THREADS * 4) {
            const float4 pp = __ldcg(reinterpret_cast<const float4*>(pv + i));
            const float4 q = __ldcg(reinterpret_cast<const float4*>(qv + i));
            float4 z = __ldcg(reinterpret_cast<const float4*>(zv + i));
            float4 r = __ldcg(reinterpret_cast<const float4*>(rv + i));
            z.x = fmaf(alpha, pp.x, z.x);
            z.y = fmaf(alpha, pp.y, z.y);
            z.z = fmaf(alpha, pp.z, z.z);
            z.w = fmaf(alpha, pp.w, z.w);
            r.x = fmaf(-alpha, q.x, r.x);
            r.y = fmaf(-alpha, q.y, r.y);
            r.z = fmaf(-alpha, q.z, r.z);
            r.w = fmaf(-alpha, q.w, r.w);
            rn += (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z + (double)r.w * r.w;
            __stcg(reinterpret_cast<float4*>(zv + i), z);
            __stcg(reinterpret_cast<float4*>(rv + i), r);
        }
        rn = block_sum(rn, s);
        const bool conv = rn <= P.tol2 * rr0;
        if (conv || its >= P.maxit) {
            if (threadIdx.x == 0) {
                __stcg(&cs->its, its);
                __stcg(&cs->rr, rn);
                __stcg(&cs->done, 1);
                __stcg(&cs->status, conv ? (int)FL_OK : (int)FL_ENOTCONV);
                atomicAdd(P.ndone + p, 1);
            }
            continue;
        }
        const float beta = (float)(rn / rr);
        __nv_bfloat16* Ph = pr.P + (size_t)j * pr.ldv;
        __nv_bfloat16* Pl = pr.P + (size_t)(pr.nr + j) * pr.ldv;
        for (int i = threadIdx.x * 4; i < rows; i += THREADS * 4) {
            const float4 r = __ldcg(reinterpret_cast<const float4*>(rv + i));
            float4 pp = __ldcg(reinterpret_cast<const float4*>(pv + i));
            pp.x = fmaf(beta, pp.x, r.x);
            pp.y = fmaf(beta, pp.y, r.y);
            pp.z = fmaf(beta, pp.z, r.z);
            pp.w = fmaf(beta, pp.w, r.w);
            __stcg(reinterpret_cast<float4*>(pv + i), pp);
            __nv_bfloat16 h[4], l[4];
            split_store(&h[0], &l[0], pp.x);
            split_store(&h[1], &l[1], pp.y);
            split_store(&h[2], &l[2], pp.z);
            split_store(&h[3], &l[3], pp.w);
            uint2 hv, lv;
            memcpy(&hv, h, 8);
            memcpy(&lv, l, 8);
            __stcg(reinterpret_cast<uint2*>(Ph + i), hv);
            __stcg(reinterpret_cast<uint2*>(Pl + i), lv);
        }
        if (threadIdx.x == 0) {
            __stcg(&cs->its, its);
            __stcg(&cs->rr, rn);
        }
    }
    tc::fence_proxy_async_global();
}

__device__ void setup(Ctl& s, const Params& P) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < P.stages; ++i) {
            tc::mbar_init(&s.full[i], 1);
            tc::mbar_init(&s.empty[i], 1);
        }
        tc::mbar_init(&s.acc_full, 1);
        tc::mbar_init(&s.acc_empty, 4);
        tc::mbar_init(&s.drain, 1);
        tc::mbar_fence_init();
        for (int p = 0; p < P.nprob; ++p) {
            tc::tma_prefetch(&P.tmA[p][0]);
            if (P.prob[p].nslices > 1) tc::tma_prefetch(&P.tmA[p][1]);
            tc::tma_prefetch(&P.tmP[p]);
        }
    }
    if (warp == 1) {
        tc::tmem_alloc(&s.tmem_base, (uint32_t)P.tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
}

// Wait (bounded) for every copy and MMA this CTA started, then free tensor memory.
__device__ void teardown(Ctl& s, const Params& P, const Roles& ro) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0 && ro.last_issued >= 0) {
        const int S = P.stages;
        for (int k = 0; k < S; ++k) {
            const int pc = ro.last_issued - k;
            if (pc < 0) break;
            if (!tc::mbar_wait(&s.full[pc % S], (uint32_t)(pc / S) & 1)) atomicOr(P.err, 1);
        }
    }
    if (warp == 1 && lane == 0) {
        tc::mma_commit(&s.drain);
        if (!tc::mbar_wait(&s.drain, 0)) atomicOr(P.err, 1);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(s.tmem_base, (uint32_t)P.tmem_cols);
}

// One GEMM phase over the problems flagged in P.active (the standalone product).
__global__ void __launch_bounds__(THREADS, 1) gemm_kernel(const __grid_constant__ Params P) {
    __shared__ Ctl s;
    setup(s, P);
    Roles ro;
    plan_phase(s, P, gridDim.x, false);
    gemm_phase(s, P, blockIdx.x, ro);
    __syncthreads();
    teardown(s, P, ro);
}

// Persistent CG: GEMM phase, grid barrier, vector phase, grid barrier, until every
// column of every problem has converged or P.maxit steps were taken.
__global__ void __launch_bounds__(THREADS, 1) cg_kernel(const __grid_constant__ Params P) {
    __shared__ Ctl s;
    setup(s, P);
    Roles ro;
    const int G = gridDim.x;
    int it = 0;
    for (; it < P.maxit; ++it) {
        plan_phase(s, P, G, true);
        if (s.na == 0) break;
        gemm_phase(s, P, blockIdx.x, ro);
        if (!tc::grid_barrier(P.gbar, G, P.err)) break;
        if (__ldcg(P.err) != 0) break;
        vector_phase(s, P, blockIdx.x, G);
        if (!tc::grid_barrier(P.gbar, G, P.err)) break;
        if (__ldcg(P.err) != 0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.iters = it;
    __syncthreads();
    teardown(s, P, ro);
}

// ----------------------------------------------------- standalone product --
// Slots -> Y[j][i] (float32, rhs-major) for one problem.
__global__ void slots_reduce_kernel(const __grid_constant__ Params P, int G, float* Y, int64_t ldy) {
    __shared__ Ctl s;
    plan_phase(s, P, G, false);
    const int j = blockIdx.x;
    owner_table(s, P, 0);
    const ProbDev& pr = P.prob[s.act[0]];
    for (int i = threadIdx.x * 4; i < pr.mtiles * BM; i += blockDim.x * 4) {
        const float4 q = gather_q(s, P, j, i);
        const float v[4] = {q.x, q.y, q.z, q.w};
        for (int e = 0; e < 4; ++e)
            if (i + e < pr.n) Y[(size_t)j * ldy + i + e] = v[e];
    }
}

// X (float32, [nr][ldx]) -> P = [x_hi ; x_lo] (bf16, [2 nr][ldv]), zero beyond n.
__global__ void split_vec_kernel(int n, int nr, int ldv, int rows, const float* X, int64_t ldx,
                                 __nv_bfloat16* Pb) {
    const int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const float v = (i < n) ? X[(size_t)j * ldx + i] : 0.f;
        split_store(Pb + (size_t)j * ldv + i, Pb + (size_t)(nr + j) * ldv + i, v);
    }
}

// ------------------------------------------------- slices of the matrix --
// float64 -> bfloat16, round to nearest, ties to even, in one rounding (written from
// the binary formats: 7 stored significand bits kept, the 45 dropped bits rounded).
// Magnitudes below 2^-126 flush to zero.
__device__ __forceinline__ uint16_t bf16_bits_rn(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(u >> 63) << 15;
    const int e = (int)((u >> 52) & 0x7ff);
    const unsigned long long m = u & ((1ull << 52) - 1);
    const int eb = e - 1023 + 127;
    if (e == 0 || eb <= 0) return (uint16_t)sign;
    if (eb >= 255) return (uint16_t)(sign | 0x7f80u);
    const uint32_t keep = (uint32_t)(m >> 45);
    const unsigned long long rem = m & ((1ull << 45) - 1), half = 1ull << 44;
    uint32_t bits = ((uint32_t)eb << 7) | keep;
    if (rem > half || (rem == half && (keep & 1u))) ++bits;
    return (uint16_t)(sign | bits);
}
__device__ __forceinline__ double bf16_value(uint16_t b) {
    return (double)__uint_as_float((uint32_t)b << 16);
}

__global__ void dscale_kernel(int64_t n, const double* A, int64_t lda, double* d) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = 1.0 / sqrt(A[i * lda + i]);
}

// S_0 = bf16(Ã), S_1 = bf16(Ã - S_0) with Ã_ij = (d_i d_j) a_ij (exactly symmetric)
__global__ void split_matrix_kernel(int64_t n, const double* A, int64_t lda, const double* d, int nslices,
                                    uint16_t* S, int64_t lds) {
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        const double di = d[i];
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x) {
            const double a = A[i * lda + j] * (di * d[j]);
            const uint16_t h = bf16_bits_rn(a);
            S[i * lds + j] = h;
            if (nslices > 1) S[n * lds + i * lds + j] = bf16_bits_rn(a - bf16_value(h));
        }
    }
}

// ------------------------------------------------- float64 refinement --
constexpr int RES_ROWS = 16, RES_COLS = 64, RES_K = 32, RES_THREADS = 128;

struct RefProb {
    int n, nrhs, nrp;
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* U;
    int64_t ldu;
    const double* d;
    double* R;      // [n][nrp]
    double* rpart;  // [ceil(n/16)][nrp]
    ColOuter* co;   // [nrp]
    int* odone;     // outer-finished columns
};
struct RefParams {
    RefProb prob[MAXP];
    int nprob;
};

// R = B - A U (U = 0 on the first pass: R = B), per 16-row block the column sums of R^2.
__global__ void __launch_bounds__(RES_THREADS) residual_kernel(const __grid_constant__ RefParams RP, int zero_u) {
    const RefProb& pr = RP.prob[blockIdx.z];
    const int r0 = blockIdx.x * RES_ROWS, c0 = blockIdx.y * RES_COLS;
    if (r0 >= pr.n || c0 >= pr.nrp || __ldcg(pr.odone) >= pr.nrhs) return;
    __shared__ double As[RES_ROWS][RES_K + 1];
    __shared__ double Us[RES_K][RES_COLS];
    __shared__ double Rs[RES_ROWS][RES_COLS + 1];
    const int t = threadIdx.x, row = t >> 3, cl = t & 7;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (!zero_u) {
        for (int k0 = 0; k0 < pr.n; k0 += RES_K) {
            for (int e = t; e < RES_ROWS * RES_K; e += RES_THREADS) {
                const int rr = e / RES_K, kk = e % RES_K;
                const int i = r0 + rr, k = k0 + kk;
                As[rr][kk] = (i < pr.n && k < pr.n) ? pr.A[(int64_t)i * pr.lda + k] : 0.0;
            }
            for (int e = t; e < RES_K * RES_COLS; e += RES_THREADS) {
                const int kk = e / RES_COLS, cc = e % RES_COLS;
                const int k = k0 + kk, c = c0 + cc;
                Us[kk][cc] = (k < pr.n && c < pr.nrhs) ? pr.U[(int64_t)k * pr.ldu + c] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < RES_K; ++kk) {
                const double a = As[row][kk];
#pragma unroll
                for (int m = 0; m < 8; ++m) acc[m] = fma(a, Us[kk][cl + 8 * m], acc[m]);
            }
            __syncthreads();
        }
    }
    const int i = r0 + row;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int c = c0 + cl + 8 * m;
        double v = 0.0;
        if (i < pr.n && c < pr.nrhs) v = pr.B[(int64_t)i * pr.ldb + c] - acc[m];
        if (i < pr.n && c < pr.nrp) pr.R[(int64_t)i * pr.nrp + c] = v;
        Rs[row][cl + 8 * m] = v;
    }
    __syncthreads();
    if (t < RES_COLS && c0 + t < pr.nrp) {
        double ss = 0.0;
        for (int rr = 0; rr < RES_ROWS; ++rr) ss += Rs[rr][t] * Rs[rr][t];
        pr.rpart[(int64_t)blockIdx.x * pr.nrp + c0 + t] = ss;
    }
}

// ------------------------------------------------- double-float residual --
// R = B - A U with A and U in float64, evaluated on the float32 pipe in
// double-float arithmetic: every float64 operand is split into hi + lo float32
// parts (hi = fl32(x), lo = fl32(x - hi)), the product a_hi u_hi is formed
// exactly (hi part by a float32 multiply, its rounding error by an FMA), the
// cross terms a_hi u_lo + a_lo u_hi are added to it in float32, and the running
// sum is kept as an unevaluated pair (s_hi, s_lo) updated with the error-free
// two-sum.  Relative accuracy of each product and addition is about 2^-48.
// Work items are (column tile, 128-row block, 32-wide K chunk); contiguous ranges
// of them go to the CTAs (balanced to one chunk; never more CTAs than items, so no
// range is empty), and every CTA writes one partial (s_hi, s_lo) tile per row
// block it touched.
constexpr int DF_ROWS = 128, DF_COLS = 64, DF_K = 32, DF_THREADS = 256;
constexpr size_t DF_SMEM = (size_t)DF_K * (DF_ROWS + 1) * sizeof(float2) + (size_t)DF_K * DF_COLS * sizeof(float2);

struct DfProb {
    int n, nrhs, nrp, rblocks, kch, ctiles;
    const double* A;
    int64_t lda;
    const double* U;
    int64_t ldu;
};
struct DfParams {
    DfProb prob[MAXP];
    int na, rmax;
    int act[MAXP];
    long long ubase[MAXP + 1], tbase[MAXP + 1];
    float2* slots;  // [G][rmax][DF_COLS][DF_ROWS]
    int* err;
};

struct DfUnit {
    int k, p, ct, rb, kc;
};
__device__ __forceinline__ DfUnit df_decode(const DfParams& D, long long g) {
    int k = 0;
    while (k + 1 < D.na && g >= D.ubase[k + 1]) ++k;
    const int p = D.act[k];
    const DfProb& pr = D.prob[p];
    long long l = g - D.ubase[k];
    const int kc = (int)(l % pr.kch);
    l /= pr.kch;
    return {k, p, (int)(l / pr.rblocks), (int)(l % pr.rblocks), kc};
}
__device__ __forceinline__ long long df_tile(const DfParams& D, long long g) {
    const DfUnit u = df_decode(D, g);
    return D.tbase[u.k] + (long long)u.ct * D.prob[u.p].rblocks + u.rb;
}

__device__ __forceinline__ void df_split(double x, float2& v) {
    const float hi = __double2float_rn(x);
    v = make_float2(hi, __double2float_rn(x - (double)hi));
}

// (sh, sl) += (ah + al)(uh + ul), dropping al ul
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float uh, float ul) {
    const float p = __fmul_rn(ah, uh);
    const float e = __fmaf_rn(ah, uh, -p);
    const float l = __fmaf_rn(ah, ul, __fmaf_rn(al, uh, e));
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, l));
}

__global__ void __launch_bounds__(DF_THREADS, 2) residual_df_kernel(const __grid_constant__ DfParams D) {
    extern __shared__ float2 df_smem[];
    float2(*As)[DF_ROWS + 1] = reinterpret_cast<float2(*)[DF_ROWS + 1]>(df_smem);
    float2(*Us)[DF_COLS] = reinterpret_cast<float2(*)[DF_COLS]>(df_smem + DF_K * (DF_ROWS + 1));
    const int b = blockIdx.x, G = gridDim.x;
    const long long Utot = D.ubase[D.na];
    const long long u0 = range_start(Utot, G, b), u1 = range_start(Utot, G, b + 1);
    const int t = threadIdx.x, rg = t & 15, cg = t >> 4;
    float sh[8][4], sl[8][4];
    int r = 0;
    for (long long g = u0; g < u1; ++g) {
        const DfUnit u = df_decode(D, g);
        const DfProb& pr = D.prob[u.p];
        if (g == u0 || u.kc == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
        }
        const int r0 = u.rb * DF_ROWS, k0 = u.kc * DF_K, c0 = u.ct * DF_COLS;
        for (int e = t; e < DF_ROWS * DF_K; e += DF_THREADS) {
            const int row = e >> 5, kk = e & 31;
            const int i = r0 + row, kcol = k0 + kk;
            df_split((i < pr.n && kcol < pr.n) ? pr.A[(int64_t)i * pr.lda + kcol] : 0.0, As[kk][row]);
        }
        for (int e = t; e < DF_K * DF_COLS; e += DF_THREADS) {
            const int kk = e >> 6, c = e & 63;
            const int krow = k0 + kk, col = c0 + c;
            df_split((krow < pr.n && col < pr.nrhs) ? pr.U[(int64_t)krow * pr.ldu + col] : 0.0, Us[kk][c]);
        }
        __syncthreads();
#pragma unroll 1
        for (int kk = 0; kk < DF_K; ++kk) {
            float2 a[8], v[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][rg + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = Us[kk][cg + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) df_fma(sh[i][j], sl[i][j], a[i].x, a[i].y, v[j].x, v[j].y);
        }
        __syncthreads();
        if (g == u1 - 1 || u.kc == pr.kch - 1) {
            if (r < D.rmax) {
                float2* slot = D.slots + (size_t)(b * D.rmax + r) * DF_COLS * DF_ROWS;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        slot[(cg + 16 * j) * DF_ROWS + rg + 16 * i] = make_float2(sh[i][j], sl[i][j]);
            } else if (t == 0) {
                atomicOr(D.err, 2);
            }
            ++r;
        }
    }
}

// Sum the partial tiles of each (problem, column tile, row block) in a fixed order:
// R = B - sum (float64), and the column sums of R^2 per 16-row block.
// Block (row block, column tile, active problem index).
__global__ void __launch_bounds__(256) residual_df_reduce_kernel(const __grid_constant__ DfParams D,
                                                                 const __grid_constant__ RefParams RP, int G) {
    const int k = blockIdx.z;
    if (k >= D.na) return;
    const int p = D.act[k];
    const DfProb& pr = D.prob[p];
    const RefProb& rp = RP.prob[p];
    const int rb = blockIdx.x, ct = blockIdx.y;
    if (rb >= pr.rblocks || ct >= pr.ctiles) return;
    __shared__ double Rs[DF_ROWS][DF_COLS / 2 + 1];
    __shared__ int own[3];
    const long long Utot = D.ubase[D.na];
    if (threadIdx.x == 0) {
        const long long g0 = D.ubase[k] + ((long long)ct * pr.rblocks + rb) * pr.kch, g1 = g0 + pr.kch - 1;
        const int bf = owner(g0, Utot, G), bl = owner(g1, Utot, G);
        own[0] = bf;
        own[1] = bl - bf + 1;
        own[2] = (int)(df_tile(D, g0) - df_tile(D, range_start(Utot, G, bf)));
    }
    __syncthreads();
    constexpr int HC = DF_COLS / 2;  // columns per half
    const int row = threadIdx.x & 127, sub = threadIdx.x >> 7;
    const int i = rb * DF_ROWS + row;
    for (int half = 0; half < 2; ++half) {
        for (int cc = sub; cc < HC; cc += 2) {
            const int c = half * HC + cc;
            double sum = 0.0;
            for (int o = 0; o < own[1]; ++o) {
                const int sl = (o == 0) ? (own[0] * D.rmax + own[2]) : ((own[0] + o) * D.rmax);
                const float2 v = D.slots[((size_t)sl * DF_COLS + c) * DF_ROWS + row];
                sum += (double)v.x + (double)v.y;
            }
            const int col = ct * DF_COLS + c;
            double rv = 0.0;
            if (i < pr.n && col < pr.nrhs) rv = rp.B[(int64_t)i * rp.ldb + col] - sum;
            Rs[row][cc] = rv;
        }
        __syncthreads();
        // coalesced row-major store of R, then per 16-row block column sums of squares
        for (int e = threadIdx.x; e < DF_ROWS * HC; e += blockDim.x) {
            const int rr = e / HC, c = e % HC;
            const int ii = rb * DF_ROWS + rr, col = ct * DF_COLS + half * HC + c;
            if (ii < pr.n && col < pr.nrp) rp.R[(int64_t)ii * pr.nrp + col] = Rs[rr][c];
        }
        for (int e = threadIdx.x; e < (DF_ROWS / RES_ROWS) * HC; e += blockDim.x) {
            const int sb = e / HC, c = e % HC;
            const int col = ct * DF_COLS + half * HC + c, blk = rb * (DF_ROWS / RES_ROWS) + sb;
            if (col >= pr.nrp || blk * RES_ROWS >= pr.n) continue;
            double ss = 0.0;
            for (int rr = 0; rr < RES_ROWS; ++rr) ss += Rs[sb * RES_ROWS + rr][c] * Rs[sb * RES_ROWS + rr][c];
            rp.rpart[(int64_t)blk * pr.nrp + col] = ss;
        }
        __syncthreads();
    }
}

// Per column: relative residual, convergence, and the start of the next inner solve
// (r = D R_j in float32, z = 0, p = r, P = split(p)).  Block (j, problem).
__global__ void __launch_bounds__(256) prep_kernel(const __grid_constant__ RefParams RP,
                                                   const __grid_constant__ Params P, int first, double tol,
                                                   int last_pass, int* odone_total) {
    const int pi = blockIdx.y, j = blockIdx.x;
    const RefProb& rp = RP.prob[pi];
    const ProbDev& pr = P.prob[pi];
    if (j >= pr.nr) return;
    __shared__ double red[8];
    __shared__ int fresh, decide;
    ColOuter* co = rp.co + j;
    ColState* cs = pr.col + j;
    // fresh: this column's residual was recomputed in this pass (not finished before,
    // and its problem not skipped by the residual kernel)
    if (threadIdx.x == 0) fresh = (co->odone == 0 && __ldcg(rp.odone) < rp.nrhs) ? 1 : 0;
    __syncthreads();
    if (fresh) {
        const int nrb = (rp.n + RES_ROWS - 1) / RES_ROWS;
        double ss = 0.0;
        for (int k = threadIdx.x; k < nrb; k += blockDim.x) ss += rp.rpart[(int64_t)k * rp.nrp + j];
        ss = warp_sum(ss);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
            if (first) co->bb = tot;
            const double bb = co->bb;
            const double rel = (bb > 0.0) ? sqrt(tot / bb) : 0.0;
            co->rel = rel;
            int od = 0;
            if (j >= rp.nrhs || rel <= tol) {
                od = 1;
                co->status = FL_OK;
            } else if (!first && cs->status == FL_ENOTSPD) {
                od = 1;
                co->status = FL_ENOTSPD;
            } else {
                co->status = FL_ENOTCONV;
            }
            if (od) {
                co->odone = 1;
                if (j < rp.nrhs) {
                    atomicAdd(rp.odone, 1);
                    atomicAdd(odone_total, 1);
                }
            }
            decide = od;
        }
        __syncthreads();
    } else {
        if (threadIdx.x == 0) decide = 1;
        __syncthreads();
    }
    if (decide || last_pass) {
        if (threadIdx.x == 0) {
            cs->done = 1;
            atomicAdd(P.ndone + pi, 1);
        }
        return;
    }
    // start of the inner solve
    const int rows = pr.mtiles * BM;
    double rr = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const float v = (i < pr.n) ? (float)(rp.d[i] * rp.R[(int64_t)i * rp.nrp + j]) : 0.f;
        pr.r[(size_t)j * pr.ldv + i] = v;
        pr.p[(size_t)j * pr.ldv + i] = v;
        pr.z[(size_t)j * pr.ldv + i] = 0.f;
        split_store(pr.P + (size_t)j * pr.ldv + i, pr.P + (size_t)(pr.nr + j) * pr.ldv + i, v);
        rr += (double)v * v;
    }
    rr = warp_sum(rr);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        cs->rr = tot;
        cs->rr0 = tot;
        cs->its = 0;
        cs->status = FL_OK;
        cs->done = (tot > 0.0) ? 0 : 1;
        if (!(tot > 0.0)) atomicAdd(P.ndone + pi, 1);
    }
    tc::fence_proxy_async_global();
}

// U_j += D z_j for the columns still iterating.  Block (j, problem).
__global__ void update_kernel(const __grid_constant__ RefParams RP, const __grid_constant__ Params P) {
    const int pi = blockIdx.y, j = blockIdx.x;
    const RefProb& rp = RP.prob[pi];
    const ProbDev& pr = P.prob[pi];
    if (j >= rp.nrhs || rp.co[j].odone) return;
    for (int i = threadIdx.x; i < rp.n; i += blockDim.x)
        rp.U[(int64_t)i * rp.ldu + j] += rp.d[i] * (double)pr.z[(size_t)j * pr.ldv + i];
}

__global__ void zero_u_kernel(const __grid_constant__ RefParams RP) {
    const RefProb& rp = RP.prob[blockIdx.y];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rp.n * rp.nrhs;
         e += (int64_t)gridDim.x * blockDim.x)
        rp.U[(e / rp.nrhs) * rp.ldu + e % rp.nrhs] = 0.0;
}

// ------------------------------------------------------------------ host --
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

static EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    });
    return fn;
}

// 2D bf16 tensor [rows][cols] with row pitch ld elements, tile box (64 x box_rows),
// 128-byte swizzle, zero fill outside.
static bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    if (((uintptr_t)base & 15) != 0 || (ld * 2) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int round_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b * b); }

struct Geometry {
    int G = 0, stages = 0, rmax = 0, nrmax = 0, nsmax = 0, tmem_cols = 0;
    size_t smem = 0;
};

static int tmem_cols_for(int nrmax) {
    int c = 32;
    while (c < 2 * nrmax) c <<= 1;
    return c;
}

// Grid, pipeline depth and run-slot bound for a set of problems.
static bool geometry(const std::vector<ProbDev>& pr, int sms, int want_ctas, int want_stages, Geometry& g) {
    long long U = 0;
    int chmin = 1 << 30;
    for (const ProbDev& p : pr) {
        g.nrmax = std::max(g.nrmax, p.nr);
        g.nsmax = std::max(g.nsmax, p.nslices);
        U += (long long)p.mtiles * p.chunks;
        chmin = std::min(chmin, p.chunks);
    }
    g.G = (want_ctas > 0) ? std::min(want_ctas, sms) : sms;
    const size_t stage_bytes = (size_t)A_TILE * g.nsmax + (size_t)g.nrmax * 2 * BK * 2;
    const size_t budget = 220 * 1024;
    int st = (int)std::min<size_t>(MAX_STAGES, (budget - 1024) / stage_bytes);
    if (want_stages > 0) st = std::min(st, want_stages);
    if (st < 2) return false;
    g.stages = st;
    g.smem = (size_t)st * stage_bytes + 1024;
    // runs per CTA: chunks of at most ceil(U / G_eff) + 1 consecutive units, each run
    // within one tile; U / G_eff <= max(U / G, 2 UMIN) for any subset of problems
    const long long per = std::max<long long>((U + g.G - 1) / g.G, 2 * UMIN) + 1;
    g.rmax = (int)((per + chmin - 1) / chmin) + 1;
    g.tmem_cols = tmem_cols_for(g.nrmax);
    return true;
}

static bool launch_cfg(const void* fn, size_t smem) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

}  // namespace bt
}  // namespace fl

using namespace fl;
using namespace fl::bt;

extern "C" {

int fl_split_bf16(const double* A_dev, int64_t lda, int64_t n, int nslices, void* S_dev, int64_t lds,
                  double* dscale_dev, void* stream) {
    if (!A_dev || !S_dev || !dscale_dev || n < 1 || n > 65536 || lda < n || lds < n || (lds % 8) != 0 ||
        (nslices != 1 && nslices != 2) || ((uintptr_t)S_dev & 15) != 0)
        return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    dscale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, A_dev, lda, dscale_dev);
    fl::count_launch();
    dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 32), (unsigned)std::min<int64_t>(n, 65535));
    split_matrix_kernel<<<grid, 256, 0, st>>>(n, A_dev, lda, dscale_dev, nslices, (uint16_t*)S_dev, lds);
    fl::count_launch();
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

int fl_matmul_bf16(const void* S_dev, int64_t lds, int64_t n, int nslices, int nrhs, const float* X_dev,
                   int64_t ldx, float* Y_dev, int64_t ldy, void* stream) {
    if (!S_dev || !X_dev || !Y_dev || n < 1 || n > 65536 || lds < n || (lds % 8) != 0 || ldx < n || ldy < n ||
        nrhs < 16 || nrhs > 128 || (nrhs % 16) != 0 || (nslices != 1 && nslices != 2) ||
        ((uintptr_t)S_dev & 15) != 0)
        return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ProbDev pd{};
    pd.n = (int)n;
    pd.nr = nrhs;
    pd.nslices = nslices;
    pd.mtiles = (int)((n + BM - 1) / BM);
    pd.chunks = (int)((n + BK - 1) / BK);
    pd.ldv = round_up(pd.mtiles * BM, 64);
    Geometry g;
    if (!geometry({pd}, sms, 0, 0, g)) return FL_EINVAL;
    // G: enough CTAs that each takes at least 2 UMIN chunks
    const long long U = (long long)pd.mtiles * pd.chunks;
    g.G = (int)std::max<long long>(1, std::min<long long>(sms, U / (2 * UMIN)));
    {
        const long long per = std::max<long long>((U + g.G - 1) / g.G, 2 * UMIN) + 1;
        g.rmax = (int)((per + pd.chunks - 1) / pd.chunks) + 1;
    }
    const size_t pbytes = (size_t)2 * nrhs * pd.ldv * sizeof(__nv_bfloat16);
    const size_t sbytes = (size_t)g.G * g.rmax * g.nrmax * BM * sizeof(float);
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, pbytes + sbytes + 256, st) != cudaSuccess) return FL_ENOMEM;
    char* c = (char*)ws;
    pd.P = (__nv_bfloat16*)c;
    float* slots = (float*)(c + ((pbytes + 255) & ~size_t(255)));
    int* flags = nullptr;
    if (cudaMallocAsync((void**)&flags, 256, st) != cudaSuccess) {
        cudaFreeAsync(ws, st);
        return FL_ENOMEM;
    }
    static Params P;  // large (tensor maps); filled under a lock
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    memset(&P, 0, sizeof(P));
    P.nprob = 1;
    P.prob[0] = pd;
    P.stages = g.stages;
    P.rmax = g.rmax;
    P.nrmax = g.nrmax;
    P.nsmax = g.nsmax;
    P.tmem_cols = g.tmem_cols;
    P.maxit = 1;
    P.slots = slots;
    P.err = flags;
    P.active = flags + 16;
    P.ndone = flags + 32;
    P.iters = flags + 48;
    int rc = FL_OK;
    if (!make_map(&P.tmA[0][0], S_dev, n, n, lds, BM) ||
        (nslices > 1 && !make_map(&P.tmA[0][1], (const uint16_t*)S_dev + n * lds, n, n, lds, BM)) ||
        !make_map(&P.tmP[0], pd.P, 2 * nrhs, n, pd.ldv, 2 * nrhs)) {
        rc = FL_EINVAL;
    } else {
        const int one = 1;
        cudaMemsetAsync(flags, 0, 256, st);
        cudaMemcpyAsync(P.active, &one, sizeof(int), cudaMemcpyHostToDevice, st);
        split_vec_kernel<<<dim3(16, nrhs), 256, 0, st>>>((int)n, nrhs, pd.ldv, pd.mtiles * BM, X_dev, ldx, pd.P);
        fl::count_launch();
        if (!launch_cfg((const void*)gemm_kernel, g.smem)) {
            rc = FL_ECUDA;
        } else {
            gemm_kernel<<<g.G, THREADS, g.smem, st>>>(P);
            fl::count_launch();
            slots_reduce_kernel<<<nrhs, THREADS, 0, st>>>(P, g.G, Y_dev, ldy);
            fl::count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = FL_ECUDA;
        }
        int err = 0;
        if (rc == FL_OK) {
            if (cudaMemcpyAsync(&err, flags, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = FL_ECUDA;
            else if (err != 0)
                rc = FL_ETIMEOUT;
        }
    }
    cudaFreeAsync(flags, st);
    cudaFreeAsync(ws, st);
    return rc;
}

void fl_default_batch_opts(fl_batch_opts* o) {
    if (!o) return;
    o->tol = 1e-8;
    o->max_outer = 8;
    o->inner_tol = 1e-5;
    o->inner_maxit = 5000;
    o->ctas = 0;
    o->stages = 0;
    o->residual = FL_RESID_DF;
}

int fl_batch_solve(fl_handle h, int nprob, const fl_batch_problem* probs, const fl_batch_opts* o_in,
                   fl_batch_info* info, double* rel_host, int* status_host, void* stream) {
    if (!h) return FL_EINVAL;
    h->err.clear();
    if (nprob < 1 || nprob > MAXP || !probs) return set_err(h, FL_EINVAL, "nprob must lie in [1, FL_BATCH_MAXPROB]");
    fl_batch_opts o;
    fl_default_batch_opts(&o);
    if (o_in) o = *o_in;
    if (!(o.tol > 0) || !(o.inner_tol > 0) || o.max_outer < 1 || o.inner_maxit < 1 ||
        (o.residual != FL_RESID_F64 && o.residual != FL_RESID_DF))
        return set_err(h, FL_EINVAL, "bad batch options");
    for (int p = 0; p < nprob; ++p) {
        const fl_batch_problem& q = probs[p];
        if (q.n < 1 || q.n > 65536 || !q.A_dev || q.lda < q.n || !q.S_dev || q.lds < q.n || (q.lds % 8) != 0 ||
            (q.nslices != 1 && q.nslices != 2) || !q.dscale_dev || q.nrhs < 1 || q.nrhs > 128 || !q.B_dev ||
            q.ldb < q.nrhs || !q.U_dev || q.ldu < q.nrhs || ((uintptr_t)q.S_dev & 15) != 0)
            return set_err(h, FL_EINVAL, "bad batch problem " + std::to_string(p));
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, FL_ECUDA, "cudaSetDevice");
    int sms = 0, coop = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (!coop) return set_err(h, FL_ENOTIMPL, "device without cooperative launch");

    std::vector<ProbDev> pd(nprob);
    for (int p = 0; p < nprob; ++p) {
        const fl_batch_problem& q = probs[p];
        ProbDev& d = pd[p];
        d.n = (int)q.n;
        d.nr = round_up(q.nrhs, 16);
        d.nslices = q.nslices;
        d.mtiles = (d.n + BM - 1) / BM;
        d.chunks = (d.n + BK - 1) / BK;
        d.ldv = round_up((int64_t)d.mtiles * BM, 64);
    }
    Geometry g;
    if (!geometry(pd, sms, o.ctas, o.stages, g)) return set_err(h, FL_EINVAL, "no pipeline fits shared memory");
    int per_sm = 0;
    if (!launch_cfg((const void*)cg_kernel, g.smem) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)cg_kernel, THREADS, g.smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return set_err(h, FL_ECUDA, "persistent CG kernel does not fit on an SM");
    }
    g.G = std::min(g.G, sms * per_sm);

    // workspace layout
    std::vector<size_t> off_vec(nprob), off_P(nprob), off_col(nprob), off_R(nprob), off_rp(nprob), off_co(nprob);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t at = total;
        total += (bytes + 255) & ~size_t(255);
        return at;
    };
    for (int p = 0; p < nprob; ++p) {
        const ProbDev& d = pd[p];
        off_vec[p] = take((size_t)4 * d.nr * d.ldv * sizeof(float));
        off_P[p] = take((size_t)2 * d.nr * d.ldv * sizeof(__nv_bfloat16));
        off_col[p] = take((size_t)d.nr * sizeof(ColState));
        off_R[p] = take((size_t)d.n * d.nr * sizeof(double));
        off_rp[p] = take((size_t)((d.n + RES_ROWS - 1) / RES_ROWS) * d.nr * sizeof(double));
        off_co[p] = take((size_t)d.nr * sizeof(ColOuter));
    }
    const size_t off_slots = take((size_t)g.G * g.rmax * g.nrmax * BM * sizeof(float));
    const size_t off_flags = take(256);
    // double-float residual: grid, run bound and partial tiles
    int df_G = 0, df_rmax = 0;
    size_t off_df = 0;
    if (o.residual == FL_RESID_DF) {
        int occ = 0;
        if (cudaFuncSetAttribute((const void*)residual_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)DF_SMEM) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)residual_df_kernel, DF_THREADS,
                                                          DF_SMEM) != cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            return set_err(h, FL_ECUDA, "double-float residual kernel does not fit on an SM");
        }
        df_G = sms * std::min(occ, 2);
        long long Uall = 0;
        int kmin = 1 << 30;
        for (const ProbDev& d : pd) {
            const int kch = (d.n + DF_K - 1) / DF_K;
            Uall += (long long)((d.nr + DF_COLS - 1) / DF_COLS) * ((d.n + DF_ROWS - 1) / DF_ROWS) * kch;
            kmin = std::min(kmin, kch);
        }
        df_rmax = (int)(((Uall + df_G - 1) / df_G + kmin - 1) / kmin) + 2;
        off_df = take((size_t)df_G * df_rmax * DF_COLS * DF_ROWS * sizeof(float2));
    }
    if (total > h->batch_ws_bytes) {
        if (h->batch_ws) cudaFree(h->batch_ws);
        h->batch_ws = nullptr;
        h->batch_ws_bytes = 0;
        if (cudaMalloc(&h->batch_ws, total) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, FL_ENOMEM, "batch workspace");
        }
        h->batch_ws_bytes = total;
    }
    if (!h->batch_host) {
        if (cudaMallocHost(&h->batch_host, 4096) != cudaSuccess) return set_err(h, FL_ENOMEM, "pinned scalars");
    }
    char* W = (char*)h->batch_ws;
    int* flags = (int*)(W + off_flags);  // [0] err, [1] outer-done total, [2..] barrier, [8..15] ndone, [16..] odone

    static Params P;
    static RefParams RP;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    memset(&P, 0, sizeof(P));
    memset(&RP, 0, sizeof(RP));
    P.nprob = nprob;
    P.stages = g.stages;
    P.rmax = g.rmax;
    P.nrmax = g.nrmax;
    P.nsmax = g.nsmax;
    P.tmem_cols = g.tmem_cols;
    P.maxit = o.inner_maxit;
    P.tol2 = o.inner_tol * o.inner_tol;
    P.slots = (float*)(W + off_slots);
    P.err = flags;
    P.gbar = (unsigned*)(flags + 2);
    P.ndone = flags + 8;
    P.active = flags + 24;
    P.iters = flags + 4;
    RP.nprob = nprob;
    for (int p = 0; p < nprob; ++p) {
        ProbDev& d = pd[p];
        float* v = (float*)(W + off_vec[p]);
        d.r = v;
        d.z = v + (size_t)d.nr * d.ldv;
        d.p = v + (size_t)2 * d.nr * d.ldv;
        d.q = v + (size_t)3 * d.nr * d.ldv;
        d.P = (__nv_bfloat16*)(W + off_P[p]);
        d.col = (ColState*)(W + off_col[p]);
        P.prob[p] = d;
        const fl_batch_problem& q = probs[p];
        if (!make_map(&P.tmA[p][0], q.S_dev, q.n, q.n, q.lds, BM) ||
            (q.nslices > 1 && !make_map(&P.tmA[p][1], (const uint16_t*)q.S_dev + q.n * q.lds, q.n, q.n, q.lds, BM)) ||
            !make_map(&P.tmP[p], d.P, 2 * d.nr, d.n, d.ldv, 2 * d.nr))
            return set_err(h, FL_EINVAL, "tensor map of problem " + std::to_string(p));
        RefProb& r = RP.prob[p];
        r.n = d.n;
        r.nrhs = q.nrhs;
        r.nrp = d.nr;
        r.A = q.A_dev;
        r.lda = q.lda;
        r.B = q.B_dev;
        r.ldb = q.ldb;
        r.U = q.U_dev;
        r.ldu = q.ldu;
        r.d = q.dscale_dev;
        r.R = (double*)(W + off_R[p]);
        r.rpart = (double*)(W + off_rp[p]);
        r.co = (ColOuter*)(W + off_co[p]);
        r.odone = flags + 16 + p;
    }
    int nmax = 0, nrmax = 0;
    for (const ProbDev& d : pd) {
        nmax = std::max(nmax, d.n);
        nrmax = std::max(nrmax, d.nr);
    }
    // column records start clean
    for (int p = 0; p < nprob; ++p) {
        if (cudaMemsetAsync(W + off_co[p], 0, (size_t)pd[p].nr * sizeof(ColOuter), st) != cudaSuccess ||
            cudaMemsetAsync(W + off_col[p], 0, (size_t)pd[p].nr * sizeof(ColState), st) != cudaSuccess)
            return set_err(h, FL_ECUDA, "memset");
    }
    if (cudaMemsetAsync(flags, 0, 256, st) != cudaSuccess) return set_err(h, FL_ECUDA, "memset");
    zero_u_kernel<<<dim3(64, nprob), 256, 0, st>>>(RP);
    fl::count_launch();

    int total_rhs = 0;
    for (int p = 0; p < nprob; ++p) total_rhs += probs[p].nrhs;
    int* hs = (int*)h->batch_host;
    memset(hs, 0, 256);
    int outer = 0, inner_total = 0;
    bool all_done = false;
    for (int pass = 0; pass <= o.max_outer; ++pass) {
        const bool last = (pass == o.max_outer);
        if (pass == 0 || o.residual == FL_RESID_F64) {
            residual_kernel<<<dim3((nmax + RES_ROWS - 1) / RES_ROWS, (nrmax + RES_COLS - 1) / RES_COLS, nprob),
                              RES_THREADS, 0, st>>>(RP, pass == 0 ? 1 : 0);
            fl::count_launch();
        } else {
            DfParams D;
            memset(&D, 0, sizeof(D));
            long long u = 0, tt = 0;
            int rbmax = 0, ctmax = 0;
            for (int p = 0; p < nprob; ++p) {
                DfProb& q = D.prob[p];
                q.n = pd[p].n;
                q.nrhs = probs[p].nrhs;
                q.nrp = pd[p].nr;
                q.rblocks = (q.n + DF_ROWS - 1) / DF_ROWS;
                q.kch = (q.n + DF_K - 1) / DF_K;
                q.ctiles = (q.nrp + DF_COLS - 1) / DF_COLS;
                q.A = probs[p].A_dev;
                q.lda = probs[p].lda;
                q.U = probs[p].U_dev;
                q.ldu = probs[p].ldu;
                if (hs[16 + p] >= probs[p].nrhs) continue;  // every column finished
                D.act[D.na] = p;
                D.ubase[D.na] = u;
                D.tbase[D.na] = tt;
                u += (long long)q.ctiles * q.rblocks * q.kch;
                tt += (long long)q.ctiles * q.rblocks;
                rbmax = std::max(rbmax, q.rblocks);
                ctmax = std::max(ctmax, q.ctiles);
                ++D.na;
            }
            D.ubase[D.na] = u;
            D.tbase[D.na] = tt;
            D.rmax = df_rmax;
            D.slots = (float2*)(W + off_df);
            D.err = flags;
            if (D.na > 0) {
                // at most one CTA per work item, so that every CTA's range is non-empty and
                // the CTAs covering a row block are consecutive
                const int G = (int)std::min<long long>(df_G, u);
                residual_df_kernel<<<G, DF_THREADS, DF_SMEM, st>>>(D);
                residual_df_reduce_kernel<<<dim3(rbmax, ctmax, D.na), 256, 0, st>>>(D, RP, G);
                fl::count_launch(2);
            }
        }
        if (cudaMemsetAsync(P.ndone, 0, MAXP * sizeof(int), st) != cudaSuccess)
            return set_err(h, FL_ECUDA, "memset");
        prep_kernel<<<dim3(nrmax, nprob), 256, 0, st>>>(RP, P, pass == 0 ? 1 : 0, o.tol, last ? 1 : 0, flags + 1);
        fl::count_launch();
        if (cudaGetLastError() != cudaSuccess) return set_err(h, FL_ECUDA, "refinement kernels");
        if (cudaMemcpyAsync(hs, flags, 256, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return set_err(h, FL_ECUDA, "batch scalars");
        if (hs[1] >= total_rhs) {
            all_done = true;
            break;
        }
        if (last) break;
        void* args[] = {(void*)&P};
        const cudaError_t e =
            cudaLaunchCooperativeKernel((const void*)cg_kernel, dim3(g.G), dim3(THREADS), args, g.smem, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, FL_ECUDA, std::string("persistent CG launch: ") + cudaGetErrorString(e));
        }
        fl::count_launch();
        update_kernel<<<dim3(nrmax, nprob), 256, 0, st>>>(RP, P);
        fl::count_launch();
        ++outer;
        if (cudaMemcpyAsync(hs, flags, 256, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return set_err(h, FL_ECUDA, "batch scalars");
        inner_total += hs[4];
        if (hs[0] != 0) return set_err(h, FL_ETIMEOUT, "a bounded device wait gave up (code " + std::to_string(hs[0]) + ")");
    }
    // per-column results
    std::vector<ColOuter> co;
    std::vector<ColState> cs;
    int worst = FL_OK, k = 0;
    for (int p = 0; p < nprob; ++p) {
        co.resize(pd[p].nr);
        cs.resize(pd[p].nr);
        if (cudaMemcpyAsync(co.data(), W + off_co[p], pd[p].nr * sizeof(ColOuter), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return set_err(h, FL_ECUDA, "batch results");
        for (int j = 0; j < probs[p].nrhs; ++j, ++k) {
            const int stt = co[j].odone ? co[j].status : FL_ENOTCONV;
            if (rel_host) rel_host[k] = co[j].rel;
            if (status_host) status_host[k] = stt;
            if (stt != FL_OK && worst == FL_OK) worst = stt;
        }
    }
    if (info) {
        info->outer_iterations = outer;
        info->inner_iterations = inner_total;
        info->status = all_done ? FL_OK : worst;
        info->ctas = g.G;
        info->stages = g.stages;
    }
    return all_done ? FL_OK : (worst == FL_OK ? FL_ENOTCONV : worst);
}

}  // extern "C"
