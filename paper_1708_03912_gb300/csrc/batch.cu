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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

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
constexpr int UMIN = 8;            // fewest chunks a CTA takes in a GEMM phase

struct ColState {
    double gam[2], alp[2];  // gamma = r.r and alpha of the step of even / odd parity (a step reads
                            // the previous step's pair and writes its own)
    double rr0;             // r.r at the start of the inner solve
    int done, its, status, pad;
};
struct ColOuter {
    double bb, rel;  // ||b||^2 and the last relative float64 residual
    int odone, status;
};

// Operand tiles in global memory are stored exactly as the MMA reads them from
// shared memory: 128-byte rows (64 bf16 along K) with the 128-byte swizzle (the
// 16-byte unit u of row r sits at unit position u XOR (r mod 8)), so that one
// contiguous bulk copy moves a whole tile.  Byte offset of element (r, q):
__host__ __device__ constexpr uint32_t sw128(uint32_t r, uint32_t q) {
    return r * 128u + ((((q >> 3) ^ (r & 7u)) << 4)) + (q & 7u) * 2u;
}

struct ProbDev {
    int n, nr, nslices, mtiles, chunks, ldv;
    const uint8_t* S;      // slices: [nslices][mtiles][chunks] tiles of 128 x 64 (16 KiB)
    float *r, *z, *p, *q, *sv;  // [nr][ldv]: residual, solution, direction, w = Ã r, s = Ã p
    __nv_bfloat16* P;      // [2 mtiles] tiles of 2 nr x 64: p_hi rows then p_lo rows (the GEMM reads
                           // the first `chunks`; the vector phases write all mtiles * 128 rows)
    ColState* col;         // [nr]
    float *pq, *rq;        // [nr][ngroups] partial r.w and r.r per group of VT row tiles
    int ngroups;
};

struct Params {
    ProbDev prob[MAXP];
    int nprob, stages, rmax, nrmax, maxit, tmem_cols, nsmax;
    int nacc;  // independent TMEM accumulators the K steps of a chunk rotate over (1, 2 or 4)
    double tol2;
    float* slots;    // [G][rmax][nrmax][128] per-run partial products
    unsigned* gbar;  // grid barrier arrival counter (own cache line, zero at launch)
    unsigned long long barrier_ns;  // bound of each grid-barrier wait
    int* err;        // bit 0: mbarrier timeout, 1: run-slot overflow, 2: grid barrier timeout
    int* ndone;      // [MAXP] finished columns per problem
    int* active;     // [MAXP] (GEMM-only launches): problem takes part
    int* iters;      // CG steps taken by the last persistent launch
    int4* owners;    // per row tile (ordinal over the active problems) of the current GEMM phase:
                     // x = first CTA, y = its run index for the tile, z = last CTA
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
    long long vbase[MAXP + 1];  // vector work items (column, group of row tiles) per active problem
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

// Active problems of this phase, the unit (chunk) numbering over them and the
// number of CTAs that take part in the GEMM.  Run by every CTA on data that no
// CTA modifies during the phase, so all CTAs agree.
__device__ void plan_phase(Ctl& s, const Params& P, int G, bool cg_mode) {
    if (threadIdx.x == 0) {
        int na = 0, tt = 0;
        long long u = 0, vi = 0;
        for (int p = 0; p < P.nprob; ++p) {
            const bool on = cg_mode ? (__ldcg(P.ndone + p) < P.prob[p].nr) : (__ldcg(P.active + p) != 0);
            if (!on) continue;
            s.act[na] = p;
            s.ubase[na] = u;
            s.tbase[na] = tt;
            s.vbase[na] = vi;
            u += (long long)P.prob[p].mtiles * P.prob[p].chunks;
            tt += P.prob[p].mtiles;
            vi += (long long)P.prob[p].nr * P.prob[p].ngroups;
            ++na;
        }
        s.ubase[na] = u;
        s.tbase[na] = tt;
        s.vbase[na] = vi;
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
    uint32_t pc = 0;   // chunks issued (producer) / consumed (MMA)
    uint32_t st = 0;   // stage of chunk pc
    uint32_t ph = 0;   // parity of the ring pass of chunk pc
    uint32_t rc = 0;   // runs accumulated (MMA) / drained (epilogue)
    int last_issued = -1;
    __device__ __forceinline__ void next(int S) {
        ++pc;
        if (++st == (uint32_t)S) {
            st = 0;
            ph ^= 1u;
        }
    }
};

// One GEMM phase: for every active problem, Y = Ã P over its row tiles, the
// chunks (64-wide K slices) of all tiles split into G_eff contiguous ranges, one
// per CTA.  A CTA accumulates consecutive chunks of one tile in tensor memory
// (a "run") and writes each run's 128 x nr product to its slot.  The producer and
// the MMA issuer walk their range with running indices (one division per phase).
__device__ void gemm_phase(Ctl& s, const Params& P, int b, Roles& ro) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (s.U == 0 || b >= s.geff) return;
    const long long u0 = range_start(s.U, s.geff, b), u1 = range_start(s.U, s.geff, b + 1);
    if (u0 >= u1) return;
    const int S = P.stages;
    const uint32_t stage_bytes = A_TILE * P.nsmax + P.nrmax * 2 * BK * 2;
    uint8_t* base = stage_base(S);
    const int nitems = (int)(u1 - u0);

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pol_a = tc::policy_evict_first(), pol_b = tc::policy_evict_last();
            tc::fence_proxy_async_global();
            const Unit u = decode(s, P, u0);
            int k = u.k, t = u.t, c = u.c;
            const ProbDev* pr = &P.prob[u.p];
            uint32_t pbytes = pr->nr * 2 * BK * 2;
            size_t sstride = (size_t)pr->mtiles * pr->chunks * A_TILE;
            const uint8_t* ga = pr->S + ((size_t)t * pr->chunks + c) * A_TILE;
            const uint8_t* gp = reinterpret_cast<const uint8_t*>(pr->P) + (size_t)c * pbytes;
            for (int it = 0; it < nitems; ++it) {
                if (!tc::mbar_wait(&s.empty[ro.st], ro.ph ^ 1)) {
                    atomicOr(P.err, 1);
                    break;
                }
                tc::mbar_arrive_expect_tx(&s.full[ro.st], A_TILE * pr->nslices + pbytes);
                uint8_t* sa = base + ro.st * stage_bytes;
                tc::bulk_load(sa, ga, A_TILE, &s.full[ro.st], pol_a);
                if (pr->nslices > 1) tc::bulk_load(sa + A_TILE, ga + sstride, A_TILE, &s.full[ro.st], pol_a);
                tc::bulk_load(sa + A_TILE * P.nsmax, gp, pbytes, &s.full[ro.st], pol_b);
                ro.last_issued = (int)ro.pc;
                ro.next(S);
                // next chunk: tiles of a problem are consecutive blocks, chunk-major within a tile
                ga += A_TILE;
                gp += pbytes;
                if (++c == pr->chunks) {
                    c = 0;
                    gp = reinterpret_cast<const uint8_t*>(pr->P);
                    if (++t == pr->mtiles && ++k < s.na) {
                        t = 0;
                        pr = &P.prob[s.act[k]];
                        pbytes = pr->nr * 2 * BK * 2;
                        sstride = (size_t)pr->mtiles * pr->chunks * A_TILE;
                        ga = pr->S;
                        gp = reinterpret_cast<const uint8_t*>(pr->P);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const Unit u = decode(s, P, u0);
            int k = u.k, c = u.c, t = u.t;
            const ProbDev* pr = &P.prob[u.p];
            uint32_t id_all = tc::idesc_bf16_f32(BM, 2 * pr->nr), id_hi = tc::idesc_bf16_f32(BM, pr->nr);
            const uint64_t dbase = tc::sdesc_sw128(tc::smem_addr(base));
            bool first = true;
            for (int it = 0; it < nitems; ++it) {
                const bool last = (it == nitems - 1) || (c == pr->chunks - 1);
                if (first) {
                    if (!tc::mbar_wait(&s.acc_empty, (ro.rc & 1) ^ 1)) {
                        atomicOr(P.err, 1);
                        break;
                    }
                    tc::tc_fence_after();
                }
                if (!tc::mbar_wait(&s.full[ro.st], ro.ph)) {
                    atomicOr(P.err, 1);
                    break;
                }
                tc::tc_fence_after();
                // descriptors of this stage: start address field advanced by (offset >> 4)
                const uint64_t da = dbase + ((ro.st * stage_bytes) >> 4);
                const uint64_t db = da + ((A_TILE * P.nsmax) >> 4);
                // K step kk accumulates into accumulator kk mod nacc, so consecutive MMAs do not
                // wait on each other's result; the S_1 products follow all S_0 products of the chunk
                const uint32_t acc_cols = 2 * pr->nr;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint32_t a = kk & (P.nacc - 1);
                    tc::mma_bf16(s.tmem_base + a * acc_cols, da + 2 * kk, db + 2 * kk, id_all,
                                 (first && kk < P.nacc) ? 0u : 1u);
                }
                if (pr->nslices > 1) {
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t a = kk & (P.nacc - 1);
                        tc::mma_bf16(s.tmem_base + a * acc_cols + pr->nr, da + (A_TILE >> 4) + 2 * kk, db + 2 * kk,
                                     id_hi, 1u);
                    }
                }
                tc::mma_commit(&s.empty[ro.st]);
                first = false;
                if (last) {
                    tc::mma_commit(&s.acc_full);
                    ++ro.rc;
                    first = true;
                }
                ro.next(S);
                if (++c == pr->chunks) {
                    c = 0;
                    if (++t == pr->mtiles && ++k < s.na) {
                        t = 0;
                        pr = &P.prob[s.act[k]];
                        id_all = tc::idesc_bf16_f32(BM, 2 * pr->nr);
                        id_hi = tc::idesc_bf16_f32(BM, pr->nr);
                    }
                }
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
            if (quarter == 0 && lane == 0) {
                int4* ow = P.owners + (s.tbase[u.k] + u.t);
                if (u.c == 0) {
                    __stcg(&ow->x, b);
                    __stcg(&ow->y, r);
                }
                if (u.c + (int)(gend - g) == pr.chunks) __stcg(&ow->z, b);
            }
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
                    float y[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) y[i] = 0.f;
                    for (int acc = 0; acc < P.nacc; ++acc) {
                        float a[16], c[16];
                        const uint32_t tacc = ta + acc * 2 * pr.nr;
                        tc::tmem_ld16(tacc + jc, a);
                        tc::tmem_ld16(tacc + pr.nr + jc, c);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 16; ++i) y[i] += a[i] + c[i];
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) __stcg(slot + (size_t)(jc + i) * BM + row, y[i]);
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

// The CTAs whose runs cover row tile t of active problem k: the first one, the
// index of its run for that tile, and how many consecutive CTAs contribute (the
// later ones through their run 0).
struct Owners {
    int first, count, r;
};
__device__ __forceinline__ Owners tile_owners(const Ctl& s, const Params& P, int k, int t) {
    const int4 o = __ldcg(P.owners + (s.tbase[k] + t));
    // entries are written by the GEMM epilogues; anything out of range means a phase did
    // not complete: contribute nothing (the error flag is already set by the waits)
    if (o.x < 0 || o.z < o.x || o.z >= s.geff || o.y < 0 || o.y >= P.rmax) return {0, 0, 0};
    return {o.x, o.z - o.x + 1, o.y};
}

// q[off .. off+3] of column j in a row tile: the sum of the run slots covering it
__device__ __forceinline__ float4 gather_q(const Params& P, const Owners& ow, int j, int off) {
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int o = 0; o < ow.count; ++o) {
        const int sl = (o == 0) ? (ow.first * P.rmax + ow.r) : ((ow.first + o) * P.rmax);
        const float4 v = __ldcg(reinterpret_cast<const float4*>(P.slots + ((size_t)sl * P.nrmax + j) * BM + off));
        q.x += v.x;
        q.y += v.y;
        q.z += v.z;
        q.w += v.w;
    }
    return q;
}

__device__ __forceinline__ void split_store(__nv_bfloat16* hi, __nv_bfloat16* lo, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    *hi = h;
    *lo = l;
}
// entry i of column j of P (hi at row j, lo at row nr + j of the 2 nr-row tiles)
__device__ __forceinline__ void p_store(__nv_bfloat16* P, int nr, int j, int i, float v) {
    uint8_t* Pt = reinterpret_cast<uint8_t*>(P);
    const size_t tb = (size_t)(i >> 6) * (2 * nr) * 128;
    split_store(reinterpret_cast<__nv_bfloat16*>(Pt + tb + sw128(j, i & 63)),
                reinterpret_cast<__nv_bfloat16*>(Pt + tb + sw128(nr + j, i & 63)), v);
}

// Vector work is split into items (active problem, column j, group of VT row tiles =
// VT * 128 rows); each warp of the grid takes a contiguous range of items, each lane
// four consecutive rows of every tile of the group.  Dot products are summed per item
// and written as partials; a column's total is the sum of its partials in group
// order, computed identically by every warp that needs it.
constexpr int VT = 4;

struct VItem {
    int k, p, j, g;
};
__device__ __forceinline__ VItem vdecode(const Ctl& s, const Params& P, long long i) {
    int k = 0;
    while (k + 1 < s.na && i >= s.vbase[k + 1]) ++k;
    const int p = s.act[k];
    const long long l = i - s.vbase[k];
    const int ng = P.prob[p].ngroups;
    return {k, p, (int)(l / ng), (int)(l % ng)};
}

// sum of part[0 .. m) in index order within each lane's stride, then across lanes.
// The inner iteration keeps its inner products in float32: its vectors are float32,
// and the float64 pipe of this part is too slow to spend on them.
__device__ __forceinline__ float column_total(const float* part, int m) {
    const int lane = threadIdx.x & 31;
    float a = 0.f;
    for (int i = lane; i < m; i += 32) a += __ldcg(part + i);
    return warp_sum(a);
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// The inner iteration is conjugate gradients in the Chronopoulos-Gear arrangement:
// the product is taken of the residual (w = Ã r) and s = Ã p is carried by
// recurrence, so that both inner products of a step (gamma = r.r, delta = r.w) come
// from one pass, and a step needs two vector phases:
//   X: w = Ã r (sum of the run slots); partial gamma and delta per item.
//   Y: beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//      (beta = 0, alpha = gamma / delta on the first step); p = r + beta p,
//      s = w + beta s, z += alpha p, r -= alpha s; bf16 split of the new r.
// In exact arithmetic this is the same sequence of iterates as the textbook form.

// Phase X
__device__ void vec_phase_x(const Ctl& s, const Params& P, int gw, int W) {
    const long long I = s.vbase[s.na];
    const long long i0 = range_start(I, W, gw), i1 = range_start(I, W, gw + 1);
    const int lane = threadIdx.x & 31;
    for (long long i = i0; i < i1; ++i) {
        const VItem v = vdecode(s, P, i);
        const ProbDev& pr = P.prob[v.p];
        const int done = __ldcg(&pr.col[v.j].done);
        const size_t base = (size_t)v.j * pr.ldv;
        const int tn = min(VT, pr.mtiles - v.g * VT);
        Owners ow[VT];
        float4 rv[VT];
#pragma unroll
        for (int u = 0; u < VT; ++u) {
            if (u < tn) {
                ow[u] = tile_owners(s, P, v.k, v.g * VT + u);
                rv[u] = __ldcg(reinterpret_cast<const float4*>(pr.r + base + (v.g * VT + u) * BM + lane * 4));
            }
        }
        if (done) continue;
        float d = 0.f, g = 0.f;
#pragma unroll
        for (int u = 0; u < VT; ++u) {
            if (u < tn) {
                const float4 w = gather_q(P, ow[u], v.j, lane * 4);
                __stcg(reinterpret_cast<float4*>(pr.q + base + (v.g * VT + u) * BM + lane * 4), w);
                d += dot4(rv[u], w);
                g += dot4(rv[u], rv[u]);
            }
        }
        d = warp_sum(d);
        g = warp_sum(g);
        if (lane == 0) {
            __stcg(pr.pq + (size_t)v.j * pr.ngroups + v.g, d);
            __stcg(pr.rq + (size_t)v.j * pr.ngroups + v.g, g);
        }
    }
}

// Phase Y
__device__ void vec_phase_y(const Ctl& s, const Params& P, int gw, int W, int it) {
    const long long I = s.vbase[s.na];
    const long long i0 = range_start(I, W, gw), i1 = range_start(I, W, gw + 1);
    const int lane = threadIdx.x & 31;
    int cp = -1, cj = -1;
    float gam = 0.f, del = 0.f;
    for (long long i = i0; i < i1; ++i) {
        const VItem v = vdecode(s, P, i);
        const ProbDev& pr = P.prob[v.p];
        ColState* cs = pr.col + v.j;
        const size_t base = (size_t)v.j * pr.ldv;
        const int tn = min(VT, pr.mtiles - v.g * VT);
        // every load of the item is independent of the step scalars: issue them all first
        float4 w[VT], r[VT], pp[VT], sv[VT], z[VT];
#pragma unroll
        for (int u = 0; u < VT; ++u) {
            if (u < tn) {
                const size_t o = base + (v.g * VT + u) * BM + lane * 4;
                w[u] = __ldcg(reinterpret_cast<const float4*>(pr.q + o));
                r[u] = __ldcg(reinterpret_cast<const float4*>(pr.r + o));
                pp[u] = __ldcg(reinterpret_cast<const float4*>(pr.p + o));
                sv[u] = __ldcg(reinterpret_cast<const float4*>(pr.sv + o));
                z[u] = __ldcg(reinterpret_cast<const float4*>(pr.z + o));
            }
        }
        const float gprev = (float)__ldcg(&cs->gam[it & 1]), aprev = (float)__ldcg(&cs->alp[it & 1]);
        const float rr0 = (float)__ldcg(&cs->rr0);
        if (__ldcg(&cs->done)) continue;
        if (v.p != cp || v.j != cj) {
            gam = column_total(pr.rq + (size_t)v.j * pr.ngroups, pr.ngroups);
            del = column_total(pr.pq + (size_t)v.j * pr.ngroups, pr.ngroups);
            cp = v.p;
            cj = v.j;
        }
        // every warp of the column computes the same totals and takes the same branch
        if (gam <= (float)P.tol2 * rr0) {
            if (v.g == 0 && lane == 0) {
                __stcg(&cs->its, it);
                __stcg(&cs->status, (int)FL_OK);
                __stcg(&cs->done, 1);
                atomicAdd(P.ndone + v.p, 1);
            }
            continue;
        }
        float beta = 0.f, alpha;
        if (it == 0) {
            alpha = gam / del;
        } else {
            beta = gam / gprev;
            alpha = gam / (del - beta * gam / aprev);
        }
        if (!(alpha > 0.f) || !isfinite(alpha)) {  // loss of positive definiteness
            if (v.g == 0 && lane == 0) {
                __stcg(&cs->status, (int)FL_ENOTSPD);
                __stcg(&cs->its, it + 1);
                __stcg(&cs->done, 1);
                atomicAdd(P.ndone + v.p, 1);
            }
            continue;
        }
        const float a = alpha, bt = beta;
        uint8_t* Pt = reinterpret_cast<uint8_t*>(pr.P);
        const int nr2 = 2 * pr.nr;
#pragma unroll
        for (int u = 0; u < VT; ++u) {
            if (u >= tn) break;
            const int row = (v.g * VT + u) * BM + lane * 4;
            const size_t o = base + row;
            pp[u].x = fmaf(bt, pp[u].x, r[u].x);
            pp[u].y = fmaf(bt, pp[u].y, r[u].y);
            pp[u].z = fmaf(bt, pp[u].z, r[u].z);
            pp[u].w = fmaf(bt, pp[u].w, r[u].w);
            sv[u].x = fmaf(bt, sv[u].x, w[u].x);
            sv[u].y = fmaf(bt, sv[u].y, w[u].y);
            sv[u].z = fmaf(bt, sv[u].z, w[u].z);
            sv[u].w = fmaf(bt, sv[u].w, w[u].w);
            z[u].x = fmaf(a, pp[u].x, z[u].x);
            z[u].y = fmaf(a, pp[u].y, z[u].y);
            z[u].z = fmaf(a, pp[u].z, z[u].z);
            z[u].w = fmaf(a, pp[u].w, z[u].w);
            r[u].x = fmaf(-a, sv[u].x, r[u].x);
            r[u].y = fmaf(-a, sv[u].y, r[u].y);
            r[u].z = fmaf(-a, sv[u].z, r[u].z);
            r[u].w = fmaf(-a, sv[u].w, r[u].w);
            __stcg(reinterpret_cast<float4*>(pr.p + o), pp[u]);
            __stcg(reinterpret_cast<float4*>(pr.sv + o), sv[u]);
            __stcg(reinterpret_cast<float4*>(pr.z + o), z[u]);
            __stcg(reinterpret_cast<float4*>(pr.r + o), r[u]);
            __nv_bfloat16 h[4], l[4];
            split_store(&h[0], &l[0], r[u].x);
            split_store(&h[1], &l[1], r[u].y);
            split_store(&h[2], &l[2], r[u].z);
            split_store(&h[3], &l[3], r[u].w);
            uint2 hv, lv;
            memcpy(&hv, h, 8);
            memcpy(&lv, l, 8);
            const size_t tb = (size_t)(row >> 6) * nr2 * 128;
            __stcg(reinterpret_cast<uint2*>(Pt + tb + sw128(v.j, row & 63)), hv);
            __stcg(reinterpret_cast<uint2*>(Pt + tb + sw128(pr.nr + v.j, row & 63)), lv);
        }
        if (v.g == 0 && lane == 0) {
            __stcg(&cs->gam[(it + 1) & 1], gam);
            __stcg(&cs->alp[(it + 1) & 1], alpha);
            __stcg(&cs->its, it + 1);
            if (it + 1 >= P.maxit) {
                __stcg(&cs->status, (int)FL_ENOTCONV);
                __stcg(&cs->done, 1);
                atomicAdd(P.ndone + v.p, 1);
            }
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
    unsigned epoch = 0;
    int it = 0;
    for (; it < P.maxit; ++it) {
        plan_phase(s, P, G, true);
        if (s.na == 0) break;
        gemm_phase(s, P, blockIdx.x, ro);
        if (!tc::grid_barrier(P.gbar, epoch, G, P.err, P.barrier_ns) || __ldcg(P.err) != 0) break;
        const int W = G * (THREADS / 32), gw = blockIdx.x * (THREADS / 32) + (threadIdx.x >> 5);
        vec_phase_x(s, P, gw, W);
        if (!tc::grid_barrier(P.gbar, epoch, G, P.err, P.barrier_ns) || __ldcg(P.err) != 0) break;
        vec_phase_y(s, P, gw, W, it);
        if (!tc::grid_barrier(P.gbar, epoch, G, P.err, P.barrier_ns) || __ldcg(P.err) != 0) break;
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
    const ProbDev& pr = P.prob[s.act[0]];
    for (int i = threadIdx.x * 4; i < pr.mtiles * BM; i += blockDim.x * 4) {
        const Owners ow = tile_owners(s, P, 0, i / BM);
        const float4 q = gather_q(P, ow, j, i % BM);
        const float v[4] = {q.x, q.y, q.z, q.w};
        for (int e = 0; e < 4; ++e)
            if (i + e < pr.n) Y[(size_t)j * ldy + i + e] = v[e];
    }
}

// X (float32, column j at X + j ldx) -> P tiles (x_hi, x_lo), zero beyond n.
__global__ void split_vec_kernel(int n, int nr, int rows, const float* X, int64_t ldx, __nv_bfloat16* Pb) {
    const int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
        p_store(Pb, nr, j, i, (i < n) ? X[(size_t)j * ldx + i] : 0.f);
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

// S_0 = bf16(Ã), S_1 = bf16(Ã - S_0) with Ã_ij = (d_i d_j) a_ij (exactly symmetric),
// written as swizzled 128 x 64 tiles (zero outside n x n).  Block per tile; each
// thread converts 8 consecutive entries of a row into one 16-byte unit.
__global__ void split_matrix_kernel(int64_t n, const double* A, int64_t lda, const double* d, int nslices,
                                    uint8_t* S, int mtiles, int chunks) {
    for (int64_t blk = blockIdx.x; blk < (int64_t)mtiles * chunks; blk += gridDim.x) {
        const int t = (int)(blk / chunks), c = (int)(blk % chunks);
        uint8_t* T0 = S + (size_t)blk * A_TILE;
        uint8_t* T1 = S + ((size_t)mtiles * chunks + blk) * A_TILE;
        for (int e = threadIdx.x; e < BM * 8; e += blockDim.x) {
            const int r = e >> 3, u = e & 7;
            const int64_t i = (int64_t)t * BM + r;
            uint16_t h[8], l[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t j = (int64_t)c * BK + u * 8 + q;
                double a = 0.0;
                if (i < n && j < n) a = A[i * lda + j] * (d[i] * d[j]);
                h[q] = bf16_bits_rn(a);
                l[q] = bf16_bits_rn(a - bf16_value(h[q]));
            }
            uint4 hv, lv;
            memcpy(&hv, h, 16);
            memcpy(&lv, l, 16);
            *reinterpret_cast<uint4*>(T0 + sw128(r, u * 8)) = hv;
            if (nslices > 1) *reinterpret_cast<uint4*>(T1 + sw128(r, u * 8)) = lv;
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
constexpr size_t DF_SMEM = (size_t)DF_K * (DF_ROWS + 1) * sizeof(float2) + (size_t)DF_K * DF_COLS * sizeof(float2) +
                          (size_t)(DF_ROWS * DF_K + DF_K * DF_COLS) * sizeof(double);

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

__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_addr(dst)),
                 "l"((uint64_t)__cvta_generic_to_global(src)), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Raw float64 tiles of work item g into shared memory (asynchronous, zero-filled
// outside the matrix): A rows r0.., columns k0.. and U rows k0.., columns c0..
__device__ __forceinline__ void df_fetch(const DfParams& D, long long g, double* Araw, double* Uraw) {
    const DfUnit u = df_decode(D, g);
    const DfProb& pr = D.prob[u.p];
    const int r0 = u.rb * DF_ROWS, k0 = u.kc * DF_K, c0 = u.ct * DF_COLS;
    for (int e = threadIdx.x; e < DF_ROWS * DF_K; e += DF_THREADS) {
        const int row = e >> 5, kk = e & 31;
        const int i = r0 + row, kcol = k0 + kk;
        const bool ok = i < pr.n && kcol < pr.n;
        cp_async8(Araw + e, ok ? pr.A + (int64_t)i * pr.lda + kcol : pr.A, ok ? 8u : 0u);
    }
    for (int e = threadIdx.x; e < DF_K * DF_COLS; e += DF_THREADS) {
        const int kk = e >> 6, c = e & 63;
        const int krow = k0 + kk, col = c0 + c;
        const bool ok = krow < pr.n && col < pr.nrhs;
        cp_async8(Uraw + e, ok ? pr.U + (int64_t)krow * pr.ldu + col : pr.U, ok ? 8u : 0u);
    }
    cp_async_commit();
}

__global__ void __launch_bounds__(DF_THREADS, 2) residual_df_kernel(const __grid_constant__ DfParams D) {
    extern __shared__ float2 df_smem[];
    float2(*As)[DF_ROWS + 1] = reinterpret_cast<float2(*)[DF_ROWS + 1]>(df_smem);
    float2(*Us)[DF_COLS] = reinterpret_cast<float2(*)[DF_COLS]>(df_smem + DF_K * (DF_ROWS + 1));
    double* Araw = reinterpret_cast<double*>(df_smem + DF_K * (DF_ROWS + 1) + DF_K * DF_COLS);
    double* Uraw = Araw + DF_ROWS * DF_K;
    const int b = blockIdx.x, G = gridDim.x;
    const long long Utot = D.ubase[D.na];
    const long long u0 = range_start(Utot, G, b), u1 = range_start(Utot, G, b + 1);
    const int t = threadIdx.x, rg = t & 15, cg = t >> 4;
    float sh[8][4], sl[8][4];
    int r = 0;
    if (u0 < u1) df_fetch(D, u0, Araw, Uraw);
    for (long long g = u0; g < u1; ++g) {
        const DfUnit u = df_decode(D, g);
        const DfProb& pr = D.prob[u.p];
        if (g == u0 || u.kc == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
        }
        cp_async_wait_all();
        __syncthreads();  // raw tiles of g landed; every thread is done with the previous split tiles
        for (int e = t; e < DF_ROWS * DF_K; e += DF_THREADS) df_split(Araw[e], As[e & 31][e >> 5]);
        for (int e = t; e < DF_K * DF_COLS; e += DF_THREADS) df_split(Uraw[e], Us[e >> 6][e & 63]);
        __syncthreads();  // split tiles ready; raw buffer free
        if (g + 1 < u1) df_fetch(D, g + 1, Araw, Uraw);  // overlaps the products below
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
    cp_async_wait_all();
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
        pr.p[(size_t)j * pr.ldv + i] = 0.f;
        pr.sv[(size_t)j * pr.ldv + i] = 0.f;
        pr.z[(size_t)j * pr.ldv + i] = 0.f;
        p_store(pr.P, pr.nr, j, i, v);
        rr += (double)v * v;
    }
    rr = warp_sum(rr);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        cs->gam[0] = tot;
        cs->alp[0] = 1.0;
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
static int round_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b * b); }

struct Geometry {
    int G = 0, stages = 0, rmax = 0, nrmax = 0, nsmax = 0, tmem_cols = 0, nacc = 1;
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
    // as many accumulators (up to one per K step of a chunk) as tensor memory holds
    g.nacc = 4;
    while (g.nacc > 1 && g.nacc * 2 * g.nrmax > 512) g.nacc >>= 1;
    g.tmem_cols = tmem_cols_for(g.nacc * g.nrmax);
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

int64_t fl_split_bf16_bytes(int64_t n, int nslices) {
    if (n < 1 || n > 65536 || (nslices != 1 && nslices != 2)) return 0;
    return (int64_t)nslices * ((n + BM - 1) / BM) * ((n + BK - 1) / BK) * A_TILE;
}

int fl_split_bf16(const double* A_dev, int64_t lda, int64_t n, int nslices, void* S_dev, double* dscale_dev,
                  void* stream) {
    if (!A_dev || !S_dev || !dscale_dev || n < 1 || n > 65536 || lda < n || (nslices != 1 && nslices != 2) ||
        ((uintptr_t)S_dev & 15) != 0)
        return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    dscale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, A_dev, lda, dscale_dev);
    fl::count_launch();
    const int mt = (int)((n + BM - 1) / BM), ch = (int)((n + BK - 1) / BK);
    split_matrix_kernel<<<(unsigned)std::min<int64_t>((int64_t)mt * ch, 8192), 256, 0, st>>>(
        n, A_dev, lda, dscale_dev, nslices, (uint8_t*)S_dev, mt, ch);
    fl::count_launch();
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

int fl_matmul_bf16(const void* S_dev, int64_t n, int nslices, int nrhs, const float* X_dev, int64_t ldx,
                   float* Y_dev, int64_t ldy, void* stream) {
    if (!S_dev || !X_dev || !Y_dev || n < 1 || n > 65536 || ldx < n || ldy < n ||
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
    pd.S = (const uint8_t*)S_dev;
    Geometry g;
    if (!geometry({pd}, sms, 0, 0, g)) return FL_EINVAL;
    // G: enough CTAs that each takes at least 2 UMIN chunks
    const long long U = (long long)pd.mtiles * pd.chunks;
    g.G = (int)std::max<long long>(1, std::min<long long>(sms, U / (2 * UMIN)));
    {
        const long long per = std::max<long long>((U + g.G - 1) / g.G, 2 * UMIN) + 1;
        g.rmax = (int)((per + pd.chunks - 1) / pd.chunks) + 1;
    }
    const size_t pbytes = (size_t)2 * pd.mtiles * 2 * nrhs * BK * sizeof(__nv_bfloat16);
    const size_t sbytes = (size_t)g.G * g.rmax * g.nrmax * BM * sizeof(float);
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, pbytes + sbytes + 256, st) != cudaSuccess) return FL_ENOMEM;
    char* c = (char*)ws;
    pd.P = (__nv_bfloat16*)c;
    float* slots = (float*)(c + ((pbytes + 255) & ~size_t(255)));
    int* flags = nullptr;
    if (cudaMallocAsync((void**)&flags, 256 + (size_t)pd.mtiles * sizeof(int4), st) != cudaSuccess) {
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
    P.nacc = g.nacc;
    P.maxit = 1;
    P.slots = slots;
    P.err = flags;
    P.active = flags + 16;
    P.ndone = flags + 32;
    P.iters = flags + 48;
    P.owners = reinterpret_cast<int4*>(flags + 64);
    int rc = FL_OK;
    {
        const int one = 1;
        cudaMemsetAsync(flags, 0, 256 + (size_t)pd.mtiles * sizeof(int4), st);
        cudaMemcpyAsync(P.active, &one, sizeof(int), cudaMemcpyHostToDevice, st);
        split_vec_kernel<<<dim3(16, nrhs), 256, 0, st>>>((int)n, nrhs, pd.chunks * BK, X_dev, ldx, pd.P);
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

int fl_tune_batch(fl_handle h, int nprob, const fl_batch_problem* probs, int reps, fl_batch_opts* best,
                  double* best_ms) {
    if (!h) return FL_EINVAL;
    h->err.clear();
    if (nprob < 1 || nprob > MAXP || !probs || reps < 1) return set_err(h, FL_EINVAL, "bad tuning arguments");
    int sms = 0;
    if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, FL_ECUDA, "cudaSetDevice");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    std::vector<ProbDev> pd(nprob);
    size_t pbytes_total = 0;
    int nmx = 0, nrx = 0, nsx = 0;
    for (int p = 0; p < nprob; ++p) {
        const fl_batch_problem& q = probs[p];
        if (q.n < 1 || q.n > 65536 || !q.S_dev || (q.nslices != 1 && q.nslices != 2) || q.nrhs < 1 || q.nrhs > 128)
            return set_err(h, FL_EINVAL, "bad batch problem " + std::to_string(p));
        ProbDev& d = pd[p];
        d.n = (int)q.n;
        d.nr = round_up(q.nrhs, 16);
        d.nslices = q.nslices;
        d.mtiles = (d.n + BM - 1) / BM;
        d.chunks = (d.n + BK - 1) / BK;
        d.S = (const uint8_t*)q.S_dev;
        pbytes_total += (size_t)2 * d.mtiles * 2 * d.nr * BK * 2;
        nmx = std::max(nmx, d.n);
        nrx = std::max(nrx, d.nr);
        nsx = std::max(nsx, d.nslices);
    }
    Geometry g0;
    if (!geometry(pd, sms, 0, 0, g0)) return set_err(h, FL_EINVAL, "no pipeline fits shared memory");
    int ntiles = 0;
    for (const ProbDev& d : pd) ntiles += d.mtiles;
    // scratch: P tiles (zero), run slots for the largest grid, flags and owner table
    const size_t slot_bytes = (size_t)sms * (g0.rmax + 2) * g0.nrmax * BM * sizeof(float);
    const size_t flag_bytes = 256 + (size_t)ntiles * sizeof(int4);
    char* ws = nullptr;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return set_err(h, FL_ECUDA, "stream");
    if (cudaMalloc((void**)&ws, pbytes_total + slot_bytes + flag_bytes + 1024) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(st);
        return set_err(h, FL_ENOMEM, "tuning scratch");
    }
    cudaMemsetAsync(ws, 0, pbytes_total + slot_bytes + flag_bytes + 1024, st);
    char* c = ws;
    for (ProbDev& d : pd) {
        d.P = (__nv_bfloat16*)c;
        c += ((size_t)2 * d.mtiles * 2 * d.nr * BK * 2 + 255) & ~size_t(255);
    }
    float* slots = (float*)c;
    int* flags = (int*)(c + ((slot_bytes + 255) & ~size_t(255)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int> ctas = {sms, sms - 4, sms - 8, sms - 16, (3 * sms) / 4, sms / 2};
    int best_st = g0.stages, best_ct = sms, rc = FL_OK;
    float best_t = 1e30f;
    static Params P;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    for (int stg = 2; stg <= g0.stages && rc == FL_OK; ++stg) {
        for (int ct : ctas) {
            if (ct < 1) continue;
            Geometry g;
            if (!geometry(pd, sms, ct, stg, g)) continue;
            if (g.rmax > g0.rmax + 2) continue;  // slot scratch sized for the default grid
            memset(&P, 0, sizeof(P));
            P.nprob = nprob;
            for (int p = 0; p < nprob; ++p) P.prob[p] = pd[p];
            P.stages = g.stages;
            P.rmax = g.rmax;
            P.nrmax = g.nrmax;
            P.nsmax = g.nsmax;
            P.tmem_cols = g.tmem_cols;
            P.nacc = g.nacc;
            P.maxit = 1;
            P.slots = slots;
            P.err = flags;
            P.active = flags + 16;
            P.ndone = flags + 32;
            P.iters = flags + 48;
            P.owners = reinterpret_cast<int4*>(flags + 64);
            std::vector<int> one(MAXP, 0);
            for (int p = 0; p < nprob; ++p) one[p] = 1;
            cudaMemcpyAsync(P.active, one.data(), MAXP * sizeof(int), cudaMemcpyHostToDevice, st);
            if (!launch_cfg((const void*)gemm_kernel, g.smem)) {
                rc = FL_ECUDA;
                break;
            }
            std::vector<float> ts;
            for (int r = 0; r <= reps; ++r) {
                cudaEventRecord(e0, st);
                gemm_kernel<<<g.G, THREADS, g.smem, st>>>(P);
                cudaEventRecord(e1, st);
                fl::count_launch();
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = FL_ECUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) ts.push_back(ms);  // the first launch warms up
            }
            if (rc != FL_OK) break;
            int err = 0;
            cudaMemcpyAsync(&err, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            if (err != 0) {
                rc = FL_ETIMEOUT;
                break;
            }
            std::sort(ts.begin(), ts.end());
            const float med = ts[ts.size() / 2];
            if (med < best_t) {
                best_t = med;
                best_st = g.stages;
                best_ct = g.G;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ws);
    cudaStreamDestroy(st);
    if (rc != FL_OK) return set_err(h, rc, "tuning launch failed");
    tune_record(device_name(), "batch_gemm", nmx, nrx, nsx, best_st, best_ct, best_t);
    if (best) {
        fl_default_batch_opts(best);
        best->stages = best_st;
        best->ctas = best_ct;
    }
    if (best_ms) *best_ms = best_t;
    return FL_OK;
}

void fl_default_batch_opts(fl_batch_opts* o) {
    if (!o) return;
    o->tol = 1e-8;
    o->max_outer = 8;
    o->inner_tol = 1e-5;
    o->inner_maxit = 5000;
    o->ctas = 0;
    o->stages = 0;
    o->barrier_timeout_us = 0;
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
    if (!(o.tol > 0) || !(o.inner_tol > 0) || o.max_outer < 1 || o.inner_maxit < 1 || o.barrier_timeout_us < 0 ||
        (o.residual != FL_RESID_F64 && o.residual != FL_RESID_DF))
        return set_err(h, FL_EINVAL, "bad batch options");
    for (int p = 0; p < nprob; ++p) {
        const fl_batch_problem& q = probs[p];
        if (q.n < 1 || q.n > 65536 || !q.A_dev || q.lda < q.n || !q.S_dev ||
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
        d.ngroups = (d.mtiles + VT - 1) / VT;
    }
    int want_ctas = o.ctas, want_stages = o.stages;
    if (want_ctas == 0 && want_stages == 0) {  // launch shape from the tuning table, if measured
        int nmx = 0, nrx = 0, nsx = 0, st0 = 0, ct0 = 0;
        for (const ProbDev& d : pd) {
            nmx = std::max(nmx, d.n);
            nrx = std::max(nrx, d.nr);
            nsx = std::max(nsx, d.nslices);
        }
        if (tune_lookup(device_name(), "batch_gemm", nmx, nrx, nsx, &st0, &ct0)) {
            want_stages = st0;
            want_ctas = ct0;
        }
    }
    Geometry g;
    if (!geometry(pd, sms, want_ctas, want_stages, g)) return set_err(h, FL_EINVAL, "no pipeline fits shared memory");
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
    std::vector<size_t> off_vec(nprob), off_P(nprob), off_col(nprob), off_R(nprob), off_rp(nprob), off_co(nprob),
        off_part(nprob);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t at = total;
        total += (bytes + 255) & ~size_t(255);
        return at;
    };
    for (int p = 0; p < nprob; ++p) {
        const ProbDev& d = pd[p];
        off_vec[p] = take((size_t)5 * d.nr * d.ldv * sizeof(float));
        // P tiles for every row the vector phases write (mtiles * 128 rows = 2 mtiles chunks)
        off_P[p] = take((size_t)2 * d.mtiles * 2 * d.nr * BK * sizeof(__nv_bfloat16));
        off_col[p] = take((size_t)d.nr * sizeof(ColState));
        off_R[p] = take((size_t)d.n * d.nr * sizeof(double));
        off_rp[p] = take((size_t)((d.n + RES_ROWS - 1) / RES_ROWS) * d.nr * sizeof(double));
        off_co[p] = take((size_t)d.nr * sizeof(ColOuter));
        off_part[p] = take((size_t)2 * d.nr * d.ngroups * sizeof(float));
    }
    const size_t off_slots = take((size_t)g.G * g.rmax * g.nrmax * BM * sizeof(float));
    const size_t off_flags = take(256);
    const size_t off_bar = take(256);
    int ntiles = 0;
    for (const ProbDev& d : pd) ntiles += d.mtiles;
    const size_t off_owners = take((size_t)ntiles * sizeof(int4));
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
        if (h->batch_ws) {
            cudaDeviceSynchronize();  // the cached block must be idle before another user takes it
            pool_dev_free(h->batch_ws);
        }
        h->batch_ws = nullptr;
        h->batch_ws_bytes = 0;
        if (pool_dev_alloc(&h->batch_ws, total) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, FL_ENOMEM, "batch workspace");
        }
        h->batch_ws_bytes = total;
    }
    if (!h->batch_host) {
        if (pool_host_alloc(&h->batch_host, 4096) != cudaSuccess) return set_err(h, FL_ENOMEM, "pinned scalars");
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
    P.nacc = g.nacc;
    P.maxit = o.inner_maxit;
    P.tol2 = o.inner_tol * o.inner_tol;
    P.slots = (float*)(W + off_slots);
    P.err = flags;
    P.gbar = (unsigned*)(W + off_bar);
    P.barrier_ns = o.barrier_timeout_us > 0 ? 1000ull * (unsigned long long)o.barrier_timeout_us : 2000000000ull;
    P.ndone = flags + 8;
    P.active = flags + 24;
    P.iters = flags + 4;
    P.owners = reinterpret_cast<int4*>(W + off_owners);
    RP.nprob = nprob;
    for (int p = 0; p < nprob; ++p) {
        ProbDev& d = pd[p];
        float* v = (float*)(W + off_vec[p]);
        d.r = v;
        d.z = v + (size_t)d.nr * d.ldv;
        d.p = v + (size_t)2 * d.nr * d.ldv;
        d.q = v + (size_t)3 * d.nr * d.ldv;
        d.sv = v + (size_t)4 * d.nr * d.ldv;
        d.P = (__nv_bfloat16*)(W + off_P[p]);
        d.S = (const uint8_t*)probs[p].S_dev;
        d.col = (ColState*)(W + off_col[p]);
        d.pq = (float*)(W + off_part[p]);
        d.rq = d.pq + (size_t)d.nr * d.ngroups;
        P.prob[p] = d;
        const fl_batch_problem& q = probs[p];
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
        if (cudaMemsetAsync(P.gbar, 0, sizeof(unsigned), st) != cudaSuccess) return set_err(h, FL_ECUDA, "memset");
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
