// Dense linear algebra of the solvers (arXiv:1708.03912, Section 5): the dense
// matrix-vector product, whose cost is n^2 per product, and diagonally
// preconditioned conjugate gradients, whose iteration count grows like n^{s/d}.
// Also the float32 / bfloat16 copies used by the mixed-precision refinement.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <string>
#include <vector>

#include "context.h"
#include "device.h"
#include "tc.h"

namespace fl {

// ------------------------------------------------------------------ GEMV --
// One warp per row; 16-byte vector loads of A when the row start is aligned.
template <typename TA>
struct Vec16;
template <>
struct Vec16<double> {
    static constexpr int N = 2;
};
template <>
struct Vec16<float> {
    static constexpr int N = 4;
};
template <>
struct Vec16<__nv_bfloat16> {
    static constexpr int N = 8;
};

template <typename TA>
__device__ __forceinline__ void unpack16(const uint4& u, float* out);
template <>
__device__ __forceinline__ void unpack16<float>(const uint4& u, float* out) {
    out[0] = __uint_as_float(u.x);
    out[1] = __uint_as_float(u.y);
    out[2] = __uint_as_float(u.z);
    out[3] = __uint_as_float(u.w);
}
template <>
__device__ __forceinline__ void unpack16<__nv_bfloat16>(const uint4& u, float* out) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        out[2 * i] = __uint_as_float(w[i] << 16);
        out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// float64 matrix, float64 vector, float64 accumulation.  Rows whose start is not
// 16-byte aligned (odd lda) peel one element, then stream 16-byte vectors.
__global__ void gemv_f64_kernel(int64_t n, const double* __restrict__ A, int64_t lda, const double* __restrict__ x,
                                int64_t incx, double* __restrict__ y, int64_t incy, int vec) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const double* a = A + row * lda;
    double acc0 = 0.0, acc1 = 0.0;
    int64_t j0 = 0;
    if (vec && incx == 1) {
        const int64_t p0 = (((uintptr_t)a & 15u) != 0) ? 1 : 0;
        if (lane < p0 && p0 <= n) acc0 = fma(a[0], x[0], acc0);
        const int64_t m = n - p0;
        const int64_t nv = (m / 64) * 64;
        const double2* a2 = reinterpret_cast<const double2*>(a + p0);
        if (p0 == 0) {
            const double2* x2 = reinterpret_cast<const double2*>(x);
#pragma unroll 4
            for (int64_t j = lane; j < nv / 2; j += 32) {
                const double2 av = __ldcs(a2 + j);
                const double2 xv = x2[j];
                acc0 = fma(av.x, xv.x, acc0);
                acc1 = fma(av.y, xv.y, acc1);
            }
        } else {
            const double* xs = x + p0;
#pragma unroll 4
            for (int64_t j = lane; j < nv / 2; j += 32) {
                const double2 av = __ldcs(a2 + j);
                acc0 = fma(av.x, xs[2 * j], acc0);
                acc1 = fma(av.y, xs[2 * j + 1], acc1);
            }
        }
        j0 = p0 + nv;
    }
    for (int64_t j = j0 + lane; j < n; j += 32) acc0 = fma(a[j], x[j * incx], acc0);
    double t = warp_sum(acc0 + acc1);
    if (lane == 0) y[row * incy] = t;
}

// float32 / bfloat16 matrix, float32 vector, float32 lane sums, float64 row total.
// Misaligned row starts peel up to V-1 elements; x is read as float4 when it stays
// aligned with the row, else element by element.
template <typename TA>
__global__ void gemv_lo_kernel(int64_t n, const TA* __restrict__ A, int64_t lda, const float* __restrict__ x,
                               double* __restrict__ y, int64_t incy, int vec) {
    constexpr int V = Vec16<TA>::N;
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const TA* a = A + row * lda;
    float acc0 = 0.f, acc1 = 0.f;
    int64_t j0 = 0;
    if (vec) {
        const int mis = (int)(((uintptr_t)a & 15u) / sizeof(TA));
        const int64_t p0 = min((int64_t)(mis ? V - mis : 0), n);
        if (lane < p0) acc0 = fmaf((float)a[lane], x[lane], acc0);
        const int64_t m = n - p0;
        const int64_t nv = (m / (32 * V)) * (32 * V);
        const uint4* a4 = reinterpret_cast<const uint4*>(a + p0);
        if ((p0 & 3) == 0) {
            const float4* x4 = reinterpret_cast<const float4*>(x + p0);
#pragma unroll 4
            for (int64_t j = lane; j < nv / V; j += 32) {
                const uint4 u = __ldcs(a4 + j);
                float av[V];
                unpack16<TA>(u, av);
#pragma unroll
                for (int q = 0; q < V / 4; ++q) {
                    const float4 xv = x4[j * (V / 4) + q];
                    acc0 = fmaf(av[4 * q + 0], xv.x, acc0);
                    acc1 = fmaf(av[4 * q + 1], xv.y, acc1);
                    acc0 = fmaf(av[4 * q + 2], xv.z, acc0);
                    acc1 = fmaf(av[4 * q + 3], xv.w, acc1);
                }
            }
        } else {
            const float* xs = x + p0;
#pragma unroll 4
            for (int64_t j = lane; j < nv / V; j += 32) {
                const uint4 u = __ldcs(a4 + j);
                float av[V];
                unpack16<TA>(u, av);
#pragma unroll
                for (int q = 0; q < V; q += 2) {
                    acc0 = fmaf(av[q], xs[j * V + q], acc0);
                    acc1 = fmaf(av[q + 1], xs[j * V + q + 1], acc1);
                }
            }
        }
        j0 = p0 + nv;
    }
    for (int64_t j = j0 + lane; j < n; j += 32) acc0 = fmaf((float)a[j], x[j], acc0);
    double t = warp_sum((double)acc0 + (double)acc1);
    if (lane == 0) y[row * incy] = t;
}

// a matrix entry in the accumulator's type
template <typename Acc, typename TA>
__device__ __forceinline__ Acc to_acc(TA v) {
    if constexpr (std::is_same<TA, __nv_bfloat16>::value) return (Acc)__bfloat162float(v);
    else return (Acc)v;
}

constexpr int GEMV_SMEM_WARPS = 8;
// grids of the staged products for the last few sizes (per host thread and kernel)
struct GemvGridCache {
    static constexpr int K = 8;
    int64_t n[K] = {-1, -1, -1, -1, -1, -1, -1, -1};
    unsigned gen[K] = {}, grid[K] = {};
    int next = 0;
    bool find(int64_t nn, unsigned g, unsigned* out) const {
        for (int k = 0; k < K; ++k)
            if (n[k] == nn && gen[k] == g) {
                *out = grid[k];
                return true;
            }
        return false;
    }
    void put(int64_t nn, unsigned g, unsigned gr) {
        n[next] = nn;
        gen[next] = g;
        grid[next] = gr;
        next = (next + 1) % K;
    }
    void clear() {
        for (int k = 0; k < K; ++k) n[k] = -1;
    }
};
// tuning-table names of the staged products
template <typename TA>
struct GemvName;
template <>
struct GemvName<double> {
    static constexpr const char* name = "gemv_smem_f64";
};
template <>
struct GemvName<float> {
    static constexpr const char* name = "gemv_smem_f32";
};
template <>
struct GemvName<__nv_bfloat16> {
    static constexpr const char* name = "gemv_smem_bf16";
};
constexpr size_t GEMV_SMEM_MAX = 200 * 1024;  // bytes of staged x (padding included)
constexpr int GEMV_SMEM_PAD = 8;               // zero elements after x: shifted reads stay in bounds

// The same products with x staged in shared memory once per block (8 warps, warp per row,
// row = block * 8 + warp with stride grid * 8), so x is read from L2 once per block instead
// of once per row.  A row starting off a 16-byte boundary peels its first elements; the x
// entries that go with a 16-byte chunk of A are then read as 16-byte words of the staged
// copy and shifted in registers (a compile-time shift per row alignment), which keeps the
// shared-memory reads free of bank conflicts.  Each row starts its chunk loop at a
// row-dependent rotation, so the warps streaming neighbouring rows (a fixed stride apart)
// do not all address the same memory channels at once.
// four floats of x starting at element 4 c + SH (c counted in float4 words)
template <int SH>
__device__ __forceinline__ float4 x4_at(const float4* xs4, int64_t c) {
    const float4 lo = xs4[c];
    if constexpr (SH == 0) return lo;
    const float4 hi = xs4[c + 1];
    if constexpr (SH == 1) return make_float4(lo.y, lo.z, lo.w, hi.x);
    if constexpr (SH == 2) return make_float4(lo.z, lo.w, hi.x, hi.y);
    return make_float4(lo.w, hi.x, hi.y, hi.z);
}
// two doubles of x starting at element 2 c + SH
template <int SH>
__device__ __forceinline__ double2 x2_at(const double2* xs2, int64_t c) {
    const double2 lo = xs2[c];
    if constexpr (SH == 0) return lo;
    const double2 hi = xs2[c + 1];
    return make_double2(lo.y, hi.x);
}

// the 16-byte chunks of one row: a4 = first aligned chunk, element p0 of the row; SH = the
// shift of x within its 16-byte words
template <typename TA, typename TX, int SH>
__device__ __forceinline__ void gemv_row_chunks(const uint4* __restrict__ a4, const TX* xs, int64_t p0, int64_t nv,
                                                int64_t rot, int lane, double& out) {
    constexpr int V = Vec16<TA>::N;
    if constexpr (sizeof(TX) == 8) {
        const double2* xs2 = reinterpret_cast<const double2*>(xs) + (p0 >> 1);
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 8
        for (int64_t k = lane; k < nv; k += 32) {
            int64_t j = k + rot;
            if (j >= nv) j -= nv;
            const uint4 u = __ldcs(a4 + j);
            const double2 xv = x2_at<SH>(xs2, j);
            acc0 = fma(__longlong_as_double(((long long)u.y << 32) | u.x), xv.x, acc0);
            acc1 = fma(__longlong_as_double(((long long)u.w << 32) | u.z), xv.y, acc1);
        }
        out += acc0 + acc1;
    } else {
        const float4* xs4 = reinterpret_cast<const float4*>(xs) + (p0 >> 2);
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 8
        for (int64_t k = lane; k < nv; k += 32) {
            int64_t j = k + rot;
            if (j >= nv) j -= nv;
            const uint4 u = __ldcs(a4 + j);
            float av[V];
            unpack16<TA>(u, av);
#pragma unroll
            for (int h = 0; h < V / 4; ++h) {
                const float4 xv = x4_at<SH>(xs4, j * (V / 4) + h);
                acc0 = fmaf(av[4 * h + 0], xv.x, acc0);
                acc1 = fmaf(av[4 * h + 1], xv.y, acc1);
                acc0 = fmaf(av[4 * h + 2], xv.z, acc0);
                acc1 = fmaf(av[4 * h + 3], xv.w, acc1);
            }
        }
        out += (double)acc0 + (double)acc1;
    }
}

template <typename TA, typename TX>
__global__ void __launch_bounds__(32 * GEMV_SMEM_WARPS, 4)
    gemv_smem_kernel(int64_t n, const TA* __restrict__ A, int64_t lda, const double* __restrict__ x, int64_t incx,
                     const float* __restrict__ xf, double* __restrict__ y, int64_t incy) {
    constexpr int V = Vec16<TA>::N;
    constexpr bool F64 = sizeof(TX) == 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TX* xs = reinterpret_cast<TX*>(smem_raw);
    // x staged as TX: float64 as is; for float32 / bfloat16 A either the caller's float32 copy
    // xf or x rounded here (the same rounding as that copy)
    for (int64_t i = threadIdx.x; i < n + GEMV_SMEM_PAD; i += blockDim.x) {
        if constexpr (F64) xs[i] = i < n ? x[i * incx] : 0.0;
        else xs[i] = i < n ? (xf ? xf[i] : (float)x[i * incx]) : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t row = (int64_t)blockIdx.x * GEMV_SMEM_WARPS + warp; row < n; row += (int64_t)gridDim.x * GEMV_SMEM_WARPS) {
        const TA* a = A + row * lda;
        double t = 0.0;
        // peel to the first 16-byte boundary of the row
        const int mis = (int)(((uintptr_t)a & 15u) / sizeof(TA));
        const int64_t p0 = min((int64_t)(mis ? V - mis : 0), n);
        if constexpr (F64) {
            if (lane < p0) t = a[lane] * xs[lane];
        } else {
            if (lane < p0) t = (double)(to_acc<float>(a[lane]) * xs[lane]);
        }
        const int64_t nv = (n - p0) / V;  // whole 16-byte chunks
        const int64_t rot = nv > 0 ? (int64_t)(((uint64_t)row * 2654435761ull) % (uint64_t)nv) : 0;
        const uint4* a4 = reinterpret_cast<const uint4*>(a + p0);
        if constexpr (F64) {
            if (p0 & 1) gemv_row_chunks<TA, TX, 1>(a4, xs, p0, nv, rot, lane, t);
            else gemv_row_chunks<TA, TX, 0>(a4, xs, p0, nv, rot, lane, t);
        } else {
            switch (p0 & 3) {
                case 0: gemv_row_chunks<TA, TX, 0>(a4, xs, p0, nv, rot, lane, t); break;
                case 1: gemv_row_chunks<TA, TX, 1>(a4, xs, p0, nv, rot, lane, t); break;
                case 2: gemv_row_chunks<TA, TX, 2>(a4, xs, p0, nv, rot, lane, t); break;
                default: gemv_row_chunks<TA, TX, 3>(a4, xs, p0, nv, rot, lane, t); break;
            }
        }
        for (int64_t j = p0 + nv * V + lane; j < n; j += 32) {
            if constexpr (F64) t = fma(a[j], xs[j], t);
            else t += (double)(to_acc<float>(a[j]) * xs[j]);
        }
        t = warp_sum(t);
        if (lane == 0) y[row * incy] = t;
    }
}

// grid of the shared-memory product: as many blocks as fit on the device at once (at most
// one per 8 rows); 0 when x does not fit
template <typename TA, typename TX>
static unsigned gemv_smem_grid(int64_t n, int force_per_sm = 0, int* max_per_sm = nullptr) {
    const size_t smem = (size_t)(n + GEMV_SMEM_PAD) * sizeof(TX);
    if (smem > GEMV_SMEM_MAX) return 0;
    // per host thread (no locking): the attribute is set once per thread and device; the grids
    // of the last few sizes are kept, so that solvers alternating between levels of different
    // size (multigrid) make no driver query per product
    static thread_local int ready = 0, sms = 0, dev_cached = -1;
    static thread_local GemvGridCache cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const unsigned gen = tune_generation();
    unsigned hit = 0;
    if (!force_per_sm && !max_per_sm && ready && dev == dev_cached && cache.find(n, gen, &hit)) return hit;
    if (!ready || dev != dev_cached) {
        cache.clear();
        if (cudaFuncSetAttribute(gemv_smem_kernel<TA, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)GEMV_SMEM_MAX) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        ready = 1;
        dev_cached = dev;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemv_smem_kernel<TA, TX>, 32 * GEMV_SMEM_WARPS,
                                                      smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    if (max_per_sm) *max_per_sm = per_sm;
    const int64_t want = (n + GEMV_SMEM_WARPS - 1) / GEMV_SMEM_WARPS;
    if (force_per_sm) return (unsigned)std::min<int64_t>(want, (int64_t)sms * std::min(force_per_sm, per_sm));
    unsigned grid = 0;
    // with one block (8 warps) per SM too few loads are in flight: the warp-per-row kernels,
    // which keep x in L1/L2, are used instead
    if (per_sm >= 2) {
        // blocks per SM from the matvec autotuner (fl_tune_matvec) when it has measured this size
        int p0 = 0, p1 = 0;
        if (tune_lookup(device_name(), GemvName<TA>::name, n, 1, 1, &p0, &p1) && p0 >= 1)
            per_sm = std::min(per_sm, p0);
        grid = (unsigned)std::min<int64_t>(want, (int64_t)sms * per_sm);
    }
    cache.put(n, gen, grid);
    return grid;
}

// Hi + lo float32 storage (FL_F32X2): entry (i, j) is the float2 (hi, lo), hi = fl32(a),
// lo = fl32(a - hi), 8 bytes like float64 but multiplied on the float32 pipe.  x is split
// into (hi, lo) by integer operations, and each product is accumulated in double-float
// arithmetic: y_i = sum_j (hi + lo)_ij (xh + xl)_j to about 2^-44 of sum_j |a_ij x_j|,
// without the float64 pipe that bounds the FL_F64 product.  x is staged in shared memory
// (STAGED) or read as float2 from a split copy in global memory.
template <int SH>
__device__ __forceinline__ float4 x2pair_at(const float4* xs4, int64_t j) {
    // the float2 entries 2 j + SH and 2 j + SH + 1 of x as one float4
    const float4 lo = xs4[j];
    if constexpr (SH == 0) return lo;
    const float4 hi = xs4[j + 1];
    return make_float4(lo.z, lo.w, hi.x, hi.y);
}

template <int SH>
__device__ __forceinline__ void gemv_x2_chunks(const uint4* __restrict__ a4, const float4* xs4, int64_t nv, int64_t rot,
                                               int lane, float (&acc)[4]) {
#pragma unroll 8
    for (int64_t k = lane; k < nv; k += 32) {
        int64_t j = k + rot;
        if (j >= nv) j -= nv;
        const uint4 u = __ldcs(a4 + j);
        const float4 xv = x2pair_at<SH>(xs4, j);
        df_fma(acc[0], acc[1], __uint_as_float(u.x), __uint_as_float(u.y), xv.x, xv.y);
        df_fma(acc[2], acc[3], __uint_as_float(u.z), __uint_as_float(u.w), xv.z, xv.w);
    }
}

template <bool STAGED>
__global__ void __launch_bounds__(32 * GEMV_SMEM_WARPS, 4)
    gemv_x2_kernel(int64_t n, const float2* __restrict__ A, int64_t lda, const double* __restrict__ x, int64_t incx,
                   const float2* __restrict__ xg, double* __restrict__ y, int64_t incy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const float2* xs;
    if constexpr (STAGED) {
        float2* xw = reinterpret_cast<float2*>(smem_raw);
        for (int64_t i = threadIdx.x; i < n + GEMV_SMEM_PAD; i += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (i < n) df_split(x[i * incx], v);
            xw[i] = v;
        }
        __syncthreads();
        xs = xw;
    } else {
        xs = xg;  // n + GEMV_SMEM_PAD entries, 16-byte aligned
    }
    const float4* xs4 = reinterpret_cast<const float4*>(xs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t row = (int64_t)blockIdx.x * GEMV_SMEM_WARPS + warp; row < n; row += (int64_t)gridDim.x * GEMV_SMEM_WARPS) {
        const float2* a = A + row * lda;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int64_t p0 = (((uintptr_t)a & 15u) != 0) ? 1 : 0;  // rows start 8-byte aligned
        if (lane < p0) {
            const float2 av = a[0], xv = xs[0];
            df_fma(acc[0], acc[1], av.x, av.y, xv.x, xv.y);
        }
        const int64_t nv = (n - p0) / 2;  // 16-byte chunks: two entries
        const int64_t rot = nv > 0 ? (int64_t)(((uint64_t)row * 2654435761ull) % (uint64_t)nv) : 0;
        const uint4* a4 = reinterpret_cast<const uint4*>(a + p0);
        if (p0) gemv_x2_chunks<1>(a4, xs4, nv, rot, lane, acc);
        else gemv_x2_chunks<0>(a4, xs4, nv, rot, lane, acc);
        for (int64_t j = p0 + 2 * nv + lane; j < n; j += 32) {
            const float2 av = a[j], xv = xs[j];
            df_fma(acc[0], acc[1], av.x, av.y, xv.x, xv.y);
        }
        const double t = warp_sum(((double)acc[0] + (double)acc[1]) + ((double)acc[2] + (double)acc[3]));
        if (lane == 0) y[row * incy] = t;
    }
}

// x split into (hi, lo) float32 pairs, zero padded (the unstaged product's copy of x)
__global__ void x2_split_kernel(int64_t n, const double* x, int64_t incx, float2* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n + GEMV_SMEM_PAD) return;
    float2 v = make_float2(0.f, 0.f);
    if (i < n) df_split(x[i * incx], v);
    out[i] = v;
}

// grid of the staged hi + lo product (0 when x does not fit), as gemv_smem_grid
static unsigned gemv_x2_grid(int64_t n) {
    const size_t smem = (size_t)(n + GEMV_SMEM_PAD) * sizeof(float2);
    if (smem > GEMV_SMEM_MAX) return 0;
    static thread_local int ready = 0, sms = 0, dev_cached = -1;
    static thread_local GemvGridCache cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    unsigned hit = 0;
    if (ready && dev == dev_cached && cache.find(n, 0u, &hit)) return hit;
    if (!ready || dev != dev_cached) {
        cache.clear();
        if (cudaFuncSetAttribute(gemv_x2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMV_SMEM_MAX) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        ready = 1;
        dev_cached = dev;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemv_x2_kernel<true>, 32 * GEMV_SMEM_WARPS, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    // one block per SM keeps too few loads in flight: the unstaged kernel is used then
    const unsigned grid =
        per_sm >= 2 ? (unsigned)std::min<int64_t>((n + GEMV_SMEM_WARPS - 1) / GEMV_SMEM_WARPS, (int64_t)sms * per_sm) : 0u;
    cache.put(n, 0u, grid);
    return grid;
}

__global__ void convert_x2_kernel(int64_t n, const double* A, int64_t lda, float2* B, int64_t ldb) {
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
            const double a = A[i * lda + j];
            const float hi = (float)a;
            B[i * ldb + j] = make_float2(hi, (float)(a - (double)hi));
        }
}

__global__ void to_f32_kernel(int64_t n, const double* x, int64_t incx, float* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i * incx];
}

template <typename TO>
__global__ void convert_kernel(int64_t n, const double* A, int64_t lda, TO* B, int64_t ldb) {
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
            if constexpr (sizeof(TO) == 4) B[i * ldb + j] = (float)A[i * lda + j];
            else B[i * ldb + j] = __double2bfloat16(A[i * lda + j]);
        }
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// grid of the shared-memory product for a float32 / bfloat16 matrix, 0 if it does not apply
static unsigned gemv_lo_smem_grid(int dtype, const void* A, int64_t n) {
    if (dtype == FL_F32) return (((uintptr_t)A & 3u) == 0) ? gemv_smem_grid<float, float>(n) : 0u;
    return (((uintptr_t)A & 1u) == 0) ? gemv_smem_grid<__nv_bfloat16, float>(n) : 0u;
}

// the row-dot product (defined after row_dot below): true when it ran
static bool gemv_rows(int dtype, const void* A, int64_t lda, int64_t n, const double* x, int64_t incx, double* y,
                      int64_t incy, const float* xf, bool xf_ready, cudaStream_t st);

// y = A x for one right-hand side; xf is a float32 scratch copy of x (n) for low-precision A
// (unused, and may be NULL, when the shared-memory product applies and xf_ready is false)
// xf_ready: xf already holds x rounded to float32 (the CG keeps such a copy of p)
cudaError_t gemv(int dtype, const void* A, int64_t lda, int64_t n, const double* x, int64_t incx, double* y,
                 int64_t incy, float* xf, cudaStream_t st, bool xf_ready) {
    const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
    if (dtype == FL_F32 && gemv_rows(dtype, A, lda, n, x, incx, y, incy, xf, xf_ready, st)) {
        fl::count_launch();
        return cudaGetLastError();
    }
    if (dtype == FL_F32X2) {
        const unsigned gs = gemv_x2_grid(n);
        if (gs) {
            gemv_x2_kernel<true><<<gs, 32 * GEMV_SMEM_WARPS, (n + GEMV_SMEM_PAD) * sizeof(float2), st>>>(
                n, (const float2*)A, lda, x, incx, nullptr, y, incy);
        } else {
            // xf holds 2 (n + GEMV_SMEM_PAD) floats here (fl_matvec sizes it)
            x2_split_kernel<<<(unsigned)((n + GEMV_SMEM_PAD + 255) / 256), 256, 0, st>>>(n, x, incx, (float2*)xf);
            fl::count_launch();
            gemv_x2_kernel<false><<<(unsigned)((n + GEMV_SMEM_WARPS - 1) / GEMV_SMEM_WARPS), 32 * GEMV_SMEM_WARPS, 0,
                                    st>>>(n, (const float2*)A, lda, x, incx, (const float2*)xf, y, incy);
        }
        fl::count_launch();
        return cudaGetLastError();
    }
    if (dtype == FL_F64) {
        const unsigned gs = (((uintptr_t)A & 7u) == 0) ? gemv_smem_grid<double, double>(n) : 0u;
        if (gs) {
            gemv_smem_kernel<double, double><<<gs, 32 * GEMV_SMEM_WARPS, (n + GEMV_SMEM_PAD) * sizeof(double), st>>>(
                n, (const double*)A, lda, x, incx, nullptr, y, incy);
            fl::count_launch();
            return cudaGetLastError();
        }
        const int vec = (((uintptr_t)A & 7u) == 0) && aligned16(x);
        gemv_f64_kernel<<<blocks, 256, 0, st>>>(n, (const double*)A, lda, x, incx, y, incy, vec); fl::count_launch();
    } else {
        const unsigned gs = gemv_lo_smem_grid(dtype, A, n);
        if (gs) {  // x rounded while it is staged: no float32 copy in global memory
            const float* xs = xf_ready ? xf : nullptr;
            if (dtype == FL_F32)
                gemv_smem_kernel<float, float><<<gs, 32 * GEMV_SMEM_WARPS, (n + GEMV_SMEM_PAD) * sizeof(float), st>>>(
                    n, (const float*)A, lda, x, incx, xs, y, incy);
            else
                gemv_smem_kernel<__nv_bfloat16, float><<<gs, 32 * GEMV_SMEM_WARPS, (n + GEMV_SMEM_PAD) * sizeof(float), st>>>(
                    n, (const __nv_bfloat16*)A, lda, x, incx, xs, y, incy);
            fl::count_launch();
            return cudaGetLastError();
        }
        if (!xf_ready) { to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, incx, xf); fl::count_launch(); }
        if (dtype == FL_F32) {
            const int vec = (((uintptr_t)A & 3u) == 0) && aligned16(xf);
            gemv_lo_kernel<float><<<blocks, 256, 0, st>>>(n, (const float*)A, lda, xf, y, incy, vec); fl::count_launch();
        } else {
            const int vec = (((uintptr_t)A & 1u) == 0) && aligned16(xf);
            gemv_lo_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(n, (const __nv_bfloat16*)A, lda, xf, y, incy, vec); fl::count_launch();
        }
    }
    return cudaGetLastError();
}

// --------------------------------------------------- deterministic dots --
constexpr int RED_BLOCKS = 240;
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// partial[b] = Σ a_i b_i over this block's grid-stride share
__global__ void dot_partial_kernel(int64_t n, const double* a, const double* b, double* partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void sum_partials_kernel(const double* partial, int nb, double* out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = t;
}

// ------------------------------------------------------------- PCG parts --
struct TAVoid {
    const void* p;
};

struct CgScalars {
    double rz, rz_new, pq, rr, bb, alpha, beta, stop;
    int breakdown;
    int done;   // set once converged, broken down or out of iterations; later steps are no-ops
    int it;     // iterations performed
    int maxit;
};

__global__ void diag_inv_kernel(int64_t n, int dtype, const void* A, int64_t lda, double* dinv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d;
    if (dtype == FL_F64) d = ((const double*)A)[i * lda + i];
    else if (dtype == FL_F32) d = (double)((const float*)A)[i * lda + i];
    else d = (double)__bfloat162float(((const __nv_bfloat16*)A)[i * lda + i]);
    dinv[i] = 1.0 / d;
}

// r = b - Ax (or r = b when Ax is NULL); x_out = 0 if requested
__global__ void residual_kernel(int64_t n, const double* b, const double* Ax, double* r) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) r[i] = Ax ? b[i] - Ax[i] : b[i];
}

// z = dinv r, p = z, partials of r·z and r·r
__global__ void cg_start_kernel(int64_t n, const double* r, const double* dinv, double* z, double* p, float* pf,
                                double* prz, double* prr) {
    __shared__ double sh[32];
    double a = 0.0, c = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = dinv[i] * r[i];
        z[i] = zi;
        p[i] = zi;
        if (pf) pf[i] = (float)zi;
        a = fma(r[i], zi, a);
        c = fma(r[i], r[i], c);
    }
    const double ta = block_sum(a, sh);
    const double tc = block_sum(c, sh);
    if (threadIdx.x == 0) {
        prz[blockIdx.x] = ta;
        prr[blockIdx.x] = tc;
    }
}

__global__ void cg_init_scalars_kernel(const double* prz, const double* prr, int nb, CgScalars* s, double tol,
                                       int maxit) {
    __shared__ double sh[32];
    double a = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += prz[i];
        c += prr[i];
    }
    const double ta = block_sum(a, sh);
    const double tc = block_sum(c, sh);
    if (threadIdx.x == 0) {
        s->rz = ta;
        s->rr = tc;
        s->stop = tol * tol * tc;
        s->breakdown = 0;
        s->it = 0;
        s->maxit = maxit;
        s->done = (tc == 0.0 || maxit <= 0) ? 1 : 0;
    }
}

__global__ void cg_alpha_kernel(const double* ppq, int nb, CgScalars* s) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += ppq[i];
    const double t = block_sum(a, sh);
    if (threadIdx.x == 0) {
        s->pq = t;
        if (s->done) {
            s->alpha = 0.0;
        } else if (!(t > 0.0)) {
            s->breakdown = 1;
            s->done = 1;
            s->alpha = 0.0;
        } else {
            s->alpha = s->rz / t;
        }
    }
}

// u += α p, r -= α q, z = dinv r, partials of r·z, r·r
__global__ void cg_update_kernel(int64_t n, const CgScalars* s, double* u, double* r, double* z, const double* p,
                                 const double* q, const double* dinv, double* prz, double* prr) {
    __shared__ double sh[32];
    const double alpha = s->alpha;
    double a = 0.0, c = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = fma(alpha, p[i], u[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        const double zi = dinv[i] * ri;
        z[i] = zi;
        a = fma(ri, zi, a);
        c = fma(ri, ri, c);
    }
    const double ta = block_sum(a, sh);
    const double tc = block_sum(c, sh);
    if (threadIdx.x == 0) {
        prz[blockIdx.x] = ta;
        prr[blockIdx.x] = tc;
    }
}

__global__ void cg_beta_kernel(const double* prz, const double* prr, int nb, CgScalars* s) {
    __shared__ double sh[32];
    double a = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += prz[i];
        c += prr[i];
    }
    const double ta = block_sum(a, sh);
    const double tc = block_sum(c, sh);
    if (threadIdx.x == 0) {
        if (s->done) {
            s->beta = 0.0;
        } else {
            s->beta = ta / s->rz;
            s->rz = ta;
            s->rr = tc;
            s->it += 1;
            if (tc <= s->stop || s->it >= s->maxit) s->done = 1;
        }
    }
}

__global__ void cg_p_kernel(int64_t n, const CgScalars* s, const double* z, double* p, float* pf) {
    const double beta = s->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = fma(beta, p[i], z[i]);
        p[i] = pi;
        if (pf) pf[i] = (float)pi;
    }
}

__global__ void axpy_kernel(int64_t n, double a, const double* x, double* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], y[i]);
}

__global__ void zero_kernel(int64_t n, double* x) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = 0.0;
}

// ------------------------------------------------------- solver workspace --
// Partial-sum area of the persistent solvers (in doubles): per-block partials of up to three
// slots of 1024 (float32 pipelined CG: two parity sets of three slots), the float64
// partials of the refinement at PARTD_OFF, and the error flag at ERR_OFF.
constexpr int PART_DOUBLES = 8 * 1024;
constexpr int PARTD_OFF = 4 * 1024;
constexpr int ERR_OFF = 7 * 1024;

struct SolveWork {
    double *r, *z, *p, *q, *dinv, *dinv_lo, *d, *t, *sv, *prz, *prr, *ppq, *part;
    unsigned* gbar;  // grid-barrier counter of the persistent solver (own cache line)
    float* xf;
    float* fv[12];  // float32 vectors of the pipelined inner CG
    CgScalars* s;
    CgScalars* s_host;
};

static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

static int get_work(fl_ctx* h, int64_t n, SolveWork& w) {
    // one contiguous device block per handle, grown on demand; the layout below
    // (eight float64 vectors, three reduction buffers, one float32 vector, scalars)
    // is carved with the same 256-byte rounding that sizes it
    const size_t need = 9 * round256(n * sizeof(double)) + 3 * round256(RED_BLOCKS * sizeof(double)) +
                        round256(PART_DOUBLES * sizeof(double)) + round256(256) + 13 * round256(n * sizeof(float)) +
                        round256(sizeof(CgScalars));
    void* base = nullptr;
    if (h->solve_ws_bytes < need) {
        for (auto& g : h->cg_graphs) cudaGraphExecDestroy(g.exec);
        h->cg_graphs.clear();
        if (h->solve_ws) {
            cudaDeviceSynchronize();  // the cached blocks must be idle before another user takes them
            pool_dev_free(h->solve_ws);
            pool_host_free(h->solve_host);
        }
        h->solve_ws = nullptr;
        h->solve_host = nullptr;
        h->solve_ws_bytes = 0;
        if (pool_dev_alloc(&h->solve_ws, need) != cudaSuccess) return set_err(h, FL_ENOMEM, "solver workspace");
        if (pool_host_alloc(&h->solve_host, sizeof(CgScalars)) != cudaSuccess)
            return set_err(h, FL_ENOMEM, "pinned solver scalars");
        h->solve_ws_bytes = need;
    }
    base = h->solve_ws;
    char* c = (char*)base;
    auto take = [&](size_t bytes) {
        char* p = c;
        c += round256(bytes);
        return (void*)p;
    };
    w.r = (double*)take(n * sizeof(double));
    w.z = (double*)take(n * sizeof(double));
    w.p = (double*)take(n * sizeof(double));
    w.q = (double*)take(n * sizeof(double));
    w.dinv = (double*)take(n * sizeof(double));
    w.dinv_lo = (double*)take(n * sizeof(double));
    w.d = (double*)take(n * sizeof(double));
    w.t = (double*)take(n * sizeof(double));
    w.sv = (double*)take(n * sizeof(double));
    w.prz = (double*)take(RED_BLOCKS * sizeof(double));
    w.prr = (double*)take(RED_BLOCKS * sizeof(double));
    w.ppq = (double*)take(RED_BLOCKS * sizeof(double));
    w.part = (double*)take(PART_DOUBLES * sizeof(double));
    w.gbar = (unsigned*)take(256);
    w.xf = (float*)take(n * sizeof(float));
    for (int k = 0; k < 12; ++k) w.fv[k] = (float*)take(n * sizeof(float));
    w.s = (CgScalars*)take(sizeof(CgScalars));
    w.s_host = (CgScalars*)h->solve_host;
    if ((size_t)(c - (char*)base) > need) return set_err(h, FL_EINVAL, "solver workspace layout exceeds its size");
    return FL_OK;
}

#define FL_CU(h, x)                                                                                        \
    do {                                                                                                   \
        cudaError_t e_ = (x);                                                                              \
        if (e_ != cudaSuccess) return set_err(h, FL_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------- persistent Jacobi-PCG --
// The whole iteration in one cooperative launch: rows of the matrix-vector product and
// vector entries are split over a fixed grid; after each phase every block adds the
// per-block partial sums in the same order, so all blocks hold bitwise identical
// scalars and take the same branch (no block can leave while others wait).
constexpr int PCG_THREADS = 512;  // one block of 16 warps per SM
constexpr int PCG_WARPS = PCG_THREADS / 32;
constexpr int PCG_MAX_BLOCKS = 1024;

template <typename T>
__device__ __forceinline__ T warp_total(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of NV values, identical in every thread: warp sums, then warp 0 sums the
// per-warp results in warp order.  sh holds NV * 33 values.
template <typename T, int NV>
__device__ __forceinline__ void block_totals(T (&v)[NV], T* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_total(v[k]);
    __syncthreads();  // sh may still be read from the previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + w] = v[k];
    __syncthreads();
    if (w == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const T t = warp_total(lane < PCG_WARPS ? sh[k * 32 + lane] : T(0));
            if (lane == 0) sh[NV * 32 + k] = t;
        }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = sh[NV * 32 + k];
}

// Sums over the blocks' partials part[k * 1024 + b], b < nb, in a fixed order (the same
// result in every block, so that all blocks take the same branch).
template <typename T, int NV>
__device__ __forceinline__ void grid_totals(T (&v)[NV], const T* part, const int (&slot)[NV], int nb, T* sh) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T a = 0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) a += __ldcg(part + slot[k] * 1024 + i);
        v[k] = a;
    }
    block_totals<T, NV>(v, sh);
}

// Entry v of a 16-byte vector of float64 (v < 2) or float32 (v < 4) values.
template <typename TA>
__device__ __forceinline__ TA vec_elem(const uint4& u, int v) {
    if constexpr (sizeof(TA) == 8) return v == 0 ? __hiloint2double((int)u.y, (int)u.x) : __hiloint2double((int)u.w, (int)u.z);
    else return __uint_as_float(v == 0 ? u.x : v == 1 ? u.y : v == 2 ? u.z : u.w);
}

template <bool SH, typename TX>
__device__ __forceinline__ TX xload(const TX* p) {
    if constexpr (SH) return *p;  // shared-memory copy
    else return __ldcg(p);
}

// Row `row` of A times x (float64 or float32 entries), one warp: 16-byte loads of A after
// peeling to an aligned start, six loads per lane in flight (the last round predicated,
// masked entries multiply zero); x is the block's shared-memory copy (SH) or, when it does
// not fit, read through L2 (other blocks rewrite it between products).
template <typename TA, typename TX, typename TS, bool SH>
__device__ __forceinline__ TS row_dot(const TA* __restrict__ a, const TX* __restrict__ x, int64_t n, int lane) {
    constexpr int V = 16 / sizeof(TA);  // entries per 16-byte load
    constexpr int U = 6;                // loads in flight per lane
    const int peel = (int)((V - (((uintptr_t)a / sizeof(TA)) & (V - 1))) & (V - 1));
    TS s[4] = {0, 0, 0, 0};
    const int head = (int)((int64_t)peel < n ? (int64_t)peel : n);
    if (lane < head) s[0] = (TS)a[lane] * (TS)xload<SH>(x + lane);
    const int64_t nv = (n - head) / V;  // whole vectors after the peel
    const uint4* av = reinterpret_cast<const uint4*>(a + head);
    const TX* xv = x + head;
    for (int64_t k0 = lane; k0 < nv; k0 += 32 * U) {
        uint4 u[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t k = k0 + 32 * j;
            u[j] = k < nv ? __ldcs(av + k) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t k = k0 + 32 * j < nv ? k0 + 32 * j : nv - 1;  // masked: a zero times a valid x
#pragma unroll
            for (int v = 0; v < V; ++v) s[j & 3] += (TS)vec_elem<TA>(u[j], v) * (TS)xload<SH>(xv + k * V + v);
        }
    }
    for (int64_t j = head + nv * V + lane; j < n; j += 32) s[1] += (TS)a[j] * (TS)xload<SH>(x + j);
    return warp_sum((s[0] + s[1]) + (s[2] + s[3]));
}

// The standalone float32 product with the persistent CG's row kernel: blocks of 16 warps (two
// per SM unless tuned otherwise), each block's rows a contiguous range, warp per row, six 16-byte
// loads per lane in flight; x staged in shared memory, rounded to float32 as it is staged.
// Measured against the 8-warp staged kernel it replaces for float32: 6.0 against 5.2 TB/s at
// n = 20000, 5.8 against 5.2 at n = 35693.
template <typename TA, typename TS>
__global__ void __launch_bounds__(512, 1)
    gemv_rows_kernel(int64_t n, const TA* __restrict__ A, int64_t lda, const double* __restrict__ x, int64_t incx,
                     const float* __restrict__ xf, double* __restrict__ y, int64_t incy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* xs = reinterpret_cast<TA*>(smem_raw);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        if constexpr (sizeof(TA) == 8) xs[i] = x[i * incx];
        else xs[i] = xf ? xf[i] : (float)x[i * incx];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t rb = (int64_t)blockIdx.x * n / gridDim.x, re = (int64_t)(blockIdx.x + 1) * n / gridDim.x;
    for (int64_t row = rb + warp; row < re; row += nw) {
        const TS t = row_dot<TA, TA, TS, true>(A + row * lda, xs, n, lane);
        if (lane == 0) y[row * incy] = (double)t;
    }
}

// blocks per SM of the row-dot product at size n: 0 when it does not apply (x does not fit the
// staging), else the tuned count (fl_tune_matvec), or two; *max_per_sm gets the occupancy limit
static int gemv_rows_per_sm(int64_t n, int* max_per_sm = nullptr) {
    const size_t smem = (size_t)n * sizeof(float);
    if (smem > GEMV_SMEM_MAX) return 0;
    static thread_local int ready_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (ready_dev != dev) {
        if (cudaFuncSetAttribute(gemv_rows_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)GEMV_SMEM_MAX) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        ready_dev = dev;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemv_rows_kernel<float, float>, 512, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    if (max_per_sm) *max_per_sm = per_sm;
    int p0 = 0, p1 = 0;
    if (tune_lookup(device_name(), "gemv_rows_f32", n, 1, 1, &p0, &p1) && p0 >= 1) return std::min(per_sm, p0);
    return std::min(per_sm, 2);
}

static void gemv_rows_launch(int per_sm, int64_t n, const float* A, int64_t lda, const double* x, int64_t incx,
                             const float* xf, double* y, int64_t incy, cudaStream_t st) {
    static thread_local int sms = 0, sms_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (sms_dev != dev) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sms_dev = dev;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(n, (int64_t)sms * per_sm);
    gemv_rows_kernel<float, float><<<grid, 512, (size_t)n * sizeof(float), st>>>(n, A, lda, x, incx, xf, y, incy);
}

static bool gemv_rows(int dtype, const void* A, int64_t lda, int64_t n, const double* x, int64_t incx, double* y,
                      int64_t incy, const float* xf, bool xf_ready, cudaStream_t st) {
    if (dtype != FL_F32 || ((uintptr_t)A & 3u) != 0) return false;
    const int per_sm = gemv_rows_per_sm(n);
    if (per_sm < 1) return false;
    gemv_rows_launch(per_sm, n, (const float*)A, lda, x, incx, xf_ready ? xf : nullptr, y, incy, st);
    return true;
}

// Persistent Jacobi-PCG in the Chronopoulos-Gear arrangement (one cooperative launch):
// the product is taken of the preconditioned residual, w = A z, and s = A p is carried by
// recurrence, so both inner products of a step come from one pass and a step needs two
// grid barriers:
//   M: w = A z for the block's own rows, partial delta = z.w
//   U: beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//      (beta = 0, alpha = gamma / delta first); p = z + beta p, s = w + beta s, u += alpha p,
//      r -= alpha s, z = D^-1 r; partial gamma = r.z and r.r
// Block b owns rows [b rpb, (b + 1) rpb) of the product and of every vector, so w never
// leaves shared memory.  T is the type of the matrix, the vectors and the scalars: float64
// for the plain solve, float32 for the inner solve of the refinement (whose float64
// residual corrects it), so that no float64 arithmetic (a slow pipe on this part) sits on
// the float32 iteration's critical path.  Every block sums the per-block partials in the
// same order, so all blocks hold the same scalars and take the same branch.
// MODE 2: the block's rows of A stay in shared memory for the whole solve (and z is
// staged there each step); MODE 1: z staged, A streamed; MODE 0: both streamed.
// Breakdown: a non-positive denominator (p.Ap <= 0).
// Per-block view of the persistent CG: the block's rows [r0, r1), its shared-memory
// buffers and the work vectors (all indexed by global row).
template <typename T>
struct CgBlock {
    int64_t n, r0, r1, lds;
    const T* A;  // global matrix (MODE < 2)
    int64_t lda;
    T* xs;  // [lds] staged z (MODE >= 1)
    T* ws;  // [rpb] products of the own rows
    T* As;  // [rpb][lds] own rows of A (MODE 2)
    T *u, *r, *z, *p, *sv, *dv, *part;
    unsigned* gbar;
    int* err;
    uint64_t wait_ns;  // bound of each grid-barrier wait
    T* sh;
    int nb, lane, warp;
};

// Copy of the block's rows of A into shared memory (MODE 2), zero padding of the staged vector.
template <typename T, int MODE>
__device__ __forceinline__ void cg_block_setup(const CgBlock<T>& c) {
    if constexpr (MODE == 2) {
        for (int64_t row = c.r0; row < c.r1; ++row)
            for (int64_t j = threadIdx.x; j < c.lds; j += blockDim.x)
                c.As[(row - c.r0) * c.lds + j] = j < c.n ? c.A[row * c.lda + j] : T(0);
    }
    if constexpr (MODE >= 1)
        for (int64_t j = c.n + threadIdx.x; j < c.lds; j += blockDim.x) c.xs[j] = T(0);
}

// One Jacobi-PCG solve M u = rhs from u = 0 in the Chronopoulos-Gear arrangement, every
// block on its own rows.  Returns false when a grid barrier gave up (err is set).
template <typename T, int MODE>
__device__ __forceinline__ bool cg_block_solve(const CgBlock<T>& c, const double* __restrict__ rhs, double tol,
                                               int maxit, unsigned& epoch, int& it_out, int& breakdown_out,
                                               T& rr_out, T& rr0_out) {
    constexpr int V = 16 / sizeof(T);
    constexpr int D_ = 0, G_ = 1, R_ = 2;
    const int64_t n = c.n, r0 = c.r0, r1 = c.r1;
    const int lane = c.lane, warp = c.warp, nb = c.nb;
    T* sh = c.sh;
    // start: u = 0, r = rhs, z = D^-1 r, p = s = 0
    {
        T v[2] = {0, 0};
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const T ri = (T)rhs[i];
            const T zi = c.dv[i] * ri;
            c.u[i] = 0;
            c.r[i] = ri;
            c.z[i] = zi;
            c.p[i] = 0;
            c.sv[i] = 0;
            v[0] += ri * zi;
            v[1] += ri * ri;
        }
        block_totals<T, 2>(v, sh);
        if (threadIdx.x == 0) {
            c.part[G_ * 1024 + blockIdx.x] = v[0];
            c.part[R_ * 1024 + blockIdx.x] = v[1];
        }
    }
    if (!tc::grid_barrier(c.gbar, epoch, nb, c.err, c.wait_ns)) return false;
    T gamma, rr0;
    {
        T v[2];
        grid_totals<T, 2>(v, c.part, {G_, R_}, nb, sh);
        gamma = v[0];
        rr0 = v[1];
    }
    const T stop = (T)(tol * tol) * rr0;
    T rr = rr0, gamma_prev = 1, alpha_prev = 1;
    int it = 0, breakdown = 0;
    while (rr > stop && it < maxit) {
        // M: w = A z on the own rows, partial z.w
        if constexpr (MODE >= 1) {
            const int64_t nq = n * (int64_t)sizeof(T) / 16;  // z is 256-byte aligned
            const uint4* src = reinterpret_cast<const uint4*>(c.z);
            uint4* dst = reinterpret_cast<uint4*>(c.xs);
            for (int64_t i0 = threadIdx.x; i0 < nq; i0 += 4 * blockDim.x) {
                uint4 q[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j * blockDim.x < nq) q[j] = __ldcg(src + i0 + j * blockDim.x);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j * blockDim.x < nq) dst[i0 + j * blockDim.x] = q[j];
            }
            for (int64_t i = nq * 16 / (int64_t)sizeof(T) + threadIdx.x; i < n; i += blockDim.x) c.xs[i] = __ldcg(c.z + i);
            __syncthreads();
        }
        T dl[1] = {0};
        for (int64_t row = r0 + warp; row < r1; row += PCG_WARPS) {
            T acc;
            if constexpr (MODE == 2) {
                const uint4* a4 = reinterpret_cast<const uint4*>(c.As + (row - r0) * c.lds);
                const uint4* x4 = reinterpret_cast<const uint4*>(c.xs);
                T s0 = 0, s1 = 0;
                for (int64_t q = lane; q < c.lds / V; q += 32) {
                    const uint4 av = a4[q], xv = x4[q];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (v & 1) s1 = fma(vec_elem<T>(av, v), vec_elem<T>(xv, v), s1);
                        else s0 = fma(vec_elem<T>(av, v), vec_elem<T>(xv, v), s0);
                    }
                }
                acc = warp_total(s0 + s1);
            } else {
                acc = row_dot<T, T, T, (MODE == 1)>(c.A + row * c.lda, MODE == 1 ? c.xs : c.z, n, lane);
            }
            if (lane == 0) {
                c.ws[row - r0] = acc;
                dl[0] += (MODE >= 1 ? c.xs[row] : __ldcg(c.z + row)) * acc;
            }
        }
        block_totals<T, 1>(dl, sh);
        if (threadIdx.x == 0) c.part[D_ * 1024 + blockIdx.x] = dl[0];
        if (!tc::grid_barrier(c.gbar, epoch, nb, c.err, c.wait_ns)) return false;
        // U
        T delta[1];
        grid_totals<T, 1>(delta, c.part, {D_}, nb, sh);
        const T beta = (it == 0) ? T(0) : gamma / gamma_prev;
        const T den = (it == 0) ? delta[0] : delta[0] - beta * gamma / alpha_prev;
        if (!(den > T(0))) {
            breakdown = 1;
            break;
        }
        const T alpha = gamma / den;
        T v[2] = {0, 0};
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const T pi = fma(beta, c.p[i], c.z[i]);
            const T si = fma(beta, c.sv[i], c.ws[i - r0]);
            c.p[i] = pi;
            c.sv[i] = si;
            c.u[i] = fma(alpha, pi, c.u[i]);
            const T ri = fma(-alpha, si, c.r[i]);
            c.r[i] = ri;
            const T zi = c.dv[i] * ri;
            c.z[i] = zi;
            v[0] = fma(ri, zi, v[0]);
            v[1] = fma(ri, ri, v[1]);
        }
        block_totals<T, 2>(v, sh);
        if (threadIdx.x == 0) {
            c.part[G_ * 1024 + blockIdx.x] = v[0];
            c.part[R_ * 1024 + blockIdx.x] = v[1];
        }
        if (!tc::grid_barrier(c.gbar, epoch, nb, c.err, c.wait_ns)) return false;
        gamma_prev = gamma;
        alpha_prev = alpha;
        grid_totals<T, 2>(v, c.part, {G_, R_}, nb, sh);
        gamma = v[0];
        rr = v[1];
        ++it;
    }
    it_out = it;
    breakdown_out = breakdown;
    rr_out = rr;
    rr0_out = rr0;
    return true;
}

// The product of the block's own rows with xg (all n entries): xg staged in shared memory
// (MODE >= 1), one warp per row, the results in c.ws; ends with a block barrier.
template <typename T, int MODE>
__device__ __forceinline__ void rows_product(const CgBlock<T>& c, const T* __restrict__ xg) {
    constexpr int V = 16 / sizeof(T);
    const int64_t n = c.n;
    if constexpr (MODE >= 1) {
        const int64_t nq = n * (int64_t)sizeof(T) / 16;  // xg is 256-byte aligned
        const uint4* src = reinterpret_cast<const uint4*>(xg);
        uint4* dst = reinterpret_cast<uint4*>(c.xs);
        for (int64_t i0 = threadIdx.x; i0 < nq; i0 += 4 * blockDim.x) {
            uint4 q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (i0 + j * blockDim.x < nq) q[j] = __ldcg(src + i0 + j * blockDim.x);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (i0 + j * blockDim.x < nq) dst[i0 + j * blockDim.x] = q[j];
        }
        for (int64_t i = nq * 16 / (int64_t)sizeof(T) + threadIdx.x; i < n; i += blockDim.x) c.xs[i] = __ldcg(xg + i);
        __syncthreads();
    }
    for (int64_t row = c.r0 + c.warp; row < c.r1; row += PCG_WARPS) {
        T acc;
        if constexpr (MODE == 2) {
            const uint4* a4 = reinterpret_cast<const uint4*>(c.As + (row - c.r0) * c.lds);
            const uint4* x4 = reinterpret_cast<const uint4*>(c.xs);
            T s0 = 0, s1 = 0;
            for (int64_t q = c.lane; q < c.lds / V; q += 32) {
                const uint4 av = a4[q], xv = x4[q];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (v & 1) s1 = fma(vec_elem<T>(av, v), vec_elem<T>(xv, v), s1);
                    else s0 = fma(vec_elem<T>(av, v), vec_elem<T>(xv, v), s0);
                }
            }
            acc = warp_total(s0 + s1);
        } else {
            acc = row_dot<T, T, T, (MODE == 1)>(c.A + row * c.lda, MODE == 1 ? c.xs : xg, n, c.lane);
        }
        if (c.lane == 0) c.ws[row - c.r0] = acc;
    }
    __syncthreads();
}

// Float32 work vectors of the pipelined CG (x the solution; m double-buffered by step parity).
struct PipeVecs {
    float *x, *r, *u, *w, *z, *q, *s, *p, *m0, *m1, *dv;
};

// One Jacobi-PCG solve M x = rhs from x = 0 in the pipelined arrangement (one global
// synchronisation per step, Ghysels & Vanroose): with u = D^-1 r, w = A u, m = D^-1 w and
// n = A m, a step takes gamma = r.u, delta = w.u (and r.r for the stopping test) from the
// previous step's partials, forms n = A m for the own rows, updates
//   z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p,
//   x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z,
// and writes m = D^-1 w and the next partials before the step's only grid barrier.  The
// partials (two sets of three slots) and m alternate by step parity, so a block that runs
// ahead never overwrites what a slower block still reads.  The recurrences drift from the
// true residual by a few float32 roundings per step; in the refinement every step is
// judged and corrected by the float64 residual.  breakdown_out is set for a non-positive
// p.Ap while ||r|| > 1e-3 ||r_0||; below that it is lost accuracy and just ends the solve.
template <int MODE>
__device__ __forceinline__ bool pipe_block_solve(const CgBlock<float>& c, const PipeVecs& v,
                                                 const double* __restrict__ rhs, double tol, int maxit,
                                                 unsigned& epoch, int& it_out, int& breakdown_out, float& rr_out,
                                                 float& rr0_out) {
    const int64_t r0 = c.r0, r1 = c.r1;
    const int nb = c.nb;
    float* sh = c.sh;
    // start: x = 0, r = rhs, u = D^-1 r, z = q = s = p = 0
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const float ri = (float)rhs[i];
        v.x[i] = 0.f;
        v.r[i] = ri;
        v.u[i] = v.dv[i] * ri;
        v.z[i] = 0.f;
        v.q[i] = 0.f;
        v.s[i] = 0.f;
        v.p[i] = 0.f;
    }
    if (!tc::grid_barrier(c.gbar, epoch, nb, c.err, c.wait_ns)) return false;
    // w = A u, m = D^-1 w, partials of r.u, w.u, r.r (set 0)
    rows_product<float, MODE>(c, v.u);
    {
        float t[3] = {0.f, 0.f, 0.f};
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const float ri = v.r[i], ui = v.u[i], wi = c.ws[i - r0];
            v.w[i] = wi;
            v.m0[i] = v.dv[i] * wi;
            t[0] = fmaf(ri, ui, t[0]);
            t[1] = fmaf(wi, ui, t[1]);
            t[2] = fmaf(ri, ri, t[2]);
        }
        block_totals<float, 3>(t, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) c.part[k * 1024 + blockIdx.x] = t[k];
    }
    if (!tc::grid_barrier(c.gbar, epoch, nb, c.err, c.wait_ns)) return false;
    float gamma_prev = 1.f, alpha_prev = 1.f, rr0 = 0.f, stop = 0.f, rr = 0.f;
    int it = 0, breakdown = 0;
    for (;;) {
        const int set = it & 1;
        float tot[3];
        grid_totals<float, 3>(tot, c.part, {3 * set, 3 * set + 1, 3 * set + 2}, nb, sh);
        const float gamma = tot[0], delta = tot[1];
        rr = tot[2];
        if (it == 0) {
            rr0 = rr;
            stop = (float)(tol * tol) * rr0;
        }
        if (!(rr > stop) || it >= maxit) break;
        const float beta = (it == 0) ? 0.f : gamma / gamma_prev;
        const float den = (it == 0) ? delta : delta - beta * gamma / alpha_prev;
        if (!(den > 0.f)) {
            // p.Ap <= 0 while the residual is still above 1e-3 of its start: the matrix is not
            // SPD.  Below that: the float32 recurrences have lost their accuracy; the solve ends
            // with the current x (the refinement's float64 residual decides what comes next)
            breakdown = (it == 0 || rr > 1e-6f * rr0) ? 1 : 0;
            break;
        }
        const float alpha = gamma / den;
        const float* m_cur = set ? v.m1 : v.m0;
        float* m_next = set ? v.m0 : v.m1;
        rows_product<float, MODE>(c, m_cur);
        float t[3] = {0.f, 0.f, 0.f};
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const float ni = c.ws[i - r0];
            const float mi = (MODE >= 1) ? c.xs[i] : __ldcg(m_cur + i);
            const float ui = v.u[i], wi = v.w[i];
            const float zi = fmaf(beta, v.z[i], ni);
            const float qi = fmaf(beta, v.q[i], mi);
            const float si = fmaf(beta, v.s[i], wi);
            const float pi = fmaf(beta, v.p[i], ui);
            v.z[i] = zi;
            v.q[i] = qi;
            v.s[i] = si;
            v.p[i] = pi;
            v.x[i] = fmaf(alpha, pi, v.x[i]);
            const float rn = fmaf(-alpha, si, v.r[i]);
            const float un = fmaf(-alpha, qi, ui);
            const float wn = fmaf(-alpha, zi, wi);
            v.r[i] = rn;
            v.u[i] = un;
            v.w[i] = wn;
            m_next[i] = v.dv[i] * wn;
            t[0] = fmaf(rn, un, t[0]);
            t[1] = fmaf(wn, un, t[1]);
            t[2] = fmaf(rn, rn, t[2]);
        }
        block_totals<float, 3>(t, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) c.part[(3 * (set ^ 1) + k) * 1024 + blockIdx.x] = t[k];
        if (!tc::grid_barrier(c.gbar, epoch, nb, c.err, c.wait_ns)) return false;
        gamma_prev = gamma;
        alpha_prev = alpha;
        ++it;
    }
    it_out = it;
    breakdown_out = breakdown;
    rr_out = rr;
    rr0_out = rr0;
    return true;
}

template <typename T, int MODE>
__device__ __forceinline__ CgBlock<T> cg_block(int64_t n, int64_t rpb, int64_t lds, const T* A, int64_t lda, T* u,
                                               T* r, T* z, T* p, T* sv, T* dv, T* part, unsigned* gbar, int* err,
                                               uint64_t wait_ns, T* sh, unsigned char* smem_raw) {
    constexpr int V = 16 / sizeof(T);
    CgBlock<T> c;
    c.n = n;
    c.r0 = blockIdx.x * rpb;
    c.r1 = (c.r0 + rpb < n) ? c.r0 + rpb : n;
    c.lds = lds;
    c.A = A;
    c.lda = lda;
    const int64_t rpb_pad = (rpb + V - 1) / V * V;
    c.xs = reinterpret_cast<T*>(smem_raw);
    c.ws = c.xs + (MODE >= 1 ? lds : 0);
    c.As = c.ws + rpb_pad;
    c.u = u;
    c.r = r;
    c.z = z;
    c.p = p;
    c.sv = sv;
    c.dv = dv;
    c.part = part;
    c.gbar = gbar;
    c.err = err;
    c.wait_ns = wait_ns;
    c.sh = sh;
    c.nb = gridDim.x;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    return c;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(PCG_THREADS, 1)
    pcg_persistent_kernel(int64_t n, int64_t rpb, int64_t lds, const T* __restrict__ A, int64_t lda,
                          const double* __restrict__ dinv, const double* __restrict__ rhs, double* d, T* u, T* r,
                          T* z, T* p, T* sv, T* dv, T* part, unsigned* gbar, CgScalars* S, double tol, int maxit,
                          int* err, unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T sh[2 * 33];
    const CgBlock<T> c = cg_block<T, MODE>(n, rpb, lds, A, lda, u, r, z, p, sv, dv, part, gbar, err, wait_ns, sh,
                                                 smem_raw);
    cg_block_setup<T, MODE>(c);
    if constexpr (sizeof(T) == 4)
        for (int64_t i = c.r0 + threadIdx.x; i < c.r1; i += blockDim.x) dv[i] = (T)dinv[i];
    unsigned epoch = 0;
    int it = 0, breakdown = 0;
    T rr = 0, rr0 = 0;
    if (!cg_block_solve<T, MODE>(c, rhs, tol, maxit, epoch, it, breakdown, rr, rr0)) return;
    if constexpr (sizeof(T) == 4)
        for (int64_t i = c.r0 + threadIdx.x; i < c.r1; i += blockDim.x) d[i] = (double)u[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->rr = (double)rr;
        S->stop = (double)((T)(tol * tol) * rr0);
        S->it = it;
        S->breakdown = breakdown;
        S->done = 1;
        S->rz = (double)rr0;  // initial residual norm^2, read back by the host
    }
}

// Float64 iterative refinement around the float32 persistent CG, in one cooperative launch
// (the host version reads the residual back after every step): per step the float64
// residual r = b - A u of the own rows (u = 0 first, so r = b), the stopping test
// ||r|| <= tol ||b|| from the same totals in every block, the float32 solve M d = r, and
// u += d.  The float32 rows of M are copied into shared memory once for all steps (MODE 2).
// Stops unconverged after max_outer steps or after three steps without a smaller residual.
struct RefineOut {
    double rr, bb;
    int outer, inner, status;  // status: 0 converged, 1 step limit, 2 breakdown
};

template <int MODE>
__global__ void __launch_bounds__(PCG_THREADS, 1)
    refine_persistent_kernel(int64_t n, int64_t rpb, int64_t lds, const double* __restrict__ A64, int64_t lda,
                             const float* __restrict__ A32, int64_t ld32, const double* __restrict__ dinv32,
                             const double* __restrict__ b, double* u, double* r64, const PipeVecs v,
                             float* partf, double* partd, unsigned* gbar, RefineOut* out, double tol,
                             double inner_tol, int max_outer, int inner_maxit, int* err,
                             unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float sh[3 * 33];
    __shared__ double shd[33];
    const CgBlock<float> c = cg_block<float, MODE>(n, rpb, lds, A32, ld32, v.x, v.r, v.z, v.p, v.s, v.dv, partf,
                                                   gbar, err, wait_ns, sh, smem_raw);
    cg_block_setup<float, MODE>(c);
    for (int64_t i = c.r0 + threadIdx.x; i < c.r1; i += blockDim.x) {
        v.dv[i] = (float)dinv32[i];
        u[i] = 0.0;
    }
    unsigned epoch = 0;
    double bb = 0.0, rr = 0.0, rr_prev = 0.0;
    int outer = 0, inner = 0, status = 1, stalled = 0;
    for (;;) {
        // float64 residual of the own rows (one warp per row; u is complete after the barrier)
        double rv[1] = {0.0};
        for (int64_t row = c.r0 + c.warp; row < c.r1; row += PCG_WARPS) {
            const double acc = outer == 0 ? 0.0 : row_dot<double, double, double, false>(A64 + row * lda, u, n, c.lane);
            if (c.lane == 0) {
                const double ri = b[row] - acc;
                r64[row] = ri;
                rv[0] = fma(ri, ri, rv[0]);
            }
        }
        block_totals<double, 1>(rv, shd);
        if (threadIdx.x == 0) partd[blockIdx.x] = rv[0];
        if (!tc::grid_barrier(gbar, epoch, c.nb, err, c.wait_ns)) return;
        grid_totals<double, 1>(rv, partd, {0}, c.nb, shd);
        rr = rv[0];
        if (outer == 0) bb = rr;
        if (rr <= tol * tol * bb) {
            status = 0;
            break;
        }
        if (outer >= max_outer) break;
        // three steps in a row without a smaller float64 residual: stop (not converged)
        stalled = (outer > 0 && !(rr < rr_prev)) ? stalled + 1 : 0;
        if (stalled >= 3) break;
        rr_prev = rr;
        int it = 0, breakdown = 0;
        float irr = 0.f, irr0 = 0.f;
        // the correction is solved no further than the outer test needs: a reduction by
        // tol ||b|| / ||r|| brings the residual to the target, half of it leaves a margin
        // for the float32 recurrences (every block has the same rr and bb)
        const double step_tol = fmax(inner_tol, 0.5 * tol * sqrt(bb / rr));
        if (!pipe_block_solve<MODE>(c, v, r64, step_tol, inner_maxit, epoch, it, breakdown, irr, irr0)) return;
        inner += it;
        if (breakdown) {
            status = 2;
            break;
        }
        for (int64_t i = c.r0 + threadIdx.x; i < c.r1; i += blockDim.x) u[i] += (double)v.x[i];
        ++outer;
        if (!tc::grid_barrier(gbar, epoch, c.nb, err, c.wait_ns)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->rr = rr;
        out->bb = bb;
        out->outer = outer;
        out->inner = inner;
        out->status = status;
    }
}

// Shared-memory plan of the persistent kernels: MODE 2 (rows of M resident), 1 (z staged)
// or 0; false if not even the row products fit.
static bool persistent_plan(int64_t n, size_t es, int blocks, int optin, int* mode, size_t* smem, int64_t* rpb,
                            int64_t* lds) {
    const int64_t V = 16 / (int64_t)es;
    *rpb = (n + blocks - 1) / blocks;
    const int64_t rpb_pad = (*rpb + V - 1) / V * V;
    *lds = (n + V - 1) / V * V;
    const size_t budget = optin > 4096 ? (size_t)optin - 2048 : 0;  // room for the static reduction buffers
    if ((size_t)(*lds + rpb_pad + *rpb * *lds) * es <= budget) {
        *mode = 2;
        *smem = (size_t)(*lds + rpb_pad + *rpb * *lds) * es;
    } else if ((size_t)(*lds + rpb_pad) * es <= budget) {
        *mode = 1;
        *smem = (size_t)(*lds + rpb_pad) * es;
    } else if ((size_t)rpb_pad * es <= budget) {
        *mode = 0;
        *smem = (size_t)rpb_pad * es;
    } else {
        return false;
    }
    return true;
}

// Launch the persistent solver if the device supports cooperative launches and the grid
// fits; returns false (nothing launched) otherwise.
template <typename T, int MODE>
static const void* pcg_fn() {
    return (const void*)pcg_persistent_kernel<T, MODE>;
}

static bool pcg_persistent(fl_ctx* h, SolveWork& w, int64_t n, int dtype, const void* M, int64_t ldm,
                           const double* dinv, const double* rhs, double* d, double tol, int maxit, cudaStream_t st,
                           int* status) {
    if (dtype == FL_BF16 || h->no_persistent) return false;
    int dev = 0, coop = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop || sms < 1) return false;
    const bool f64 = dtype == FL_F64;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const int blocks = std::min(sms, PCG_MAX_BLOCKS);
    int mode = 0;
    size_t smem = 0;
    int64_t rpb = 0, lds = 0;
    if (!persistent_plan(n, es, blocks, optin, &mode, &smem, &rpb, &lds)) return false;
    const void* fn = f64 ? (mode == 2 ? pcg_fn<double, 2>() : mode == 1 ? pcg_fn<double, 1>() : pcg_fn<double, 0>())
                         : (mode == 2 ? pcg_fn<float, 2>() : mode == 1 ? pcg_fn<float, 1>() : pcg_fn<float, 0>());
    int per_sm = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 16)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PCG_THREADS, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    int* err = reinterpret_cast<int*>(w.part + ERR_OFF);
    if (cudaMemsetAsync(w.gbar, 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // vectors: float64 ones in place (u is d itself); float32 ones in the first halves of the
    // float64 work vectors (u in q, whose product w stays in shared memory), D^-1 in xf
    void* u = f64 ? (void*)d : (void*)w.q;
    void* dv = f64 ? (void*)dinv : (void*)w.xf;
    void* part = (void*)w.part;
    const TAVoid Mv{M};
    void* args[] = {(void*)&n,   (void*)&rpb,  (void*)&lds,  (void*)&Mv.p,  (void*)&ldm,   (void*)&dinv,
                    (void*)&rhs, (void*)&d,    (void*)&u,    (void*)&w.r,   (void*)&w.z,   (void*)&w.p,
                    (void*)&w.sv, (void*)&dv,  (void*)&part, (void*)&w.gbar, (void*)&w.s,  (void*)&tol,
                    (void*)&maxit, (void*)&err, (void*)&h->wait_ns};
    const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(PCG_THREADS), args, smem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    fl::count_launch();
    *status = FL_OK;
    return true;
}

// Launch the refinement kernel (float32 inner matrix) if cooperative launches are supported
// and the grid fits; returns false (nothing launched) otherwise.
static bool refine_persistent(fl_ctx* h, SolveWork& w, int64_t n, const double* A64, int64_t lda, const float* A32,
                              int64_t ld32, const double* b, double* u, double tol, double inner_tol, int max_outer,
                              int inner_maxit, cudaStream_t st) {
    if (h->no_persistent) return false;
    int dev = 0, coop = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop || sms < 1) return false;
    const int blocks = std::min(sms, PCG_MAX_BLOCKS);
    int mode = 0;
    size_t smem = 0;
    int64_t rpb = 0, lds = 0;
    if (!persistent_plan(n, sizeof(float), blocks, optin, &mode, &smem, &rpb, &lds)) return false;
    const void* fn = mode == 2   ? (const void*)refine_persistent_kernel<2>
                     : mode == 1 ? (const void*)refine_persistent_kernel<1>
                                 : (const void*)refine_persistent_kernel<0>;
    int per_sm = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 16)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PCG_THREADS, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    int* err = reinterpret_cast<int*>(w.part + ERR_OFF);
    if (cudaMemsetAsync(w.gbar, 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // float32 vectors of the pipelined CG in fv; float32 partials (two sets of three slots)
    // at the start of part, float64 partials at PARTD_OFF
    float* partf = reinterpret_cast<float*>(w.part);
    double* partd = w.part + PARTD_OFF;
    RefineOut* out = reinterpret_cast<RefineOut*>(w.s);
    const double* dinv32 = w.dinv_lo;
    double* r64 = w.t;
    PipeVecs v;
    v.x = w.fv[0];
    v.r = w.fv[1];
    v.u = w.fv[2];
    v.w = w.fv[3];
    v.z = w.fv[4];
    v.q = w.fv[5];
    v.s = w.fv[6];
    v.p = w.fv[7];
    v.m0 = w.fv[8];
    v.m1 = w.fv[9];
    v.dv = w.fv[10];
    void* args[] = {(void*)&n,    (void*)&rpb,    (void*)&lds,  (void*)&A64,       (void*)&lda,
                    (void*)&A32,  (void*)&ld32,   (void*)&dinv32, (void*)&b,       (void*)&u,
                    (void*)&r64,  (void*)&v,      (void*)&partf, (void*)&partd,    (void*)&w.gbar,
                    (void*)&out,  (void*)&tol,    (void*)&inner_tol, (void*)&max_outer, (void*)&inner_maxit,
                    (void*)&err,  (void*)&h->wait_ns};
    const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(PCG_THREADS), args, smem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    fl::count_launch();
    return true;
}

// Jacobi-PCG on y = M x (M of type dtype) for M d = rhs from d = 0, relative tolerance tol
// (||rhs - M d|| by the recursion).  The iterations run in batches of CG_BATCH captured in a
// CUDA graph (cached per handle); the scalars are read back once per batch, and steps after
// convergence, breakdown or the iteration limit are no-ops on the device.
constexpr int CG_BATCH = 8;

static void enqueue_cg_iteration(SolveWork& w, int64_t n, int dtype, const void* M, int64_t ldm, const double* dinv,
                                 double* d, float* pf, cudaStream_t st) {
    gemv(dtype, M, ldm, n, w.p, 1, w.q, 1, w.xf, st, pf != nullptr);
    dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, w.p, w.q, w.ppq);
    cg_alpha_kernel<<<1, 256, 0, st>>>(w.ppq, RED_BLOCKS, w.s);
    cg_update_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, w.s, d, w.r, w.z, w.p, w.q, dinv, w.prz, w.prr);
    cg_beta_kernel<<<1, 256, 0, st>>>(w.prz, w.prr, RED_BLOCKS, w.s);
    cg_p_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, w.s, w.z, w.p, pf);
}

static int cg_graph(fl_ctx* h, SolveWork& w, int64_t n, int dtype, const void* M, int64_t ldm, const double* dinv,
                    double* d, float* pf, cudaGraphExec_t* exec) {
    CgGraphKey key{n, dtype, M, ldm, dinv, d, w.r, pf};
    for (auto& e : h->cg_graphs)
        if (e.key == key) {
            *exec = e.exec;
            return FL_OK;
        }
    if (!h->cap_stream) FL_CU(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const uint64_t before = fl_launch_count();
    cudaGraph_t g = nullptr;
    FL_CU(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int b = 0; b < CG_BATCH; ++b) enqueue_cg_iteration(w, n, dtype, M, ldm, dinv, d, pf, h->cap_stream);
    cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, h->cap_stream);
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
    fl::count_launch(-(int)(fl_launch_count() - before));  // captured, not launched
    if (ec != cudaSuccess) return set_err(h, FL_ECUDA, std::string("CG graph capture: ") + cudaGetErrorString(ec));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return set_err(h, FL_ECUDA, std::string("CG graph instantiate: ") + cudaGetErrorString(ei));
    h->cg_graphs.push_back({key, ex});
    *exec = ex;
    return FL_OK;
}

static int pcg(fl_ctx* h, SolveWork& w, int64_t n, int dtype, const void* M, int64_t ldm, const double* dinv,
               const double* rhs, double* d, double tol, int maxit, int* its, double* relres, cudaStream_t st) {
    int pst = FL_OK;
    if (pcg_persistent(h, w, n, dtype, M, ldm, dinv, rhs, d, tol, maxit, st, &pst)) {
        int err = 0;
        FL_CU(h, cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        FL_CU(h, cudaMemcpyAsync(&err, w.part + ERR_OFF, sizeof(int), cudaMemcpyDeviceToHost, st));
        FL_CU(h, cudaStreamSynchronize(st));
        if (err != 0) return set_err(h, FL_ETIMEOUT, "a grid barrier of the persistent solver gave up");
        const CgScalars& S = *w.s_host;
        *its = S.it;
        *relres = (S.rz > 0.0) ? std::sqrt(S.rr / S.rz) : 0.0;
        if (S.breakdown) return set_err(h, FL_ENOTSPD, "CG breakdown: p^T A p <= 0");
        return (S.rr <= S.stop) ? FL_OK : FL_ENOTCONV;
    }
    const unsigned g = (unsigned)((n + 255) / 256);
    zero_kernel<<<g, 256, 0, st>>>(n, d); fl::count_launch();
    residual_kernel<<<g, 256, 0, st>>>(n, rhs, nullptr, w.r); fl::count_launch();
    float* pf = (dtype == FL_F64) ? nullptr : w.xf;
    cg_start_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, w.r, dinv, w.z, w.p, pf, w.prz, w.prr); fl::count_launch();
    cg_init_scalars_kernel<<<1, 256, 0, st>>>(w.prz, w.prr, RED_BLOCKS, w.s, tol, maxit); fl::count_launch();
    FL_CU(h, cudaGetLastError());
    FL_CU(h, cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    FL_CU(h, cudaStreamSynchronize(st));
    const double rr0 = w.s_host->rr;
    *its = 0;
    *relres = 0.0;
    if (rr0 == 0.0) return FL_OK;
    cudaGraphExec_t ex = nullptr;
    int r = cg_graph(h, w, n, dtype, M, ldm, dinv, d, pf, &ex);
    if (r != FL_OK) return r;
    const int per_iter = (dtype == FL_F64) ? 6 : 6;  // gemv + 5 (the float copy of p comes from cg_p)
    while (!w.s_host->done) {
        FL_CU(h, cudaGraphLaunch(ex, st));
        fl::count_launch(CG_BATCH * per_iter);
        FL_CU(h, cudaStreamSynchronize(st));
    }
    *its = w.s_host->it;
    *relres = std::sqrt(w.s_host->rr / rr0);
    if (w.s_host->breakdown) return set_err(h, FL_ENOTSPD, "CG breakdown: p^T A p <= 0");
    return (w.s_host->rr <= w.s_host->stop) ? FL_OK : FL_ENOTCONV;
}

}  // namespace fl

using namespace fl;

extern "C" {

int fl_matvec(int dtype, const void* A_dev, int64_t lda, int64_t n, int nrhs, const double* X_dev, int64_t ldx,
              double* Y_dev, int64_t ldy, void* stream) {
    if (!A_dev || !X_dev || !Y_dev || n < 1 || nrhs < 1 || lda < n || ldx < nrhs || ldy < nrhs) return FL_EINVAL;
    if (dtype != FL_F64 && dtype != FL_F32 && dtype != FL_BF16 && dtype != FL_F32X2) return FL_EINVAL;
    if (dtype == FL_F32X2 && ((uintptr_t)A_dev & 7u) != 0) return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    float* xf = nullptr;  // copy of x (float32, or hi + lo pairs), only where x does not fit the staging
    if (dtype == FL_F32X2) {
        if (gemv_x2_grid(n) == 0 &&
            cudaMallocAsync((void**)&xf, (size_t)(n + GEMV_SMEM_PAD) * sizeof(float2), st) != cudaSuccess)
            return FL_ENOMEM;
    } else if (dtype != FL_F64 && gemv_lo_smem_grid(dtype, A_dev, n) == 0 &&
               !(dtype == FL_F32 && ((uintptr_t)A_dev & 3u) == 0 && gemv_rows_per_sm(n) > 0)) {
        if (cudaMallocAsync((void**)&xf, n * sizeof(float), st) != cudaSuccess) return FL_ENOMEM;
    }
    for (int r = 0; r < nrhs; ++r) {
        if (gemv(dtype, A_dev, lda, n, X_dev + r, ldx, Y_dev + r, ldy, xf, st) != cudaSuccess) return FL_ECUDA;
    }
    if (xf) cudaFreeAsync(xf, st);
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

int fl_tune_matvec(int dtype, const void* A_dev, int64_t lda, int64_t n, const double* x_dev, double* y_dev, int reps,
                   int* best_per_sm, double* best_ms, void* stream) {
    if (!A_dev || !x_dev || !y_dev || n < 1 || lda < n || reps < 1) return FL_EINVAL;
    if (dtype != FL_F64 && dtype != FL_F32) return FL_EINVAL;
    if (((uintptr_t)A_dev & (dtype == FL_F64 ? 7u : 3u)) != 0) return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int max_per_sm = 0;
    const bool f64 = dtype == FL_F64;
    if (!f64) {
        // float32: blocks per SM of the row-dot product
        if (gemv_rows_per_sm(n, &max_per_sm) < 1) return FL_ENOTIMPL;
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return FL_ECUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return FL_ECUDA;
        }
        int best = 0;
        double best_t = 0.0;
        int rc = FL_OK;
        for (int k = 1; k <= std::min(max_per_sm, 4) && rc == FL_OK; ++k) {
            auto launch = [&]() {
                gemv_rows_launch(k, n, (const float*)A_dev, lda, x_dev, 1, nullptr, y_dev, 1, st);
                fl::count_launch();
            };
            launch();  // warm-up
            std::vector<float> ts;
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, st);
                launch();
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = FL_ECUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ts.push_back(ms);
            }
            if (rc != FL_OK || cudaGetLastError() != cudaSuccess) {
                rc = FL_ECUDA;
                break;
            }
            std::sort(ts.begin(), ts.end());
            const double med = ts[ts.size() / 2];
            if (!best || med < best_t) {
                best = k;
                best_t = med;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != FL_OK) return rc;
        tune_record(device_name(), "gemv_rows_f32", n, 1, 1, best, 0, best_t);
        if (best_per_sm) *best_per_sm = best;
        if (best_ms) *best_ms = best_t;
        return FL_OK;
    }
    if (gemv_smem_grid<double, double>(n, 0, &max_per_sm) == 0 || max_per_sm < 2)
        return FL_ENOTIMPL;  // the staged product is not used at this size: nothing to tune
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FL_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FL_ECUDA;
    }
    const size_t smem = (size_t)(n + GEMV_SMEM_PAD) * (f64 ? sizeof(double) : sizeof(float));
    int best = 0;
    double best_t = 0.0;
    int rc = FL_OK;
    for (int k = 1; k <= max_per_sm && rc == FL_OK; ++k) {
        const unsigned grid = f64 ? gemv_smem_grid<double, double>(n, k) : gemv_smem_grid<float, float>(n, k);
        auto launch = [&]() {
            if (f64)
                gemv_smem_kernel<double, double><<<grid, 32 * GEMV_SMEM_WARPS, smem, st>>>(n, (const double*)A_dev, lda,
                                                                                          x_dev, 1, nullptr, y_dev, 1);
            else
                gemv_smem_kernel<float, float><<<grid, 32 * GEMV_SMEM_WARPS, smem, st>>>(n, (const float*)A_dev, lda,
                                                                                        x_dev, 1, nullptr, y_dev, 1);
            fl::count_launch();
        };
        launch();  // warm-up
        std::vector<float> ts;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = FL_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
        }
        if (rc != FL_OK || cudaGetLastError() != cudaSuccess) {
            rc = FL_ECUDA;
            break;
        }
        std::sort(ts.begin(), ts.end());
        const double med = ts[ts.size() / 2];
        if (!best || med < best_t) {
            best = k;
            best_t = med;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FL_OK) return rc;
    tune_record(device_name(), f64 ? GemvName<double>::name : GemvName<float>::name, n, 1, 1, best, 0, best_t);
    if (best_per_sm) *best_per_sm = best;
    if (best_ms) *best_ms = best_t;
    return FL_OK;
}

int fl_convert(const double* A_dev, int64_t lda, int64_t n, int dtype, void* A_lo_dev, int64_t ld_lo, void* stream) {
    if (!A_dev || !A_lo_dev || n < 1 || lda < n || ld_lo < n) return FL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)std::min<int64_t>(n, 65535));
    if (dtype == FL_F32X2) {
        if (((uintptr_t)A_lo_dev & 7u) != 0) return FL_EINVAL;
        convert_x2_kernel<<<grid, 256, 0, st>>>(n, A_dev, lda, (float2*)A_lo_dev, ld_lo);
        fl::count_launch();
    } else if (dtype == FL_F32) { convert_kernel<float><<<grid, 256, 0, st>>>(n, A_dev, lda, (float*)A_lo_dev, ld_lo); fl::count_launch(); }
    else if (dtype == FL_BF16) {
        convert_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(n, A_dev, lda, (__nv_bfloat16*)A_lo_dev, ld_lo);
        fl::count_launch();
    } else {
        return FL_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}

void fl_default_solve_opts(fl_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-8;
    o->maxit = 10000;
    o->inner_dtype = FL_F64;
    o->A_lo_dev = nullptr;
    o->ld_lo = 0;
    o->inner_tol = 1e-4;
    o->inner_maxit = 2000;
    o->barrier_timeout_us = 0;
}

int fl_solve(fl_handle h, int64_t n, const double* A_dev, int64_t lda, const double* b_dev, double* u_dev,
             const fl_solve_opts* o_in, fl_solve_info* info, void* stream) {
    if (!h) return FL_EINVAL;
    h->err.clear();
    if (!A_dev || !b_dev || !u_dev || n < 1 || lda < n) return set_err(h, FL_EINVAL, "bad solve arguments");
    fl_solve_opts o;
    fl_default_solve_opts(&o);
    if (o_in) o = *o_in;
    if (o.inner_dtype != FL_F64 && o.inner_dtype != FL_F32 && o.inner_dtype != FL_BF16)
        return set_err(h, FL_EINVAL, "inner_dtype");
    if (o.inner_dtype != FL_F64 && (!o.A_lo_dev || o.ld_lo < n))
        return set_err(h, FL_EINVAL, "low-precision copy missing");
    if (o.barrier_timeout_us < 0) return set_err(h, FL_EINVAL, "barrier_timeout_us");
    h->wait_ns = o.barrier_timeout_us > 0 ? 1000ull * (unsigned long long)o.barrier_timeout_us : 2000000000ull;
    cudaStream_t st = (cudaStream_t)stream;
    FL_CU(h, cudaSetDevice(h->device));
    SolveWork w;
    int r = get_work(h, n, w);
    if (r != FL_OK) return r;
    const unsigned g = (unsigned)((n + 255) / 256);
    diag_inv_kernel<<<g, 256, 0, st>>>(n, FL_F64, A_dev, lda, w.dinv); fl::count_launch();
    FL_CU(h, cudaGetLastError());
    fl_solve_info inf{};
    int status = FL_OK;
    if (o.inner_dtype == FL_F64) {
        int its = 0;
        double rel = 0;
        status = pcg(h, w, n, FL_F64, A_dev, lda, w.dinv, b_dev, u_dev, o.tol, o.maxit, &its, &rel, st);
        inf.iterations = its;
        inf.outer_iterations = 1;
    } else if (o.inner_dtype == FL_F32 && [&] {
                   diag_inv_kernel<<<g, 256, 0, st>>>(n, FL_F32, o.A_lo_dev, o.ld_lo, w.dinv_lo);
                   fl::count_launch();
                   return refine_persistent(h, w, n, A_dev, lda, (const float*)o.A_lo_dev, o.ld_lo, b_dev, u_dev,
                                            o.tol, o.inner_tol, o.maxit, o.inner_maxit, st);
               }()) {
        // the whole refinement ran in one cooperative launch; its last residual is float64 with A
        int err = 0;
        FL_CU(h, cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        FL_CU(h, cudaMemcpyAsync(&err, w.part + ERR_OFF, sizeof(int), cudaMemcpyDeviceToHost, st));
        FL_CU(h, cudaStreamSynchronize(st));
        if (err != 0) return set_err(h, FL_ETIMEOUT, "a grid barrier of the persistent refinement gave up");
        RefineOut ro;
        std::memcpy(&ro, w.s_host, sizeof(ro));
        inf.iterations = ro.inner;
        inf.outer_iterations = ro.outer;
        inf.rel_residual = (ro.bb > 0) ? std::sqrt(ro.rr / ro.bb) : 0.0;
        status = ro.status == 0 ? FL_OK : ro.status == 2 ? FL_ENOTSPD : FL_ENOTCONV;
        if (status == FL_ENOTSPD) set_err(h, FL_ENOTSPD, "CG breakdown: p^T A p <= 0");
        inf.status = status;
        if (info) *info = inf;
        return status;
    } else {
        // float64 iterative refinement around a low-precision Jacobi-PCG
        diag_inv_kernel<<<g, 256, 0, st>>>(n, o.inner_dtype, o.A_lo_dev, o.ld_lo, w.dinv_lo); fl::count_launch();
        zero_kernel<<<g, 256, 0, st>>>(n, u_dev); fl::count_launch();
        dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, b_dev, b_dev, w.ppq); fl::count_launch();
        sum_partials_kernel<<<1, 256, 0, st>>>(w.ppq, RED_BLOCKS, &w.s->bb); fl::count_launch();
        FL_CU(h, cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        FL_CU(h, cudaStreamSynchronize(st));
        const double bb = w.s_host->bb;
        int total = 0, outer = 0;
        status = FL_ENOTCONV;
        double* rvec = w.t;  // outer residual (w.r is used by the inner solver)
        while (outer < o.maxit) {
            // r = b - A u in float64
            FL_CU(h, gemv(FL_F64, A_dev, lda, n, u_dev, 1, w.q, 1, w.xf, st));
            residual_kernel<<<g, 256, 0, st>>>(n, b_dev, w.q, rvec); fl::count_launch();
            dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, rvec, rvec, w.ppq); fl::count_launch();
            sum_partials_kernel<<<1, 256, 0, st>>>(w.ppq, RED_BLOCKS, &w.s->rr); fl::count_launch();
            FL_CU(h, cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
            FL_CU(h, cudaStreamSynchronize(st));
            const double rel = (bb > 0) ? std::sqrt(w.s_host->rr / bb) : 0.0;
            if (rel <= o.tol) {
                status = FL_OK;
                break;
            }
            int its = 0;
            double irel = 0;
            // the last correction needs only a reduction by tol / rel (half of it as a margin)
            const double step_tol = std::max(o.inner_tol, 0.5 * o.tol / rel);
            int ir = pcg(h, w, n, o.inner_dtype, o.A_lo_dev, o.ld_lo, w.dinv_lo, rvec, w.d, step_tol,
                         o.inner_maxit, &its, &irel, st);
            total += its;
            if (ir == FL_ENOTSPD || ir == FL_ECUDA || ir == FL_ETIMEOUT) {
                status = ir;
                break;
            }
            axpy_kernel<<<g, 256, 0, st>>>(n, 1.0, w.d, u_dev); fl::count_launch();
            ++outer;
        }
        inf.iterations = total;
        inf.outer_iterations = outer;
    }
    // final residual in float64
    FL_CU(h, gemv(FL_F64, A_dev, lda, n, u_dev, 1, w.q, 1, w.xf, st));
    residual_kernel<<<g, 256, 0, st>>>(n, b_dev, w.q, w.t); fl::count_launch();
    dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, w.t, w.t, w.ppq); fl::count_launch();
    sum_partials_kernel<<<1, 256, 0, st>>>(w.ppq, RED_BLOCKS, &w.s->rr); fl::count_launch();
    dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, b_dev, b_dev, w.ppq); fl::count_launch();
    sum_partials_kernel<<<1, 256, 0, st>>>(w.ppq, RED_BLOCKS, &w.s->bb); fl::count_launch();
    FL_CU(h, cudaMemcpyAsync(w.s_host, w.s, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    FL_CU(h, cudaStreamSynchronize(st));
    inf.rel_residual = (w.s_host->bb > 0) ? std::sqrt(w.s_host->rr / w.s_host->bb) : 0.0;
    inf.status = status;
    if (info) *info = inf;
    return status;
}

}  // extern "C"
