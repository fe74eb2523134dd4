// Allocation-free float32 matrix-vector product.
//
// fl_matvec with FL_F32 stages a float32 copy of x in device memory that it
// allocates on every call.  Some callers cannot allocate device memory: code that
// runs under a caller-owned memory budget or inside another allocator's arena,
// real-time loops that must not enter the driver's allocator, and host code that
// has no CUDA context of its own to allocate from (it only receives device
// pointers).  fl_matvec_f32_static gives them the same product with the staging
// copy held in a fixed file-scope device array instead.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/fraclap.h"

namespace fl {
void count_launch(int n);
}

namespace {

// Staging copy of x (float32).  Every GPU that loads the library holds these
// FL_STATIC_MAX_N * 4 bytes until the process exits.
static __device__ __align__(256) float g_xf_static[FL_STATIC_MAX_N];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
float* g_xf_ptr[kMaxDevices] = {};  // device address of g_xf_static per device, set once (not valid
                                    // after a reset of that device's primary context)

// In host code g_xf_static names a host-side stand-in, not device memory, so the
// device address is looked up once per device with that device current.
int static_scratch(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FL_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_xf_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_xf_static) != cudaSuccess || !p) return FL_ECUDA;
        g_xf_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_xf_ptr[dev];
    return FL_OK;
}

__global__ void xf_from_f64(int64_t n, const double* __restrict__ x, float* __restrict__ xf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) xf[i] = (float)x[i];
}

// one warp per row; float32 lane sums, float64 row total
__global__ void gemv_f32_static(int64_t n, const float* __restrict__ A, int64_t lda, const float* __restrict__ xf,
                                double* __restrict__ y, int vec) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float* a = A + row * lda;
    float acc0 = 0.f, acc1 = 0.f;
    int64_t j0 = 0;
    if (vec) {
        const int64_t nv = (n / 128) * 128;
        const float4* a4 = reinterpret_cast<const float4*>(a);
        const float4* x4 = reinterpret_cast<const float4*>(xf);
#pragma unroll 4
        for (int64_t j = lane; j < nv / 4; j += 32) {
            const float4 av = __ldcs(a4 + j);
            const float4 xv = x4[j];
            acc0 = fmaf(av.x, xv.x, acc0);
            acc1 = fmaf(av.y, xv.y, acc1);
            acc0 = fmaf(av.z, xv.z, acc0);
            acc1 = fmaf(av.w, xv.w, acc1);
        }
        j0 = nv;
    }
    for (int64_t j = j0 + lane; j < n; j += 32) acc0 = fmaf(a[j], xf[j], acc0);
    double t = (double)acc0 + (double)acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) y[row] = t;
}

}  // namespace

extern "C" int fl_matvec_f32_static(const float* A_dev, int64_t lda, int64_t n, const double* x_dev, double* y_dev,
                                    void* stream) {
    if (n < 1 || n > FL_STATIC_MAX_N) return FL_EINVAL;
    if (!A_dev || !x_dev || !y_dev || lda < n) return FL_EINVAL;
    // an error left pending by earlier work is reported, not cleared (and not blamed on a
    // launch of this call): the caller still sees it where it came from
    if (cudaPeekAtLastError() != cudaSuccess) return FL_ECUDA;
    float* xf = nullptr;
    const int r = static_scratch(&xf);
    if (r != FL_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    // the n staged entries are rewritten before they are read, so nothing needs clearing
    xf_from_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x_dev, xf);
    fl::count_launch(1);
    if (cudaGetLastError() != cudaSuccess) return FL_ECUDA;
    const int vec = (((uintptr_t)A_dev & 15u) == 0) && (lda % 4 == 0);
    gemv_f32_static<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(n, A_dev, lda, xf, y_dev, vec);
    fl::count_launch(1);
    return cudaGetLastError() == cudaSuccess ? FL_OK : FL_ECUDA;
}
