// Unit-rate probes for the roofline of the assembly kernels: results per clock per
// SM of FFMA, paired FFMA (.f32x2), DFMA, the MUFU functions (rsqrt, sqrt, ex2, lg2)
// and two float64 library functions.  Each thread runs 8 independent chains.
#include <cstdio>
#include <cuda_runtime.h>
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d; asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c)); return d; }
template <int OP>
__global__ void k(float* out, double* outd, int iters, long long* cyc) {
  float x[8]; double y[8]; unsigned long long z[8];
  for (int i = 0; i < 8; ++i) { x[i] = 1.0f + 1e-3f * (threadIdx.x + i); y[i] = 1.0 + 1e-3 * (threadIdx.x + i); z[i] = 0x3f8000003f800000ull + i; }
  const unsigned long long za = 0x3f7ff7cf3f7ff7cfull, zb = 0x38d1b71738d1b717ull;
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (OP == 0) x[i] = fmaf(x[i], 0.9999f, 0.0001f);
      if (OP == 1) y[i] = fma(y[i], 0.9999, 0.0001);
      if (OP == 2) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
      if (OP == 3) asm volatile("sqrt.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
      if (OP == 4) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
      if (OP == 5) asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
      if (OP == 6) y[i] = rsqrt(y[i]);
      if (OP == 7) y[i] = pow(y[i], -1.75);
      if (OP == 8) z[i] = f2fma(z[i], za, zb);
    }
  }
  long long t1 = clock64();
  float s = 0; double sd = 0;
  for (int i = 0; i < 8; ++i) { s += x[i]; sd += y[i]; s += (float)(z[i] & 1); }
  if (s == 12345.f) out[0] = s;
  if (sd == 12345.) outd[0] = sd;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  float* o; double* od; long long* cyc; cudaMalloc(&o, 4); cudaMalloc(&od, 8); cudaMalloc(&cyc, 8 * 4096);
  const char* names[] = {"ffma", "dfma", "mufu.rsqrt", "mufu.sqrt", "mufu.ex2", "mufu.lg2", "rsqrt(double)", "pow(double,-1.75)", "ffma.f32x2 (pairs)"};
  for (int op = 0; op < 9; ++op) {
    int iters = (op == 7) ? 200 : (op == 1 || op == 6 ? 2000 : 20000);
    int blocks = sms, threads = 1024;
    cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(a);
      switch (op) {
        case 0: k<0><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 1: k<1><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 2: k<2><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 3: k<3><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 4: k<4><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 5: k<5><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 6: k<6><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 7: k<7><<<blocks, threads>>>(o, od, iters, cyc); break;
        case 8: k<8><<<blocks, threads>>>(o, od, iters, cyc); break;
      }
      cudaEventRecord(b); cudaEventSynchronize(b);
    }
    float ms; cudaEventElapsedTime(&ms, a, b);
    long long c[4096]; cudaMemcpy(c, cyc, 8 * blocks, cudaMemcpyDeviceToHost);
    long long cmax = 0; for (int i = 0; i < blocks; ++i) cmax = c[i] > cmax ? c[i] : cmax;
    double ops = (double)blocks * threads * iters * 8;
    printf("%-20s %8.3f ms  %10.3f Gop/s  %7.2f op/clk/SM (clk from clock64, 1 block/SM)  err=%s\n", names[op], ms,
           ops / ms / 1e6, ops / sms / (double)cmax, cudaGetErrorString(cudaGetLastError()));
  }
  return 0;
}
