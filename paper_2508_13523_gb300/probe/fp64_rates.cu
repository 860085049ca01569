// fp64_rates.cu -- throughput of the instructions the LJ kernels lean on,
// measured on the GPU the library runs on: FP64 FMA/add/mul/compare, the
// FP32<->FP64 conversions, the FP64 and FP32 reciprocal seeds, FP32 FMA,
// and FP64 and 64-bit integer atomics to global and shared memory.  The FP64-pipe rate is the ALU roofline
// of the FP64 pair kernel.  Every loop is bounded and every index in range.
//
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 \
//                   -o /tmp/fp64_rates paper_2508_13523_gb300/probe/fp64_rates.cu
//                 /tmp/fp64_rates
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int OP>
__global__ void kern(double* out, int iters, double c, double e) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double a[8];
  float fa[8];
  unsigned long long acc = 0;
  for (int k = 0; k < 8; k++) { a[k] = 1.0 + tid * 1e-9 + k * 1e-3; fa[k] = (float)a[k]; }
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      if (OP == 0) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(c), "d"(e));
      if (OP == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(a[k]) : "d"(e));
      if (OP == 2) asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(a[k]) : "d"(c));
      if (OP == 3) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(fa[k]) : "f"((float)c), "f"((float)e));
      // inputs change every iteration through cheap integer xors so that no
      // instruction is loop invariant
      if (OP == 4) { float f; asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(a[k])); int u = __float_as_int(f); a[k] = __longlong_as_double(__double_as_longlong(a[k]) ^ (long long)(u & 7)); acc += u; }
      if (OP == 5) { double d; asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(fa[k])); long long b = __double_as_longlong(d); fa[k] = __int_as_float(__float_as_int(fa[k]) ^ (int)((b >> 29) & 7)); acc += b; }
      if (OP == 6) { double r; asm volatile("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a[k])); long long b = __double_as_longlong(r); a[k] = __longlong_as_double(__double_as_longlong(a[k]) ^ (b & 7)); acc += b; }
      if (OP == 7) { int p; asm volatile("{ .reg .pred q; setp.lt.f64 q, %1, %2; selp.s32 %0, 1, 0, q; }" : "=r"(p) : "d"(a[k]), "d"(e)); a[k] = __longlong_as_double(__double_as_longlong(a[k]) ^ (long long)(p + 1)); acc += p; }
      if (OP == 8) { float r; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fa[k])); fa[k] = __int_as_float(__float_as_int(fa[k]) ^ (__float_as_int(r) & 7)); acc += __float_as_int(r); }
      if (OP == 9) { double r; asm volatile("rcp.rn.f64 %0, %1;" : "=d"(r) : "d"(a[k])); long long b = __double_as_longlong(r); a[k] = __longlong_as_double(__double_as_longlong(a[k]) ^ (b & 7)); acc += b; }
      if (OP == 10) { long long b = __double_as_longlong(a[k]); a[k] = __longlong_as_double(b ^ ((b >> 7) & 7)); acc += b; }
    }
  }
  double s = (double)acc;
  for (int k = 0; k < 8; k++) s += a[k] + fa[k];
  out[tid] = s;
}

__global__ void atom_kern(double* arr, long long n, int iters, int spread) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int i = 0; i < iters; i++) {
    unsigned long long h = (unsigned long long)(tid * 2654435761ull + i * 40503ull);
    long long idx = spread ? (long long)(h % (unsigned long long)n) : ((tid + i * 7) % n);
    atomicAdd(&arr[idx], 1.0);
  }
}

// The same with 64-bit integer reductions (fixed-point force sums).
__global__ void atom_u64_kern(unsigned long long* arr, long long n, int iters, int spread) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int i = 0; i < iters; i++) {
    unsigned long long h = (unsigned long long)(tid * 2654435761ull + i * 40503ull);
    long long idx = spread ? (long long)(h % (unsigned long long)n) : ((tid + i * 7) % n);
    atomicAdd(&arr[idx], 1ull);
  }
}

// Shared-memory 64-bit integer atomics, 32 distinct slots per warp.
__global__ void satom_u64_kern(unsigned long long* out, int iters) {
  __shared__ unsigned long long acc[8][32 * 3];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < 96; k += 32) acc[w][k] = 0ull;
  __syncwarp();
  unsigned long long v = 1ull + lane;
  for (int i = 0; i < iters; i++) {
    const int s = (lane + i) & 31;
    atomicAdd(&acc[w][3 * s], v);
    atomicAdd(&acc[w][3 * s + 1], v);
    atomicAdd(&acc[w][3 * s + 2], v);
    v ^= 1ull;
  }
  __syncwarp();
  if (lane == 0) out[blockIdx.x * 8 + w] = acc[w][0] + acc[w][1];
}

// Shared-memory FP64 atomics: each lane adds into one of `slots` doubles of
// its warp's region (slots = 32: no two lanes collide; slots = 8: four-way).
__global__ void satom_kern(double* out, int iters, int slots) {
  __shared__ double acc[8][32 * 3];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < 96; k += 32) acc[w][k] = 0.0;
  __syncwarp();
  double v = 1.0 + lane * 1e-3;
  for (int i = 0; i < iters; i++) {
    const int s = (lane + i) % slots;
    atomicAdd(&acc[w][3 * s], v);
    atomicAdd(&acc[w][3 * s + 1], v);
    atomicAdd(&acc[w][3 * s + 2], v);
    v = __longlong_as_double(__double_as_longlong(v) ^ 1);
  }
  __syncwarp();
  if (lane == 0) out[blockIdx.x * 8 + w] = acc[w][0] + acc[w][1];
}

int main() {
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  int clk = 0, memclk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  cudaDeviceGetAttribute(&memclk, cudaDevAttrMemoryClockRate, 0);
  printf("device %s sm %d.%d SMs %d l2 %d MB smem/SM %zu smem/block optin %zu regs/SM %d clock %d kHz\n",
         p.name, p.major, p.minor, p.multiProcessorCount, p.l2CacheSize >> 20,
         p.sharedMemPerMultiprocessor, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor, clk);
  const int blocks = p.multiProcessorCount * 8, threads = 256, iters = 4096;
  double* out;
  CK(cudaMalloc(&out, sizeof(double) * blocks * threads));
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0); cudaEventCreate(&t1);
  const char* names[] = {"dfma", "dadd", "dmul", "ffma", "cvt.f32.f64", "cvt.f64.f32", "rcp.approx.f64", "setp.f64", "rcp.approx.f32", "rcp.rn.f64", "int-xor-only"};
  void (*ks[])(double*, int, double, double) = {kern<0>, kern<1>, kern<2>, kern<3>, kern<4>, kern<5>, kern<6>, kern<7>, kern<8>, kern<9>, kern<10>};
  for (int op = 0; op < 11; op++) {
    int it = (op == 3 || op == 8) ? iters * 8 : iters;
    ks[op]<<<blocks, threads>>>(out, 16, 0.999999, 1e-7);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(t0);
    ks[op]<<<blocks, threads>>>(out, it, 0.999999, 1e-7);
    cudaEventRecord(t1);
    CK(cudaEventSynchronize(t1));
    float ms; cudaEventElapsedTime(&ms, t0, t1);
    double ops = (double)blocks * threads * it * 8;
    printf("%-16s %10.3f Gop/s  (%.3f ms)  %.2f op/clk/SM at %d MHz\n", names[op], ops / ms / 1e6, ms,
           ops / (ms * 1e-3) / p.multiProcessorCount / (clk * 1e3), clk / 1000);
  }
  // FP64 atomics
  long long n = 8ll << 20;  // 64 MB of doubles
  double* arr;
  CK(cudaMalloc(&arr, sizeof(double) * n));
  CK(cudaMemset(arr, 0, sizeof(double) * n));
  for (int spread = 0; spread < 2; spread++) {
    int ab = p.multiProcessorCount * 16, at = 256, ai = 256;
    atom_kern<<<ab, at>>>(arr, n, 4, spread);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(t0);
    atom_kern<<<ab, at>>>(arr, n, ai, spread);
    cudaEventRecord(t1);
    CK(cudaEventSynchronize(t1));
    float ms; cudaEventElapsedTime(&ms, t0, t1);
    double ops = (double)ab * at * ai;
    printf("atomicAdd f64 %s %10.3f Gatom/s (%.3f ms)\n", spread ? "hashed " : "strided", ops / ms / 1e6, ms);
  }
  for (int slots = 32; slots >= 8; slots /= 4) {
    int sb = p.multiProcessorCount * 8, st = 256, si = 2048;
    satom_kern<<<sb, st>>>(out, 8, slots);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(t0);
    satom_kern<<<sb, st>>>(out, si, slots);
    cudaEventRecord(t1);
    CK(cudaEventSynchronize(t1));
    float ms; cudaEventElapsedTime(&ms, t0, t1);
    double ops = (double)sb * st * si * 3;
    printf("atomicAdd f64 shared, %2d slots/warp %10.3f Gatom/s (%.3f ms)  %.2f /clk/SM\n", slots,
           ops / ms / 1e6, ms, ops / (ms * 1e-3) / p.multiProcessorCount / (clk * 1e3));
  }
  unsigned long long* arr64 = (unsigned long long*)arr;
  for (int spread = 0; spread < 2; spread++) {
    int ab = p.multiProcessorCount * 16, at = 256, ai = 256;
    atom_u64_kern<<<ab, at>>>(arr64, n, 4, spread);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(t0);
    atom_u64_kern<<<ab, at>>>(arr64, n, ai, spread);
    cudaEventRecord(t1);
    CK(cudaEventSynchronize(t1));
    float ms; cudaEventElapsedTime(&ms, t0, t1);
    double ops = (double)ab * at * ai;
    printf("atomicAdd u64 %s %10.3f Gatom/s (%.3f ms)\n", spread ? "hashed " : "strided", ops / ms / 1e6, ms);
  }
  {
    int sb = p.multiProcessorCount * 8, st = 256, si = 2048;
    satom_u64_kern<<<sb, st>>>((unsigned long long*)out, 8);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(t0);
    satom_u64_kern<<<sb, st>>>((unsigned long long*)out, si);
    cudaEventRecord(t1);
    CK(cudaEventSynchronize(t1));
    float ms; cudaEventElapsedTime(&ms, t0, t1);
    double ops = (double)sb * st * si * 3;
    printf("atomicAdd u64 shared, 32 slots/warp %10.3f Gatom/s (%.3f ms)  %.2f /clk/SM\n",
           ops / ms / 1e6, ms, ops / (ms * 1e-3) / p.multiProcessorCount / (clk * 1e3));
  }
  CK(cudaFree(arr));
  CK(cudaFree(out));
  return 0;
}
