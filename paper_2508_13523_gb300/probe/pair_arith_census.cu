// pair_arith_census.cu -- which FP64 instructions the exact pair arithmetic
// issues on the GPU, counted with ncu's per-opcode counters
// (smsp__sass_thread_inst_executed_op_{dadd,dfma,dmul}_pred_on.sum), and its
// throughput.  Four variants of the same pair loop (positions gathered from a
// 128 KB table, accumulation by integer xor so that only the pair arithmetic
// uses the FP64 pipe):
//   0  minimum image guarded by "any component beyond L/2", then per component
//   1  no minimum image
//   2  as 0 with the correction written as an unconditional subtraction
//   3  as 1 with every multiply and add written as an FMA
// Each runs in a box of L = 16 (half the components wrap) and L = 1e6
// (nothing wraps).  Every index is taken modulo the table size.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/pair_arith_census \
//       paper_2508_13523_gb300/probe/pair_arith_census.cu
//   ncu --clock-control none --metrics smsp__sass_thread_inst_executed_op_dadd_pred_on.sum,\
//       smsp__sass_thread_inst_executed_op_dfma_pred_on.sum,\
//       smsp__sass_thread_inst_executed_op_dmul_pred_on.sum,\
//       sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active,gpu__time_duration.sum \
//       --csv /tmp/pair_arith_census
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__device__ __forceinline__ bool abs_gt(double d, long long h) {
  return (__double_as_longlong(d) & 0x7fffffffffffffffLL) > h;
}
__device__ __forceinline__ double min_image(double d, double L, long long h) {
  if (abs_gt(d, h)) d = __dsub_rn(d, copysign(L, d));
  return d;
}
__device__ __forceinline__ double rcp(double a) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  const double e = __fma_rn(-a, y, 1.0);
  return __fma_rn(y, __fma_rn(e, e, e), y);
}
__device__ __forceinline__ double pmul(double a, double b) {  // a*b as an FMA
  double r;
  asm("fma.rn.f64 %0, %1, %2, 0d8000000000000000;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ double psub(double a, double b) {  // a-b as an FMA
  double r;
  asm("fma.rn.f64 %0, %1, 0dBFF0000000000000, %2;" : "=d"(r) : "d"(b), "d"(a));
  return r;
}

// VAR 0: as in the kernel (branch on any component, then min_image each)
// VAR 1: no min image
// VAR 2: min image as branch on any + unconditional correction inside
// VAR 3: VAR 1 with DMUL/DADD written as FMAs
template <int VAR>
__global__ void k(const double4_32a* __restrict__ xs, int nx, int iters, double L, long long hb,
                  double lj1, double lj2, double cut, double* out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const double4_32a xi = xs[tid % nx];
  double fx = 0, fy = 0, fz = 0;
  unsigned j = tid * 2654435761u;
  for (int it = 0; it < iters; it++) {
    j = j * 1664525u + 1013904223u;
    const double4_32a xj = xs[(j >> 8) % nx];
    double dx, dy, dz;
    if (VAR == 3) { dx = psub(xj.x, xi.x); dy = psub(xj.y, xi.y); dz = psub(xj.z, xi.z); }
    else { dx = __dsub_rn(xj.x, xi.x); dy = __dsub_rn(xj.y, xi.y); dz = __dsub_rn(xj.z, xi.z); }
    if (VAR == 0) {
      if (abs_gt(dx, hb) | abs_gt(dy, hb) | abs_gt(dz, hb)) {
        dx = min_image(dx, L, hb); dy = min_image(dy, L, hb); dz = min_image(dz, L, hb);
      }
    } else if (VAR == 2) {
      if (abs_gt(dx, hb) | abs_gt(dy, hb) | abs_gt(dz, hb)) {
        dx = __dsub_rn(dx, abs_gt(dx, hb) ? copysign(L, dx) : 0.0);
        dy = __dsub_rn(dy, abs_gt(dy, hb) ? copysign(L, dy) : 0.0);
        dz = __dsub_rn(dz, abs_gt(dz, hb) ? copysign(L, dz) : 0.0);
      }
    }
    double r2 = VAR == 3 ? __fma_rn(dz, dz, __fma_rn(dy, dy, pmul(dx, dx)))
                         : __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    if (r2 < cut) {
      const double r2inv = rcp(r2);
      double r6, fp, gx, gy, gz;
      if (VAR == 3) {
        r6 = pmul(pmul(r2inv, r2inv), r2inv);
        fp = pmul(pmul(r6, __fma_rn(lj1, r6, -lj2)), r2inv);
        gx = pmul(fp, dx); gy = pmul(fp, dy); gz = pmul(fp, dz);
      } else {
        r6 = r2inv * r2inv * r2inv;
        fp = r6 * (lj1 * r6 - lj2) * r2inv;
        gx = fp * dx; gy = fp * dy; gz = fp * dz;
      }
      // integer accumulation stand-in (keeps the FP64 op count honest)
      fx = __longlong_as_double(__double_as_longlong(fx) ^ __double_as_longlong(gx));
      fy = __longlong_as_double(__double_as_longlong(fy) ^ __double_as_longlong(gy));
      fz = __longlong_as_double(__double_as_longlong(fz) ^ __double_as_longlong(gz));
    }
  }
  out[tid] = __longlong_as_double(__double_as_longlong(fx) ^ __double_as_longlong(fy) ^
                                  __double_as_longlong(fz));
}

int main() {
  const int nx = 4096, blocks = 152 * 8, threads = 256, iters = 512;
  double4_32a* xs; double* out;
  CK(cudaMalloc(&xs, sizeof(double4_32a) * nx));
  CK(cudaMalloc(&out, sizeof(double) * blocks * threads));
  static double4_32a h[4096];
  const double L = 16.0;  // positions in [0, 16)
  for (int i = 0; i < nx; i++) {  // positions in [0, L): pairs at distance up to ~L
    unsigned a = i * 2654435761u, b = a * 1664525u + 1013904223u, c = b * 1664525u + 1013904223u;
    h[i].x = L * (a >> 8) / 16777216.0;
    h[i].y = L * (b >> 8) / 16777216.0;
    h[i].z = L * (c >> 8) / 16777216.0;
    h[i].w = 0.0;
  }
  CK(cudaMemcpy(xs, h, sizeof(h), cudaMemcpyHostToDevice));
  for (int pass = 0; pass < 2; pass++) {
  const double Lb = pass ? 1e6 : L;  // pass 1: a box so large that nothing wraps
  double halfL = Lb / 2; long long hb; memcpy(&hb, &halfL, 8);
  // cut = 64: r < 8, with |d| < 8 after min image about half the pairs are inside
  void (*ks[])(const double4_32a*, int, int, double, long long, double, double, double, double*) = {k<0>, k<1>, k<2>, k<3>};
  cudaEvent_t t0, t1; cudaEventCreate(&t0); cudaEventCreate(&t1);
  for (int v = 0; v < 4; v++) {
    ks[v]<<<blocks, threads>>>(xs, nx, 8, Lb, hb, 4.0, 2.0, 64.0, out);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(t0);
    ks[v]<<<blocks, threads>>>(xs, nx, iters, Lb, hb, 4.0, 2.0, 64.0, out);
    cudaEventRecord(t1);
    CK(cudaEventSynchronize(t1));
    float ms; cudaEventElapsedTime(&ms, t0, t1);
    printf("L %g variant %d: %.3f ms, %.2f Gpair/s\n", Lb, v, ms, (double)blocks * threads * iters / ms / 1e6);
  }
  }
  return 0;
}
