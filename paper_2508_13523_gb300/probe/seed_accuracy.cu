// seed_accuracy.cu -- relative error of the hardware reciprocal and
// reciprocal-square-root seeds the FP64 pair kernels refine
// (rcp.approx.ftz.f64 in md_rcp, rsqrt.approx.ftz.f64 in md_rsqrt), over
// r^2 in [0.25, 16) (LJ and Coulomb pair distances), against the correctly
// rounded __drcp_rn and 1 / __dsqrt_rn.  The number of correct bits sets
// how many series rounds md_rcp and md_rsqrt need.  Every index in range.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/seed_accuracy \
//       paper_2508_13523_gb300/probe/seed_accuracy.cu && /tmp/seed_accuracy
#include <cmath>
#include <cstdio>
#include <cuda_runtime.h>

__global__ void k(double* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double er = 0.0, es = 0.0, e1 = 0.0;
  for (long long k = i; k < n; k += (long long)gridDim.x * blockDim.x) {
    const double a = 0.25 + 15.75 * ((double)k / (double)n);
    double y, z;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(z) : "d"(a));
    er = fmax(er, fabs(y * a - 1.0));
    const double rs = 1.0 / __dsqrt_rn(a);
    es = fmax(es, fabs(z / rs - 1.0));
    // one series round of md_rsqrt
    const double e = __fma_rn(-a, z * z, 1.0);
    const double z1 = __fma_rn(z * e, __fma_rn(0.375, e, 0.5), z);
    e1 = fmax(e1, fabs(z1 / rs - 1.0));
  }
  out[3 * i] = er;
  out[3 * i + 1] = es;
  out[3 * i + 2] = e1;
}

int main() {
  const int blocks = 152 * 4, threads = 256;
  const long long n = 1LL << 26;
  double* d;
  if (cudaMalloc(&d, sizeof(double) * 3 * blocks * threads) != cudaSuccess) return 1;
  k<<<blocks, threads>>>(d, n);
  static double h[3 * 152 * 4 * 256];
  if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  double m[3] = {0, 0, 0};
  for (int i = 0; i < blocks * threads; i++)
    for (int c = 0; c < 3; c++) m[c] = fmax(m[c], h[3 * i + c]);
  printf("rcp.approx.ftz.f64   max rel err %.3e (%.1f bits)\n", m[0], -log2(m[0]));
  printf("rsqrt.approx.ftz.f64 max rel err %.3e (%.1f bits)\n", m[1], -log2(m[1]));
  printf("rsqrt + one series round         %.3e (%.1f bits)\n", m[2], -log2(m[2] > 0 ? m[2] : 1e-300));
  cudaFree(d);
  return 0;
}
