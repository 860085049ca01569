// md_selftest.cu -- md_eval_recip: the device reciprocal and reciprocal
// square root of the pair kernels (md_rcp, md_rsqrt in md_device.cuh),
// evaluated elementwise so that tests can bound their error directly.
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_device.cuh"
#include "md_internal.cuh"

namespace {

__global__ void __launch_bounds__(MD_BLOCK)
    k_eval_recip(const double* __restrict__ a, int64_t n, double* __restrict__ rcp,
                 double* __restrict__ rsqrt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = a[i];
  if (rcp) rcp[i] = md_rcp(x);
  if (rsqrt) rsqrt[i] = md_rsqrt(x);
}

}  // namespace

extern "C" int md_eval_recip(int64_t n, const double* a, double* rcp, double* rsqrt,
                             void* stream) {
  if (n < 0 || (n > 0 && !a)) return MD_EINVAL;
  if (n == 0 || (!rcp && !rsqrt)) return MD_OK;
  const int64_t blocks = md_blocks(n);
  if (blocks > 0x7fffffffLL) return MD_EINVAL;
  k_eval_recip<<<(unsigned)blocks, MD_BLOCK, 0, (cudaStream_t)stream>>>(a, n, rcp, rsqrt);
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}
