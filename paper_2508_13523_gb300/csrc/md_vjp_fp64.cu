// md_vjp_fp64.cu -- FP64 instantiations of the force VJP kernel (md_vjp.cuh).
#include "md_vjp.cuh"

cudaError_t md_vjp_launch_fp64(const VjpArgs& a, bool half, bool single, int tpa,
                               unsigned blocks, cudaStream_t s) {
  return md_vjp_launch_prec<MD_PREC_FP64>(a, half, single, tpa, blocks, s);
}
