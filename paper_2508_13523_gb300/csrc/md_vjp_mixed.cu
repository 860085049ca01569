// md_vjp_mixed.cu -- mixed-precision instantiations of the force VJP kernel
// (md_vjp.cuh).
#include "md_vjp.cuh"

cudaError_t md_vjp_launch_mixed(const VjpArgs& a, bool half, bool single, int tpa,
                                unsigned blocks, cudaStream_t s) {
  return md_vjp_launch_prec<MD_PREC_MIXED>(a, half, single, tpa, blocks, s);
}
