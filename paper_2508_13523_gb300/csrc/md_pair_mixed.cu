// md_pair_mixed.cu -- mixed-precision instantiations of the pair kernel
// (md_pair.cuh).
#include "md_pair.cuh"

cudaError_t md_pair_launch_mixed(const PairArgs& a, bool half, bool ev, bool single, int tpa,
                                 unsigned blocks, cudaStream_t s, int carve) {
  return md_pair_launch_prec<MD_PREC_MIXED>(a, half, ev, single, tpa, blocks, s, carve);
}
