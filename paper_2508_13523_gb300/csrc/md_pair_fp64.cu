// md_pair_fp64.cu -- FP64 instantiations of the pair kernel (md_pair.cuh).
#include "md_pair.cuh"
#include "md_pair_q.cuh"

cudaError_t md_pair_launch_fp64(const PairArgs& a, bool half, bool ev, bool single, int tpa,
                                unsigned blocks, cudaStream_t s, int carve) {
  return md_pair_launch_prec<MD_PREC_FP64>(a, half, ev, single, tpa, blocks, s, carve);
}

cudaError_t md_pair_q_launch(const PairArgs& a, bool half, bool ev, bool single, float cut1,
                             const float* cut_tab, unsigned blocks, cudaStream_t s, int carve) {
  return md_pair_q_launch_t<false, false>(a, half, ev, single, cut1, cut_tab, blocks, s, carve);
}
