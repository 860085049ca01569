// md_pair_fp64.cu -- FP64 instantiations of the pair kernel (md_pair.cuh).
#include "md_pair.cuh"
#include "md_pair_q.cuh"

cudaError_t md_pair_launch_fp64(const PairArgs& a, bool half, bool ev, bool single, int tpa,
                                unsigned blocks, cudaStream_t s, int carve) {
  return md_pair_launch_prec<MD_PREC_FP64>(a, half, ev, single, tpa, blocks, s, carve);
}

cudaError_t md_pair_q_launch(const PairArgs& a, bool half, bool ev, bool single, float cut1,
                             const float* cut_tab, unsigned blocks, cudaStream_t s, int carve) {
  if (half) {
    if (ev) return single ? md_pair_q_launch3<true, true, true>(a, cut1, cut_tab, blocks, s, carve)
                          : md_pair_q_launch3<true, true, false>(a, cut1, cut_tab, blocks, s, carve);
    return single ? md_pair_q_launch3<true, false, true>(a, cut1, cut_tab, blocks, s, carve)
                  : md_pair_q_launch3<true, false, false>(a, cut1, cut_tab, blocks, s, carve);
  }
  if (ev) return single ? md_pair_q_launch3<false, true, true>(a, cut1, cut_tab, blocks, s, carve)
                        : md_pair_q_launch3<false, true, false>(a, cut1, cut_tab, blocks, s, carve);
  return single ? md_pair_q_launch3<false, false, true>(a, cut1, cut_tab, blocks, s, carve)
                : md_pair_q_launch3<false, false, false>(a, cut1, cut_tab, blocks, s, carve);
}
