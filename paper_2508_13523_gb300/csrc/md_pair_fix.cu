// md_pair_fix.cu -- the warp-compacted FP64 pair kernel with fixed-point
// force accumulators (md_pair_q.cuh, FIX = true).
#include "md_pair.cuh"
#include "md_pair_q.cuh"

cudaError_t md_pair_q_fix_launch(const PairArgs& a, bool half, bool ev, bool single, float cut1,
                                 const float* cut_tab, unsigned blocks, cudaStream_t s,
                                 int carve, int qu) {
  return md_pair_q_launch_t<true, false>(a, half, ev, single, cut1, cut_tab, blocks, s, carve, qu);
}
