// md_pair_coul.cu -- the second pair style, lj/cut/coul/cut (Eq. 1 plus a
// cut Coulomb term with per-type charges; the paper's pair styles share one
// two-body base, Sec. 4): the warp-compacted FP64 kernel with either force
// summation, and the mixed-precision per-atom kernel at 1, 2 or 4 threads
// per atom.
#include "md_pair.cuh"
#include "md_pair_q.cuh"

cudaError_t md_pair_q_coul_launch(const PairArgs& a, bool fix, bool half, bool ev, bool single,
                                  float cut1, const float* cut_tab, unsigned blocks,
                                  cudaStream_t s, int carve) {
  return fix ? md_pair_q_launch_t<true, true>(a, half, ev, single, cut1, cut_tab, blocks, s, carve)
             : md_pair_q_launch_t<false, true>(a, half, ev, single, cut1, cut_tab, blocks, s,
                                               carve);
}

template <bool HALF, bool EV, bool SINGLE>
static cudaError_t coul_tpa(const PairArgs& a, int tpa, unsigned blocks, cudaStream_t s,
                            int carve) {
  switch (tpa) {
    case 1:
      return md_launch_carved(k_pair<MD_PREC_MIXED, HALF, 1, EV, SINGLE, true>, a, blocks, s,
                              carve);
    case 2:
      return md_launch_carved(k_pair<MD_PREC_MIXED, HALF, 2, EV, SINGLE, true>, a, blocks, s,
                              carve);
    case 4:
      return md_launch_carved(k_pair<MD_PREC_MIXED, HALF, 4, EV, SINGLE, true>, a, blocks, s,
                              carve);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t md_pair_launch_mixed_coul(const PairArgs& a, bool half, bool ev, bool single,
                                      int tpa, unsigned blocks, cudaStream_t s, int carve) {
  if (half) {
    if (ev) return single ? coul_tpa<true, true, true>(a, tpa, blocks, s, carve)
                          : coul_tpa<true, true, false>(a, tpa, blocks, s, carve);
    return single ? coul_tpa<true, false, true>(a, tpa, blocks, s, carve)
                  : coul_tpa<true, false, false>(a, tpa, blocks, s, carve);
  }
  if (ev) return single ? coul_tpa<false, true, true>(a, tpa, blocks, s, carve)
                        : coul_tpa<false, true, false>(a, tpa, blocks, s, carve);
  return single ? coul_tpa<false, false, true>(a, tpa, blocks, s, carve)
                : coul_tpa<false, false, false>(a, tpa, blocks, s, carve);
}
