// md_step_fused.cu -- one launch per velocity-Verlet step: the integrator's
// kick-drift (K1 or K21) of every atom, a grid-wide barrier, then the pair
// forces of every tile at the new positions (the compacted FP64 kernel with
// fixed-point sums, persistent tile scheduling).  For a batch of replicas
// the launch covers all of them: uneven boxes share one grid.
//
// The launch is cooperative (all blocks resident at once), so the barrier
// between the two phases cannot wait on a block that is not running.  The
// barrier's wait is bounded all the same: after ~2 s it sets an error word
// (read by the host at the next rebuild, MD_ETIMEOUT) and the block returns.
//
// Visibility: phase 1 writes each atom's records (x4, xs, xq, v, f, fix)
// from the one thread that owns the atom and reads no other atom's, so no
// SM holds a stale cached copy of another atom's record when phase 2 reads
// them; the writes are fenced before the barrier.
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_device.cuh"
#include "md_integrate.cuh"
#include "md_internal.cuh"
#include "md_pair.cuh"
#include "md_pair_q.cuh"

namespace {

// Grid-wide barrier over `expect` blocks: bar[0] arrivals, bar[1]
// generation, *err set on timeout.  All threads of every block must call
// it; returns false (in every thread of the block) if this block gave up
// waiting after limit_ns.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int* err,
                                             unsigned int expect,
                                             unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int gen = atomicAdd(bar + 1, 0u);
    __threadfence();
    if (atomicAdd(bar, 1u) == expect - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long t0, t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (*(volatile unsigned int*)(bar + 1) == gen) {
        __nanosleep(64);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
          atomicExch(err, 1u);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

constexpr unsigned long long BARRIER_LIMIT_NS = 2000000000ULL;  // 2 s

// The barrier alone, for its test: a cooperative grid whose barrier waits
// for one block more than it has, so that every block's wait runs out
// (nothing faults, nothing is left waiting).  err[0] ends at 1.
__global__ void __launch_bounds__(32) k_barrier_probe(unsigned int* bar, unsigned int* err,
                                                     unsigned int missing,
                                                     unsigned long long limit_ns) {
  grid_barrier(bar, err, gridDim.x + missing, limit_ns);
}

// Phase 1 of k_step_fused, out of line so that its registers do not add to
// the pair phase's: kick and drift of every atom (grid-stride), the largest
// displacement into dmax.
template <int MODE>
__device__ __noinline__ void integrate_all(const IntArgs& ia) {
  float d2 = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < ia.n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    if (i < ia.n) d2 = fmaxf(d2, md_integrate_atom<MODE>(ia, i));
  }
  md_disp_max(d2, ia.dmax);
}

template <int MODE, bool HALF, bool SINGLE>
__global__ void __launch_bounds__(MD_BLOCK, md_pair_q_minb(true, false, true, false, 1))
    k_step_fused(const IntArgs ia, const PairArgs a, const float cut_hi1,
                 const float* __restrict__ cut_hi_tab, unsigned int* bar, unsigned int* err) {
  integrate_all<MODE>(ia);
  if (blockIdx.x == 0)  // the pair phase's tile counters start at zero
    for (int k = threadIdx.x; k < a.nslots; k += blockDim.x) a.tile_ctr[k] = 0;
  __threadfence();
  if (!grid_barrier(bar, err, gridDim.x, BARRIER_LIMIT_NS)) return;
  // phase 2: the forces at the new positions
  md_pair_q_tiles<HALF, false, SINGLE, true, false, 1>(a, cut_hi1, cut_hi_tab);
}

template <int MODE, bool HALF, bool SINGLE>
cudaError_t launch_fused(const IntArgs& ia, const PairArgs& a, float cut1, const float* cut_tab,
                         unsigned int* bar, unsigned int* err, cudaStream_t s) {
  auto kern = k_step_fused<MODE, HALF, SINGLE>;
  int occ = 1;
  cudaError_t e = md_prepare_kernel((const void*)kern, -1, &occ);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nslots * occ));
  cfg.blockDim = dim3(MD_BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, ia, a, cut1, cut_tab, bar, err);
}

}  // namespace

cudaError_t md_step_fused_launch(const IntArgs& ia, const PairArgs& a, int mode, bool half,
                                 bool single, float cut1, const float* cut_tab,
                                 unsigned int* bar, unsigned int* err, cudaStream_t s) {
  if (!a.tile_ctr) return cudaErrorInvalidValue;
  if (mode == MD_K1) {
    if (half)
      return single ? launch_fused<MD_K1, true, true>(ia, a, cut1, cut_tab, bar, err, s)
                    : launch_fused<MD_K1, true, false>(ia, a, cut1, cut_tab, bar, err, s);
    return single ? launch_fused<MD_K1, false, true>(ia, a, cut1, cut_tab, bar, err, s)
                  : launch_fused<MD_K1, false, false>(ia, a, cut1, cut_tab, bar, err, s);
  }
  if (mode != MD_K21) return cudaErrorInvalidValue;
  if (half)
    return single ? launch_fused<MD_K21, true, true>(ia, a, cut1, cut_tab, bar, err, s)
                  : launch_fused<MD_K21, true, false>(ia, a, cut1, cut_tab, bar, err, s);
  return single ? launch_fused<MD_K21, false, true>(ia, a, cut1, cut_tab, bar, err, s)
                : launch_fused<MD_K21, false, false>(ia, a, cut1, cut_tab, bar, err, s);
}

// Diagnostic: the fused step's grid barrier on its own, in a cooperative
// launch of `blocks` blocks waiting for blocks + missing arrivals, with a
// wait limit of limit_ms.  word: device, 3 unsigned ints (zeroed here).
// Returns MD_ETIMEOUT when the barrier reported a timeout, MD_OK when it
// completed.  Synchronizes the stream.
extern "C" int md_eval_barrier(int32_t blocks, int32_t missing, double limit_ms,
                               unsigned int* word, void* stream) {
  if (blocks < 1 || blocks > 1024 || missing < 0 || missing > 1 || !word ||
      !(limit_ms > 0.0) || limit_ms > 10000.0)
    return MD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  MD_CUDA(cudaMemsetAsync(word, 0, 3 * sizeof(unsigned int), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MD_CUDA(cudaLaunchKernelEx(&cfg, k_barrier_probe, word, word + 2, (unsigned int)missing,
                             (unsigned long long)(limit_ms * 1e6)));
  unsigned int err = 0;
  MD_CUDA(cudaMemcpyAsync(&err, word + 2, sizeof(err), cudaMemcpyDeviceToHost, s));
  MD_CUDA(cudaStreamSynchronize(s));
  return err ? MD_ETIMEOUT : MD_OK;
}

