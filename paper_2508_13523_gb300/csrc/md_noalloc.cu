// md_noalloc.cu -- kinetic energy and temperature of caller-held velocities
// with no device allocation (md_kinetic_noalloc in include/md.h).
//
// Who needs it: code that cannot call cudaMalloc at the moment it wants a
// reduction -- a real-time loop that must never enter the allocator
// (cudaMalloc can synchronize the device and stall), or a framework whose
// caching allocator owns all device memory and hands none to libraries.
// Such callers cannot create an md_ctx (which allocates its buffers) but can
// still sum the kinetic energy of velocities they hold.
//
// How: the per-block partial sums that md_energy keeps in context-owned
// memory live here in one file-scope device array of fixed size.  Every GPU
// that loads libmd.so holds that array until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// shadow variable), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and keeps it (per
// CUDA context, see below).
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ATOMS_PER_THREAD = 4;
constexpr int NA_ATOMS_PER_BLOCK = NA_THREADS * NA_ATOMS_PER_THREAD;  // 1024
constexpr int NA_MAX_BLOCKS = MD_NOALLOC_MAX_ATOMS / NA_ATOMS_PER_BLOCK;  // 4096
constexpr int NA_MAX_DEVICES = 64;

static_assert(MD_NOALLOC_MAX_ATOMS % NA_ATOMS_PER_BLOCK == 0, "whole blocks");

// One partial sum per block; 4096 doubles = 32 KB per device.
__device__ __align__(256) double g_ke_partials[NA_MAX_BLOCKS];

struct MassTable {
  double m[MD_MAX_TYPES];
};

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[NA_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NA_THREADS / 32; w++) s += red[w];
  return s;
}

// Block b sums 0.5 m v^2 over atoms [b*1024, (b+1)*1024) into partials[b].
__global__ void __launch_bounds__(NA_THREADS)
    k_ke_partials(const double* __restrict__ v, const int32_t* __restrict__ type, int64_t n,
                  MassTable mt, double* __restrict__ partials) {
  const int64_t base = (int64_t)blockIdx.x * NA_ATOMS_PER_BLOCK;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NA_ATOMS_PER_THREAD; k++) {
    const int64_t i = base + (int64_t)k * NA_THREADS + threadIdx.x;
    if (i < n) {
      const int t = type ? type[i] : 0;
      const double m = (unsigned)t < (unsigned)MD_MAX_TYPES ? mt.m[t] : 0.0;
      const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
      s += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Fixed-order sum of the partials of this call: out[0] = KE, out[1] = T.
__global__ void __launch_bounds__(NA_THREADS)
    k_ke_final(const double* __restrict__ partials, int nblocks, int64_t n,
               double* __restrict__ out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) s += partials[b];
  s = block_sum(s);
  if (threadIdx.x == 0) {
    out[0] = s;
    out[1] = n > 1 ? 2.0 * s / (3.0 * (double)n - 3.0) : 0.0;
  }
}

// Device address of g_ke_partials per device, looked up once per CUDA
// context: after cudaDeviceReset (or any other end of the device's primary
// context) the module is loaded again in the new context, possibly at
// another address, so each cached address is kept with the unique id of
// the context it was taken in (cuCtxGetId, reached through the runtime's
// driver entry points so that libmd.so needs no link to libcuda).
struct PartialsCache {
  unsigned long long ctx_id;
  double* addr;
};
PartialsCache g_partials[NA_MAX_DEVICES];

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Unique id of the calling thread's current CUDA context; 0 if there is
// none yet (the runtime makes the device's primary context current on its
// first call that needs one).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                         &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return 0;
    }
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

int partials_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return MD_ECUDA;
  }
  PartialsCache& c = g_partials[dev];
  const unsigned long long id = current_context_id();
  if (!c.addr || id == 0 || c.ctx_id != id) {
    // set-up for this device (or for a new context of it): with the device
    // current, the runtime resolves the array in the context that runs the
    // kernels (and creates that context if there is none yet)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ke_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return MD_ECUDA;
    }
    c.addr = static_cast<double*>(p);
    c.ctx_id = current_context_id();
  }
  *out = c.addr;
  return MD_OK;
}

}  // namespace

extern "C" int md_kinetic_noalloc(int64_t n_atoms, const double* v, const int32_t* type,
                                  int32_t n_types, const double* mass, double* out,
                                  void* stream) {
  if (n_atoms < 1 || n_atoms > MD_NOALLOC_MAX_ATOMS) return MD_EINVAL;
  if (!v || !out || !mass || n_types < 1 || n_types > MD_MAX_TYPES) return MD_EINVAL;
  MassTable mt;
  for (int t = 0; t < MD_MAX_TYPES; t++) mt.m[t] = 0.0;
  for (int t = 0; t < n_types; t++) {
    if (!(mass[t] > 0.0)) return MD_EINVAL;
    mt.m[t] = mass[t];
  }
  double* partials = nullptr;
  MD_TRY(partials_for_current_device(&partials));
  const int nblocks = (int)((n_atoms + NA_ATOMS_PER_BLOCK - 1) / NA_ATOMS_PER_BLOCK);
  cudaStream_t s = (cudaStream_t)stream;
  k_ke_partials<<<nblocks, NA_THREADS, 0, s>>>(v, type, n_atoms, mt, partials);
  k_ke_final<<<1, NA_THREADS, 0, s>>>(partials, nblocks, n_atoms, out);
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}
