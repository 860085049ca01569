// md_integrate.cuh -- the velocity-Verlet update of one atom, shared by the
// integrator kernel (md_integrate.cu) and the fused step kernel
// (md_step_fused.cu).  See md_integrate.cu for the scheme.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "md_device.cuh"
#include "md_internal.cuh"

struct IntArgs {
  double4_32a* x4;
  double* v;
  double* f;
  unsigned long long* fix;  // fixed-point sums to fold into f (then zeroed), or NULL
  int zero;                 // K1/K21: leave f = 0 for the next pair launch's sums
  XSplit* xs;
  XFix* xq;
  const XSplit* xb;
  XGrid gr;
  unsigned int* dmax;
  int64_t n;
  double dt;
  double dtf[MD_MAX_TYPES];
};

// The update of atom i < n in mode MODE; returns its squared displacement
// since the last build (FP32, from the splits; 0 for K2).
template <int MODE>
__device__ __forceinline__ float md_integrate_atom(const IntArgs& a, int64_t i) {
  const int64_t n = a.n;
  float disp2 = 0.f;
  // every load first, before any store: the kernel is bound by the latency
  // of its loads, so all of an atom's are in flight at once
  double4_32a p = a.x4[i];
  double vx = a.v[i], vy = a.v[n + i], vz = a.v[2 * n + i];
  double fx = a.f[i], fy = a.f[n + i], fz = a.f[2 * n + i];
  long long qx = 0, qy = 0, qz = 0;
  if (a.fix) {
    qx = (long long)a.fix[i];
    qy = (long long)a.fix[n + i];
    qz = (long long)a.fix[2 * n + i];
  }
  XSplit b;
  if (MODE != MD_K2) b = a.xb[i];
  const double h = a.dtf[md_type_of(p)];
  if (a.fix) {  // the last pair launch left its fixed-point sums unfolded
    fx = md_fold_add(fx, qx);
    fy = md_fold_add(fy, qy);
    fz = md_fold_add(fz, qz);
    a.fix[i] = 0ULL;
    a.fix[n + i] = 0ULL;
    a.fix[2 * n + i] = 0ULL;
  }
  if (MODE == MD_K21 || MODE == MD_K2) {
    vx = __fma_rn(h, fx, vx);
    vy = __fma_rn(h, fy, vy);
    vz = __fma_rn(h, fz, vz);
  }
  if (MODE == MD_K21 || MODE == MD_K1) {
    vx = __fma_rn(h, fx, vx);
    vy = __fma_rn(h, fy, vy);
    vz = __fma_rn(h, fz, vz);
    p.x = __fma_rn(a.dt, vx, p.x);
    p.y = __fma_rn(a.dt, vy, p.y);
    p.z = __fma_rn(a.dt, vz, p.z);
    a.x4[i] = p;
    const XSplit s = md_store_pos(p, a.gr, a.xs, a.xq, i);
    disp2 = md_disp2(s, b, a.gr, a.xq != nullptr);
  }
  a.v[i] = vx;
  a.v[n + i] = vy;
  a.v[2 * n + i] = vz;
  if (MODE != MD_K2 && a.zero) {
    a.f[i] = 0.0;
    a.f[n + i] = 0.0;
    a.f[2 * n + i] = 0.0;
  } else if (a.fix) {
    a.f[i] = fx;
    a.f[n + i] = fy;
    a.f[2 * n + i] = fz;
  }
  return disp2;
}

// Warp-wide max of the lanes' squared displacements into *dmax (bits of a
// non-negative float order like the floats).  All 32 lanes must call it.
__device__ __forceinline__ void md_disp_max(float disp2, unsigned int* dmax) {
  const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(dmax, m);
}

// The integrator's arguments for a launch in mode `mode` (md_integrate.cu).
IntArgs md_int_args(md_ctx* c, int fold, int zero);
