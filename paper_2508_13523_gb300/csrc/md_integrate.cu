// md_integrate.cu -- fused velocity-Verlet NVE update with the displacement
// check, kinetic energy, block-partial reductions and the state copies
// between the caller's atom order and the cell-sorted order.
//
// Velocity Verlet (the integrator is not described in arXiv 2508.13523; the
// step follows the usual NVE scheme): with h = dt/2/m per type,
//   K1  (start of a step):   v = v + h f;  x = x + dt v
//   K2  (end of a step):     v = v + h f            (f at the new positions)
//   K21 (end of step s fused with the start of step s+1):
//                            v = v + h f;  v = v + h f;  x = x + dt v
// K21 applies the two half kicks one after the other, so it rounds exactly
// like K2 followed by K1.  Inside a step segment the kernel also takes over
// the bookkeeping of the pair launches' force sums: it folds fixed-point
// sums into f (K21, K2) and, where the next pair launch accumulates into f,
// leaves f and the fixed-point sums at zero (K1, K21).  Every update is one FMA: v = fma(h, f, v),
// x = fma(dt, v, x).  After each drift the kernel refreshes the double-float
// split of x (FP64 contexts: its hi parts and the fixed-point record) and
// reduces max |x - x_build|^2 (FP32 from the splits; FP64 contexts: an upper
// bound from the hi parts, md_disp2) into a device word, which the rebuild
// reads to count builds that came later than a skin/2 displacement.
// Kinetic energies are summed per replica.
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_device.cuh"
#include "md_integrate.cuh"
#include "md_internal.cuh"

namespace {

template <int MODE>
__global__ void __launch_bounds__(MD_BLOCK) k_integrate(const IntArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float disp2 = i < a.n ? md_integrate_atom<MODE>(a, i) : 0.f;
  if (MODE != MD_K2) md_disp_max(disp2, a.dmax);
}

// f += fix * 2^-MD_FIX_BITS and fix = 0, element by element (3n of each):
// folds the fixed-point force sums of k_pair_q<FIX> into the FP64 forces
// (which hold the contributions too large for the accumulators).  The fold
// rounds once, in the final addition.
// Two elements per thread with 16-byte accesses (both arrays are 256-byte
// aligned); m may be odd.
__global__ void __launch_bounds__(MD_BLOCK)
    k_fix_finalize(double* __restrict__ f, unsigned long long* __restrict__ fix, int64_t m) {
  const int64_t k = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (k + 1 < m) {
    const longlong2 q = *reinterpret_cast<const longlong2*>(fix + k);
    double2 v = *reinterpret_cast<const double2*>(f + k);
    *reinterpret_cast<longlong2*>(fix + k) = make_longlong2(0, 0);
    v.x = md_fold_add(v.x, q.x);
    v.y = md_fold_add(v.y, q.y);
    *reinterpret_cast<double2*>(f + k) = v;
  } else if (k < m) {
    const long long q = (long long)fix[k];
    fix[k] = 0ULL;
    f[k] = md_fold_add(f[k], q);
  }
}

struct MassArgs {
  double m[MD_MAX_TYPES];
};

// Kinetic energy of each replica into word 8 of its accumulator rows
// (md_warp_add_rep).
__global__ void __launch_bounds__(MD_BLOCK)
    k_kinetic(const double4_32a* __restrict__ x4, const double* __restrict__ v, int64_t n,
              MassArgs ma, double* __restrict__ acc, int spread) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[1] = {0.0};
  int rep = -1;
  if (i < n) {
    const int tag = md_tag_of(x4[i]);
    rep = MD_TAG_REP(tag);
    const double m = ma.m[MD_TAG_TYPE(tag)];
    const double vx = v[i], vy = v[n + i], vz = v[2 * n + i];
    s[0] = 0.5 * m * (vx * vx + vy * vy + vz * vz);
  }
  md_warp_add_rep<1>(s, rep, acc + 8, spread, (int)((i >> 5) % spread));
}

// The virial by atoms: words 1..6 of the replica's accumulator rows += sum
// over the replica's atoms of (x_a - c) (x) F_a (xx, yy, zz, xy, xz, yz; c the box
// centre, which the sum does not depend on since the forces of a box sum to
// zero).  With the pair kernels' image terms (-sum over pairs taken through
// a periodic image of s (x) g, s the shift taken off the separation) this is
// sum over pairs of fpair d (x) d: F_i = -g and F_j = +g for each pair, and
// x_j - x_i = d + s.  Each block takes a contiguous run of `chunk` atoms (a
// replica changes only a few times along it); a thread flushes its sums when
// its replica changes, the warps reduce them at the end.
__global__ void __launch_bounds__(MD_BLOCK)
    k_virial_atoms(const double4_32a* __restrict__ x4, const double* __restrict__ f,
                   const RepGeo* __restrict__ rep, int64_t n, int64_t chunk,
                   double* __restrict__ acc, int spread) {
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  const int slot = (int)((((int64_t)blockIdx.x * MD_BLOCK + threadIdx.x) >> 5) % spread);
  double w[6] = {0, 0, 0, 0, 0, 0};
  int cur = -1;
  double cx = 0.0, cy = 0.0, cz = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += MD_BLOCK) {
    const double4_32a p = x4[i];
    const int r = MD_TAG_REP(md_tag_of(p));
    if (r != cur) {
      if (cur >= 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
          atomicAdd(acc + ((int64_t)cur * spread + slot) * MD_EV_STRIDE + 1 + k, w[k]);
          w[k] = 0.0;
        }
      }
      cur = r;
      cx = 0.5 * rep[r].L[0];
      cy = 0.5 * rep[r].L[1];
      cz = 0.5 * rep[r].L[2];
    }
    const double x = p.x - cx, y = p.y - cy, z = p.z - cz;
    const double fx = f[i], fy = f[n + i], fz = f[2 * n + i];
    w[0] = __fma_rn(x, fx, w[0]);
    w[1] = __fma_rn(y, fy, w[1]);
    w[2] = __fma_rn(z, fz, w[2]);
    w[3] = __fma_rn(x, fy, w[3]);
    w[4] = __fma_rn(x, fz, w[4]);
    w[5] = __fma_rn(y, fz, w[5]);
  }
  md_warp_add_rep<6>(w, cur, acc + 1, spread, slot);
}

// ev[r * MD_EV_STRIDE + k] += the sum of the replica's `spread` accumulator
// rows' word k, which are left at zero.  One thread per (replica, word).
__global__ void __launch_bounds__(MD_BLOCK)
    k_ev_fold(double* __restrict__ rows, double* __restrict__ ev, int nrep, int spread) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrep * MD_EV_STRIDE) return;
  const int64_t r = t / MD_EV_STRIDE, k = t % MD_EV_STRIDE;
  double* p = rows + r * spread * MD_EV_STRIDE + k;
  double s = 0.0;
  for (int j = 0; j < spread; j++) {
    s += p[(int64_t)j * MD_EV_STRIDE];
    p[(int64_t)j * MD_EV_STRIDE] = 0.0;
  }
  ev[t] += s;
}

// Caller order -> sorted arrays (identity order), tags from tag0.
__global__ void k_load_state(const double* __restrict__ x, const double* __restrict__ v,
                             const int32_t* __restrict__ tag0, int64_t n,
                             double4_32a* __restrict__ x4, double* __restrict__ vs,
                             int32_t* __restrict__ id) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4_32a p;
  p.x = x[3 * i];
  p.y = x[3 * i + 1];
  p.z = x[3 * i + 2];
  p.w = md_tag_bits(tag0[i]);
  x4[i] = p;
  vs[i] = v[3 * i];
  vs[n + i] = v[3 * i + 1];
  vs[2 * n + i] = v[3 * i + 2];
  id[i] = (int32_t)i;
}

// Caller order -> the current sorted order, keeping tags, order and list:
// x4[p].xyz = x[id[p]], v[p] = v[id[p]], split refreshed; the largest
// |x - x_build|^2 (md_disp2) goes to both words of disp, and
// disp_new[1] is set to 1 if any position differs (bit pattern) from the one
// the context held.
__global__ void k_load_keep(const double* __restrict__ x, const double* __restrict__ v,
                            const int32_t* __restrict__ id, int64_t n,
                            double4_32a* __restrict__ x4, double* __restrict__ vs,
                            XSplit* __restrict__ xs, XFix* __restrict__ xq,
                            const XSplit* __restrict__ xb, const XGrid gr,
                            unsigned int* __restrict__ disp_run,
                            unsigned int* __restrict__ disp_new) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.f;
  bool moved = false;
  if (p < n) {
    const int64_t o = id[p];
    double4_32a q = x4[p];
    const double nx = x[3 * o], ny = x[3 * o + 1], nz = x[3 * o + 2];
    const double wx = v[3 * o], wy = v[3 * o + 1], wz = v[3 * o + 2];
    const XSplit b = xb[p];  // every load before the stores
    moved = (__double_as_longlong(nx) != __double_as_longlong(q.x)) |
            (__double_as_longlong(ny) != __double_as_longlong(q.y)) |
            (__double_as_longlong(nz) != __double_as_longlong(q.z));
    q.x = nx;
    q.y = ny;
    q.z = nz;
    x4[p] = q;
    vs[p] = wx;
    vs[n + p] = wy;
    vs[2 * n + p] = wz;
    const XSplit s = md_store_pos(q, gr, xs, xq, p);
    d2 = md_disp2(s, b, gr, xq != nullptr);
    if (!(d2 < 3.0e38f)) d2 = 3.0e38f;  // non-finite input: never keep the list
  }
  const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(d2));
  const bool any_moved = __any_sync(0xffffffffu, moved);
  if ((threadIdx.x & 31) == 0) {
    if (m) {
      atomicMax(disp_run, m);
      atomicMax(disp_new, m);
    }
    if (any_moved) atomicOr(disp_new + 1, 1u);
  }
}

__global__ void k_store_state(const double4_32a* __restrict__ x4, const double* __restrict__ vs,
                              const double* __restrict__ fs, const int32_t* __restrict__ id,
                              int64_t n, double* __restrict__ x, double* __restrict__ v,
                              double* __restrict__ f) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t o = id[p];
  if (x) {
    const double4_32a q = x4[p];
    x[3 * o] = q.x;
    x[3 * o + 1] = q.y;
    x[3 * o + 2] = q.z;
  }
  if (v) {
    v[3 * o] = vs[p];
    v[3 * o + 1] = vs[n + p];
    v[3 * o + 2] = vs[2 * n + p];
  }
  if (f) {
    f[3 * o] = fs[p];
    f[3 * o + 1] = fs[n + p];
    f[3 * o + 2] = fs[2 * n + p];
  }
}

}  // namespace

IntArgs md_int_args(md_ctx* c, int fold, int zero) {
  IntArgs a;
  a.x4 = c->x4;
  a.v = c->v;
  a.f = c->f;
  a.fix = fold ? c->fix : nullptr;
  a.zero = zero;
  a.xs = c->xs;
  a.xq = c->xq;
  a.gr = c->xgrid;
  a.xb = c->xb;
  a.dmax = c->dmax;
  a.n = c->n;
  a.dt = c->dt;
  for (int t = 0; t < MD_MAX_TYPES; t++) a.dtf[t] = c->dtf[t];
  return a;
}

int md_launch_integrate(md_ctx* c, int mode, int fold, int zero) {
  const IntArgs a = md_int_args(c, fold, zero);
  const unsigned nb = (unsigned)md_blocks(c->n);
  if (mode == MD_K1)
    k_integrate<MD_K1><<<nb, MD_BLOCK, 0, c->stream>>>(a);
  else if (mode == MD_K21)
    k_integrate<MD_K21><<<nb, MD_BLOCK, 0, c->stream>>>(a);
  else
    k_integrate<MD_K2><<<nb, MD_BLOCK, 0, c->stream>>>(a);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_launch_fix_finalize(md_ctx* c) {
  static_assert(MD_FIX_BITS == 44, "the scale in k_fix_finalize is 2^-44");
  const int64_t m = 3 * c->n;
  k_fix_finalize<<<(unsigned)md_blocks((m + 1) / 2), MD_BLOCK, 0, c->stream>>>(c->f, c->fix, m);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_launch_kinetic(md_ctx* c) {
  MassArgs ma;
  for (int t = 0; t < MD_MAX_TYPES; t++) ma.m[t] = c->mass[t];
  k_kinetic<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(c->x4, c->v, c->n, ma,
                                                                   c->evs, c->ev_spread);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return md_launch_ev_fold(c);
}

int md_launch_ev_fold(md_ctx* c) {
  k_ev_fold<<<(unsigned)md_blocks((int64_t)c->nrep * MD_EV_STRIDE), MD_BLOCK, 0, c->stream>>>(
      c->evs, c->ev, c->nrep, c->ev_spread);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_launch_virial_atoms(md_ctx* c) {
  // 8 blocks per SM, each a contiguous run of whole blocks' worth of atoms
  const int64_t cap = 8 * (int64_t)(c->nsm > 0 ? c->nsm : 1);
  const int64_t nb = md_blocks(c->n) < cap ? md_blocks(c->n) : cap;
  const int64_t per = (md_blocks(c->n) + nb - 1) / nb;
  const int64_t blocks = (md_blocks(c->n) + per - 1) / per;
  k_virial_atoms<<<(unsigned)blocks, MD_BLOCK, 0, c->stream>>>(c->x4, c->f, c->rep, c->n,
                                                                per * MD_BLOCK, c->evs,
                                                                c->ev_spread);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_launch_load_state(md_ctx* c, const double* x, const double* v) {
  k_load_state<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(x, v, c->tag0, c->n,
                                                                      c->x4, c->v, c->id);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_launch_load_keep(md_ctx* c, const double* x, const double* v) {
  k_load_keep<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(
      x, v, c->id, c->n, c->x4, c->v, c->xs, c->xq, c->xb, c->xgrid, c->dmax, c->dmax + 3);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_launch_store_state(md_ctx* c, double* x, double* v, double* f) {
  k_store_state<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(c->x4, c->v, c->f, c->id,
                                                                       c->n, x, v, f);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}
