// md_adjoint.cu -- gradients of force-matching losses (the VJP of the pair
// forces, and reverse mode through velocity-Verlet steps with checkpoints),
// changes of the LJ coefficients, and steepest-descent relaxation.
//
// Reverse mode through K steps.  With h = dt/2 and a = F/m, one step is
//   v' = v + h a(x),  x1 = x + dt v',  v1 = v' + h a(x1).
// Going backwards over the force evaluations e = K, K-1, ..., 0 with the
// adjoints xbar, vbar of (x_e, v_e):
//   cotangent of F(x_e):  c_K = dL/dF(x_K) (vbar_K = 0),
//                         c_e = 2 (h/m) vbar_e for 0 < e < K (the kick that
//                               ends step e-1 and the one that starts step e
//                               see the same adjoint), c_0 = (h/m) vbar_0;
//   xbar_e += J_F(x_e)^T c_e;   then, undoing the drift of step e-1,
//   vbar_{e-1} = vbar_e + dt xbar_e,  xbar_{e-1} = xbar_e.
// The forward pass stores (x, v) every `every` steps, where `every` equals
// the list cadence; a segment is recomputed from its checkpoint (the same
// positions give the same list) and differentiated in reverse.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "md_device.cuh"
#include "md_internal.cuh"
#include "md_vjp.cuh"

namespace {

template <typename T>
int dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  if (cudaMalloc((void**)p, sizeof(T) * (size_t)count) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return MD_ENOMEM;
  }
  return MD_OK;
}

__global__ void k_caller_to_sorted(const double* __restrict__ src, const int32_t* __restrict__ id,
                                   int64_t n, double* __restrict__ soa,
                                   double4_32a* __restrict__ d4) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t o = id[p];
  const double x = src[3 * o], y = src[3 * o + 1], z = src[3 * o + 2];
  if (soa) {
    soa[p] = x;
    soa[n + p] = y;
    soa[2 * n + p] = z;
  }
  if (d4) {
    double4_32a q;
    q.x = x;
    q.y = y;
    q.z = z;
    q.w = 0.0;
    d4[p] = q;
  }
}

__global__ void k_sorted_to_caller(const double* __restrict__ soa,
                                   const double4_32a* __restrict__ d4,
                                   const int32_t* __restrict__ id, int64_t n,
                                   double* __restrict__ dst) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t o = id[p];
  if (soa) {
    dst[3 * o] = soa[p];
    dst[3 * o + 1] = soa[n + p];
    dst[3 * o + 2] = soa[2 * n + p];
  } else {
    const double4_32a q = d4[p];
    dst[3 * o] = q.x;
    dst[3 * o + 1] = q.y;
    dst[3 * o + 2] = q.z;
  }
}

__global__ void k_resplit(const double4_32a* __restrict__ x4, XSplit* __restrict__ xs,
                          XFix* __restrict__ xq, int64_t n, const XGrid gr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  md_store_pos(x4[i], gr, xs, xq, i);
}

struct DtfArgs {
  double dtf[MD_MAX_TYPES];
};

// Undo the drift of step e-1 and form the next cotangent:
// vbar += dt xbar;  c = mult (h/m) vbar.
__global__ void k_adj_step(const double4_32a* __restrict__ x4, const double* __restrict__ xbar,
                           double* __restrict__ vbar, double4_32a* __restrict__ c, int64_t n,
                           double dt, double mult, DtfArgs d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double hm = mult * d.dtf[md_type_of(x4[i])];
  double4_32a q;
  double vx = __fma_rn(dt, xbar[i], vbar[i]);
  double vy = __fma_rn(dt, xbar[n + i], vbar[n + i]);
  double vz = __fma_rn(dt, xbar[2 * n + i], vbar[2 * n + i]);
  vbar[i] = vx;
  vbar[n + i] = vy;
  vbar[2 * n + i] = vz;
  q.x = hm * vx;
  q.y = hm * vy;
  q.z = hm * vz;
  q.w = 0.0;
  c[i] = q;
}

// max_i |F_i| as the bits of a non-negative double.
__global__ void k_fmax(const double* __restrict__ f, int64_t n,
                       unsigned long long* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long b = 0;
  if (i < n) {
    const double fx = f[i], fy = f[n + i], fz = f[2 * n + i];
    b = (unsigned long long)__double_as_longlong(sqrt(fx * fx + fy * fy + fz * fz));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
    b = o > b ? o : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(out, b);
}

// x <- x + alpha F / max|F|
__global__ void k_sd_update(double4_32a* __restrict__ x4, const double* __restrict__ f,
                            int64_t n, double alpha, const unsigned long long* __restrict__ fmax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = __longlong_as_double((long long)*fmax);
  if (!(m > 0.0)) return;
  const double s = alpha / m;
  double4_32a p = x4[i];
  p.x = __fma_rn(s, f[i], p.x);
  p.y = __fma_rn(s, f[n + i], p.y);
  p.z = __fma_rn(s, f[2 * n + i], p.z);
  x4[i] = p;
}

int upload_vcoef(md_ctx* c) {
  VjpCoef tab[MD_MAX_TYPES * MD_MAX_TYPES];
  memset(tab, 0, sizeof(tab));
  for (int k = 0; k < c->nt * c->nt; k++) {
    tab[k].inv_eps = 1.0 / c->eps[k];
    tab[k].inv_sigma = 1.0 / c->sigma[k];
    tab[k].inv_epsf = (float)tab[k].inv_eps;
    tab[k].inv_sigmaf = (float)tab[k].inv_sigma;
  }
  if (!c->vcoef) MD_TRY(dalloc((VjpCoef**)&c->vcoef, MD_MAX_TYPES * MD_MAX_TYPES));
  MD_CUDA(cudaMemcpyAsync(c->vcoef, tab, sizeof(tab), cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));  // tab must outlive the copy
  return MD_OK;
}

int adj_reserve(md_ctx* c, int64_t seg_positions) {
  const int64_t n = c->n;
  if (!c->adj_c) MD_TRY(dalloc(&c->adj_c, n));
  if (!c->adj_xbar) MD_TRY(dalloc(&c->adj_xbar, 3 * n));
  if (!c->adj_vbar) MD_TRY(dalloc(&c->adj_vbar, 3 * n));
  if (!c->adj_carry) MD_TRY(dalloc(&c->adj_carry, 9 * n));
  if (!c->gbar) MD_TRY(dalloc(&c->gbar, 2 * MD_MAX_TYPES * MD_MAX_TYPES));
  if (!c->vcoef) MD_TRY(upload_vcoef(c));
  if (seg_positions > c->seg_cap) {
    if (c->seg_x) cudaFree(c->seg_x);
    c->seg_x = nullptr;
    c->seg_cap = 0;
    MD_TRY(dalloc(&c->seg_x, seg_positions * n));
    c->seg_cap = seg_positions;
  }
  return MD_OK;
}

int launch_vjp(md_ctx* c) {
  VjpArgs a;
  a.x4 = c->x4;
  a.xs = c->xs;
  a.xb = c->xb;
  a.rin = nextafterf((float)c->rlist, INFINITY);
  a.c = c->adj_c;
  a.numneigh = c->numneigh;
  a.nbr = c->nbr;
  a.xbar = c->adj_xbar;
  a.gbar = c->gbar;
  a.coef = c->coef;
  a.vcoef = (const VjpCoef*)c->vcoef;
  a.c1 = c->coef1;
  a.v1.inv_eps = 1.0 / c->eps[0];
  a.v1.inv_sigma = 1.0 / c->sigma[0];
  a.v1.inv_epsf = (float)a.v1.inv_eps;
  a.v1.inv_sigmaf = (float)a.v1.inv_sigma;
  a.rep = c->rep;
  a.n = c->n;
  a.nt = c->nt;
  a.maxneigh = c->maxneigh;
  const int tpa = c->tpa > 0 ? c->tpa : 1;
  const unsigned blocks = (unsigned)md_blocks(c->n * (int64_t)tpa);
  const bool half = c->list_kind == MD_LIST_HALF;
  cudaError_t e = (c->precision == MD_PREC_FP64)
                      ? md_vjp_launch_fp64(a, half, c->nt == 1, tpa, blocks, c->stream)
                      : md_vjp_launch_mixed(a, half, c->nt == 1, tpa, blocks, c->stream);
  c->launches++;
  MD_CUDA(e);
  return MD_OK;
}

// gbar (device, entry [min][max]) -> host, both entries of each pair.
int gbar_to_host(md_ctx* c, double* out) {
  const int nt = c->nt, nt2 = nt * nt;
  double h[2 * MD_MAX_TYPES * MD_MAX_TYPES];
  MD_CUDA(cudaMemcpyAsync(h, c->gbar, sizeof(double) * 2 * nt2, cudaMemcpyDeviceToHost,
                          c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  for (int w = 0; w < 2; w++)
    for (int a = 0; a < nt; a++)
      for (int b = 0; b < nt; b++) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        out[w * nt2 + a * nt + b] = h[w * nt2 + lo * nt + hi];
      }
  return MD_OK;
}

int to_sorted(md_ctx* c, const double* src, double* soa, double4_32a* d4) {
  k_caller_to_sorted<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(src, c->id, c->n,
                                                                          soa, d4);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int to_caller(md_ctx* c, const double* soa, const double4_32a* d4, double* dst) {
  k_sorted_to_caller<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(soa, d4, c->id,
                                                                          c->n, dst);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int resplit(md_ctx* c) {
  k_resplit<<<(unsigned)md_blocks(c->n), MD_BLOCK, 0, c->stream>>>(c->x4, c->xs, c->xq, c->n,
                                                                   c->xgrid);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int64_t n_checkpoints(int64_t nsteps, int every) { return (nsteps + every - 1) / every + 1; }

}  // namespace

extern "C" {

int md_set_lj(md_ctx* c, const double* eps, const double* sigma) {
  if (!c || !eps || !sigma) return MD_EINVAL;
  const int nt = c->nt;
  for (int a = 0; a < nt; a++)
    for (int b = 0; b < nt; b++) {
      const double e = eps[a * nt + b], s = sigma[a * nt + b];
      if (!(e > 0.0) || !(s > 0.0) || !isfinite(e) || !isfinite(s)) return MD_EINVAL;
      if (e != eps[b * nt + a] || s != sigma[b * nt + a]) return MD_EINVAL;
    }
  for (int k = 0; k < nt * nt; k++) {
    c->eps[k] = eps[k];
    c->sigma[k] = sigma[k];
  }
  MD_TRY(md_upload_coef(c));
  md_drop_graphs(c);  // graphs hold the single-type coefficients by value
  if (c->vcoef) MD_TRY(upload_vcoef(c));
  return MD_OK;
}

int md_force_vjp(md_ctx* c, const double* cot, double* xbar, double* gbar) {
  if (!c || !cot || !xbar || !gbar) return MD_EINVAL;
  if (c->coul) return MD_EINVAL;  // the adjoint is of Eq. 1 (lj/cut) only
  MD_TRY(adj_reserve(c, 0));
  MD_TRY(to_sorted(c, cot, nullptr, c->adj_c));
  MD_CUDA(cudaMemsetAsync(c->adj_xbar, 0, sizeof(double) * 3 * c->n, c->stream));
  MD_CUDA(cudaMemsetAsync(c->gbar, 0, sizeof(double) * 2 * MD_MAX_TYPES * MD_MAX_TYPES,
                          c->stream));
  MD_TRY(launch_vjp(c));
  MD_TRY(to_caller(c, c->adj_xbar, nullptr, xbar));
  return gbar_to_host(c, gbar);
}

int md_traj_forward(md_ctx* c, int64_t nsteps, int32_t every, const double* x0,
                    const double* v0, double* ckpt_x, double* ckpt_v, double* f_final) {
  if (!c || nsteps < 0 || every < 1 || !x0 || !v0 || !ckpt_x || !ckpt_v || !f_final)
    return MD_EINVAL;
  if (c->coul) return MD_EINVAL;  // the adjoint is of Eq. 1 (lj/cut) only
  if (every != c->rebuild_every) return MD_EINVAL;
  const int64_t n3 = 3 * c->n;
  const int64_t J = n_checkpoints(nsteps, every) - 1;
  MD_TRY(md_set_state(c, x0, v0, MD_MEM_DEVICE));
  for (int64_t j = 0; j < J; j++) {
    MD_TRY(md_get_state(c, ckpt_x + j * n3, ckpt_v + j * n3, nullptr, MD_MEM_DEVICE));
    const int64_t m = nsteps - j * every < every ? nsteps - j * every : every;
    MD_TRY(md_step(c, m));
  }
  return md_get_state(c, ckpt_x + J * n3, ckpt_v + J * n3, f_final, MD_MEM_DEVICE);
}

int md_traj_vjp(md_ctx* c, int64_t nsteps, int32_t every, const double* ckpt_x,
                const double* ckpt_v, const double* cot_final, double* x0bar, double* v0bar,
                double* gbar) {
  if (!c || nsteps < 0 || every < 1 || !ckpt_x || !ckpt_v || !cot_final || !x0bar || !v0bar ||
      !gbar)
    return MD_EINVAL;
  if (c->coul) return MD_EINVAL;  // the adjoint is of Eq. 1 (lj/cut) only
  if (every != c->rebuild_every) return MD_EINVAL;
  const int64_t n = c->n, n3 = 3 * n;
  const int64_t J = n_checkpoints(nsteps, every) - 1;
  MD_TRY(adj_reserve(c, every));
  double* XB = c->adj_carry;  // caller order
  double* VB = c->adj_carry + n3;
  double* CC = c->adj_carry + 2 * n3;
  MD_CUDA(cudaMemsetAsync(XB, 0, sizeof(double) * 2 * n3, c->stream));
  MD_CUDA(cudaMemcpyAsync(CC, cot_final, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                          c->stream));
  MD_CUDA(cudaMemsetAsync(c->gbar, 0, sizeof(double) * 2 * MD_MAX_TYPES * MD_MAX_TYPES,
                          c->stream));
  DtfArgs d;
  for (int t = 0; t < MD_MAX_TYPES; t++) d.dtf[t] = c->dtf[t];
  for (int64_t j = J; j >= 0; j--) {
    const int64_t s0 = j * every < nsteps ? j * every : nsteps;
    const int64_t e_hi = (j == J) ? nsteps : ((j + 1) * every < nsteps ? (j + 1) * every : nsteps) - 1;
    // recompute the segment's positions from its checkpoint
    MD_TRY(md_set_state(c, ckpt_x + j * n3, ckpt_v + j * n3, MD_MEM_DEVICE));
    const int64_t npos = e_hi - s0 + 1;
    MD_CUDA(cudaMemcpyAsync(c->seg_x, c->x4, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice,
                            c->stream));
    for (int64_t k = 1; k < npos; k++) {
      MD_TRY(md_step(c, 1));
      MD_CUDA(cudaMemcpyAsync(c->seg_x + k * n, c->x4, sizeof(double4_32a) * n,
                              cudaMemcpyDeviceToDevice, c->stream));
    }
    // carried adjoints into this segment's sorted order
    MD_TRY(to_sorted(c, XB, c->adj_xbar, nullptr));
    MD_TRY(to_sorted(c, VB, c->adj_vbar, nullptr));
    MD_TRY(to_sorted(c, CC, nullptr, c->adj_c));
    for (int64_t e = e_hi; e >= s0; e--) {
      MD_CUDA(cudaMemcpyAsync(c->x4, c->seg_x + (e - s0) * n, sizeof(double4_32a) * n,
                              cudaMemcpyDeviceToDevice, c->stream));
      MD_TRY(resplit(c));
      MD_TRY(launch_vjp(c));
      if (e == 0) break;
      const double mult = (e - 1 >= 1) ? 2.0 : 1.0;
      k_adj_step<<<(unsigned)md_blocks(n), MD_BLOCK, 0, c->stream>>>(
          c->x4, c->adj_xbar, c->adj_vbar, c->adj_c, n, c->dt, mult, d);
      c->launches++;
      MD_CUDA(cudaGetLastError());
    }
    MD_TRY(to_caller(c, c->adj_xbar, nullptr, XB));
    MD_TRY(to_caller(c, c->adj_vbar, nullptr, VB));
    MD_TRY(to_caller(c, nullptr, c->adj_c, CC));
  }
  MD_CUDA(cudaMemcpyAsync(x0bar, XB, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
  MD_CUDA(cudaMemcpyAsync(v0bar, VB, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
  // leave a consistent state: the initial positions with their forces
  MD_TRY(md_set_state(c, ckpt_x, ckpt_v, MD_MEM_DEVICE));
  return gbar_to_host(c, gbar);
}

int md_minimize(md_ctx* c, int64_t nsteps, double alpha) {
  if (!c || nsteps < 0 || !(alpha > 0.0) || !isfinite(alpha)) return MD_EINVAL;
  if (!c->fmax_bits) MD_TRY(dalloc(&c->fmax_bits, 1));
  const unsigned nb = (unsigned)md_blocks(c->n);
  for (int64_t s = 0; s < nsteps; s++) {
    if (s > 0 && s % c->rebuild_every == 0) MD_TRY(md_rebuild(c));
    MD_TRY(md_launch_pair(c, 0, c->tpa > 0 ? c->tpa : 1));
    MD_CUDA(cudaMemsetAsync(c->fmax_bits, 0, sizeof(unsigned long long), c->stream));
    k_fmax<<<nb, MD_BLOCK, 0, c->stream>>>(c->f, c->n, c->fmax_bits);
    k_sd_update<<<nb, MD_BLOCK, 0, c->stream>>>(c->x4, c->f, c->n, alpha, c->fmax_bits);
    c->launches += 2;
    MD_CUDA(cudaGetLastError());
    MD_TRY(resplit(c));  // the mixed form reads positions from the split
  }
  c->step = 0;
  return md_fresh_start(c);
}

}  // extern "C"
