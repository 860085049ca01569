// md_vjp.cuh -- the adjoint of the pair force kernel: vector-Jacobian
// products of the forces with respect to positions and to the per-type-pair
// (eps, sigma), over the same tiled neighbor list (arXiv 2508.13523, Eq. 1
// and its pairwise derivative, Sec. 4).
//
// For a pair (i, j) inside rc with d = x_j - x_i, q = |d|^2, the force on i
// is -g(q) d and on j +g(q) d, with
//   g(q)  = 24 eps (2 sigma^12 q^-7 - sigma^6 q^-4) = r^-2 r^-6 (lj1 r^-6 - lj2),
//   g'(q) = 24 eps (-14 sigma^12 q^-8 + 4 sigma^6 q^-5)
//         = r^-4 r^-6 (-7 lj1 r^-6 + 4 lj2).
// Given the cotangent c = dL/dF and w = c_i - c_j, e = -d:
//   xbar_i += J w, xbar_j -= J w,   J w = g w + 2 g' e (e . w),
//   dL/deps   += (e . w) g / eps,
//   dL/dsigma += (e . w) r^-2 r^-6 (12 lj1 r^-6 - 6 lj2) / sigma.
// Cutoffs are held fixed.  A full list visits each pair from both ends: each
// visit adds J w to its own atom only and half of the parameter terms.
#pragma once

#include <type_traits>

#include "md_device.cuh"
#include "md_internal.cuh"

struct VjpCoef {
  double inv_eps, inv_sigma;
  float inv_epsf, inv_sigmaf;
};

struct VjpArgs {
  const double4_32a* x4;
  const XSplit* xs;
  const XSplit* xb;      // positions at the last build (split)
  float rin;             // rlist rounded up: atoms this far inside every face need no image
  const double4_32a* c;  // cotangent per sorted atom (x, y, z, unused)
  const int32_t* numneigh;
  const int32_t* nbr;
  double* xbar;          // SoA per sorted atom, accumulated (+=)
  double* gbar;          // 2 nt^2: dL/deps then dL/dsigma, entry [min][max]
  const PairCoef* coef;
  const VjpCoef* vcoef;
  PairCoef c1;
  VjpCoef v1;
  const RepGeo* rep;
  int64_t n;
  int nt;
  int maxneigh;
};

template <int PREC, bool HALF, int TPA, bool SINGLE>
__global__ void __launch_bounds__(MD_BLOCK) k_vjp(const VjpArgs a) {
  __shared__ PairCoef sc[SINGLE ? 1 : MD_MAX_TYPES * MD_MAX_TYPES];
  __shared__ VjpCoef sv[SINGLE ? 1 : MD_MAX_TYPES * MD_MAX_TYPES];
  // parameter terms of each thread by partner type: [tj] eps, [MD_MAX_TYPES + tj]
  // sigma; thread-private slots, reduced once per block at the end
  __shared__ double sg[SINGLE ? 1 : MD_BLOCK][SINGLE ? 1 : 2 * MD_MAX_TYPES];
  if (!SINGLE) {
    for (int k = threadIdx.x; k < a.nt * a.nt; k += blockDim.x) {
      sc[k] = a.coef[k];
      sv[k] = a.vcoef[k];
    }
    for (int k = 0; k < 2 * MD_MAX_TYPES; k++) sg[threadIdx.x][k] = 0.0;
    __syncthreads();
  }
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid / TPA;
  const int t = (int)(gid % TPA);
  const bool active = i < a.n;
  const int64_t ia = active ? i : 0;
  const int64_t n = a.n;
  const int nin = active ? __ldg(a.numneigh + ia) : 0;
  const int nsk = active ? __ldg(a.numneigh + n + ia) : 0;
  const int32_t* row = a.nbr + (ia >> 5) * (int64_t)a.maxneigh * 32 + (ia & 31);
  const int32_t* skin = row + (int64_t)(a.maxneigh - 1) * 32;
  const double4_32a ci = a.c[ia];
  const double half = HALF ? 1.0 : 0.5;

  double bx = 0.0, by = 0.0, bz = 0.0;  // xbar_i
  double ge0 = 0.0, gs0 = 0.0;          // parameter terms when SINGLE
  double* slot = SINGLE ? nullptr : sg[threadIdx.x];
  int ti;

  if (PREC == MD_PREC_FP64) {
    const double4_32a xi = md_ld4(a.x4 + ia);
    const int tag_i = md_tag_of(xi);
    ti = MD_TAG_TYPE(tag_i);
    const RepGeo* g = a.rep + MD_TAG_REP(tag_i);
    // An atom that was at least rlist from every face at the last build has
    // no pair across the boundary until the next build (both ends of a
    // listed pair move continuously, unwrapped): its rows need no minimum
    // image.  The test is warp-uniform so that the other warps keep the
    // image code (which the compiler makes unconditional) off their pairs.
    const float4 bh = __ldg(&a.xb[ia].hi);
    const float r0 = a.rin + g->Lf[0] * 0x1p-20f, r1 = a.rin + g->Lf[1] * 0x1p-20f,
                r2b = a.rin + g->Lf[2] * 0x1p-20f;
    const bool inner_atom = bh.x >= r0 && bh.x <= g->Lf[0] - r0 && bh.y >= r1 &&
                            bh.y <= g->Lf[1] - r1 && bh.z >= r2b && bh.z <= g->Lf[2] - r2b;
    const bool no_image = __all_sync(0xffffffffu, inner_atom || !active);
    auto pairs = [&](auto wrap) {
      constexpr bool WRAP = decltype(wrap)::value;
      const double L0 = g->L[0], L1 = g->L[1], L2 = g->L[2];
      const long long h0 = g->halfL_bits[0], h1 = g->halfL_bits[1], h2 = g->halfL_bits[2];
      for (int q = t; q < nin + nsk; q += TPA) {
        const int j = __ldcs(q < nin ? row + (int64_t)q * 32 : skin - (int64_t)(q - nin) * 32);
        const double4_32a xj = md_ld4(a.x4 + j);
        double dx = __dsub_rn(xj.x, xi.x);
        double dy = __dsub_rn(xj.y, xi.y);
        double dz = __dsub_rn(xj.z, xi.z);
        if (WRAP) {
          dx = md_min_image(dx, L0, h0);
          dy = md_min_image(dy, L1, h1);
          dz = md_min_image(dz, L2, h2);
        }
        const double r2 = md_r2(dx, dy, dz);
        const int tj = SINGLE ? 0 : md_type_of(xj);
        const PairCoef& cf = SINGLE ? a.c1 : sc[ti * a.nt + tj];
        if (md_lt_pos(r2, cf.cutsq_bits)) {
          // with t = r^-2 r^-6, A = lj1 r^-6 t, B = lj2 t:
          //   g = A - B,  g' = r^-2 (-7 A + 4 B),  r^-2 r^-6 (12 lj1 r^-6 - 6 lj2) = 12 A - 6 B
          const double r2inv = md_rcp(r2);
          const double r6inv = r2inv * r2inv * r2inv;
          const double tt = r2inv * r6inv;
          const double A = (cf.lj1 * r6inv) * tt;
          const double B = cf.lj2 * tt;
          const double gq = A - B;
          const double4_32a cj = a.c[j];
          const double wx = ci.x - cj.x, wy = ci.y - cj.y, wz = ci.z - cj.z;
          const double dw = __fma_rn(dz, wz, __fma_rn(dy, wy, dx * wx));  // d . w = -(e . w)
          // J w = g w + 2 g' e (e . w) = g w + 2 g' (d . w) d
          const double sc2 = (2.0 * r2inv) * (dw * __fma_rn(-7.0, A, 4.0 * B));
          const double jx = __fma_rn(sc2, dx, gq * wx);
          const double jy = __fma_rn(sc2, dy, gq * wy);
          const double jz = __fma_rn(sc2, dz, gq * wz);
          bx += jx;
          by += jy;
          bz += jz;
          if (HALF) {
            atomicAdd(a.xbar + j, -jx);
            atomicAdd(a.xbar + n + j, -jy);
            atomicAdd(a.xbar + 2 * n + j, -jz);
          }
          // parameter terms without their 1/eps, 1/sigma factors (applied
          // once per table entry at the end); e . w = -(d . w)
          const double hw = HALF ? -dw : -0.5 * dw;
          const double de = hw * gq;
          const double ds = hw * __fma_rn(12.0, A, -6.0 * B);
          if (SINGLE) {
            ge0 += de;
            gs0 += ds;
          } else {
            slot[tj] += de;
            slot[MD_MAX_TYPES + tj] += ds;
          }
        }
      }
    };
    if (no_image)
      pairs(std::integral_constant<bool, false>{});
    else
      pairs(std::integral_constant<bool, true>{});
  } else {
    const XSplit si = md_ld_split(a.xs + ia);
    const int tag_i = __float_as_int(si.hi.w);
    ti = MD_TAG_TYPE(tag_i);
    const RepGeo* g = a.rep + MD_TAG_REP(tag_i);
    const float Lf0 = g->Lf[0], Lf1 = g->Lf[1], Lf2 = g->Lf[2];
    const float Ll0 = g->Llo[0], Ll1 = g->Llo[1], Ll2 = g->Llo[2];
    const float hf0 = g->halfLf[0], hf1 = g->halfLf[1], hf2 = g->halfLf[2];
    const float cix = (float)ci.x, ciy = (float)ci.y, ciz = (float)ci.z;
    float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f, azh = 0.f, azl = 0.f;
    for (int q = t; q < nin + nsk; q += TPA) {
      const int j = __ldcs(q < nin ? row + (int64_t)q * 32 : skin - (int64_t)(q - nin) * 32);
      const XSplit sj = md_ld_split(a.xs + j);
      float hx = sj.hi.x - si.hi.x, lx = sj.lo.x - si.lo.x;
      float hy = sj.hi.y - si.hi.y, ly = sj.lo.y - si.lo.y;
      float hz = sj.hi.z - si.hi.z, lz = sj.lo.z - si.lo.z;
      if (fabsf(hx) > hf0) {
        const float sg = copysignf(1.f, hx);
        hx -= sg * Lf0;
        lx -= sg * Ll0;
      }
      if (fabsf(hy) > hf1) {
        const float sg = copysignf(1.f, hy);
        hy -= sg * Lf1;
        ly -= sg * Ll1;
      }
      if (fabsf(hz) > hf2) {
        const float sg = copysignf(1.f, hz);
        hz -= sg * Lf2;
        lz -= sg * Ll2;
      }
      const float dx = hx + lx, dy = hy + ly, dz = hz + lz;
      const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
      const int tj = SINGLE ? 0 : MD_TAG_TYPE(__float_as_int(sj.hi.w));
      const PairCoef& cf = SINGLE ? a.c1 : sc[ti * a.nt + tj];
      // the forward kernel's cutoff decision: FP64 r^2 inside the band
      bool in = r2 < cf.cutsqf;
      if ((r2 > cf.cut_lof) & (r2 < cf.cut_hif))
        in = md_lt_pos(md_r2_split(a.xs + j, si, hf0, hf1, hf2, Lf0, Lf1, Lf2, Ll0, Ll1, Ll2),
                       cf.cutsq_bits);
      if (in) {
        const float r2inv = __frcp_rn(r2);
        const float r6inv = r2inv * r2inv * r2inv;
        const float gq = r6inv * (cf.lj1f * r6inv - cf.lj2f) * r2inv;
        const float gp = r2inv * r2inv * r6inv * (-7.0f * cf.lj1f * r6inv + 4.0f * cf.lj2f);
        const double4_32a cj = a.c[j];
        const float wx = cix - (float)cj.x, wy = ciy - (float)cj.y, wz = ciz - (float)cj.z;
        const float ew = -(dx * wx + dy * wy + dz * wz);
        const float s = -2.0f * gp * ew;
        const float jx = __fmaf_rn(s, dx, gq * wx);
        const float jy = __fmaf_rn(s, dy, gq * wy);
        const float jz = __fmaf_rn(s, dz, gq * wz);
        md_acc2(axh, axl, jx);
        md_acc2(ayh, ayl, jy);
        md_acc2(azh, azl, jz);
        if (HALF) {
          atomicAdd(a.xbar + j, -md_widen(jx));
          atomicAdd(a.xbar + n + j, -md_widen(jy));
          atomicAdd(a.xbar + 2 * n + j, -md_widen(jz));
        }
        const float hw = (float)half * ew;
        const double de = md_widen(hw * gq);
        const double ds = md_widen(hw * r2inv * r6inv * (12.0f * cf.lj1f * r6inv - 6.0f * cf.lj2f));
        if (SINGLE) {
          ge0 += de;
          gs0 += ds;
        } else {
          slot[tj] += de;
          slot[MD_MAX_TYPES + tj] += ds;
        }
      }
    }
    bx = md_widen(axh) + md_widen(axl);
    by = md_widen(ayh) + md_widen(ayl);
    bz = md_widen(azh) + md_widen(azl);
  }

  if (TPA > 1) {
#pragma unroll
    for (int off = TPA / 2; off > 0; off >>= 1) {
      bx += __shfl_xor_sync(0xffffffffu, bx, off);
      by += __shfl_xor_sync(0xffffffffu, by, off);
      bz += __shfl_xor_sync(0xffffffffu, bz, off);
    }
  }
  if (active && t == 0) {
    if (HALF) {
      atomicAdd(a.xbar + i, bx);
      atomicAdd(a.xbar + n + i, by);
      atomicAdd(a.xbar + 2 * n + i, bz);
    } else {  // only this thread touches atom i's entries
      a.xbar[i] += bx;
      a.xbar[n + i] += by;
      a.xbar[2 * n + i] += bz;
    }
  }
  // parameter terms: entry [min(ti,tj)][max(ti,tj)] of each table
  const int nt2 = a.nt * a.nt;
  if (SINGLE) {
    double v[2] = {ge0, gs0};
#pragma unroll
    for (int k = 0; k < 2; k++) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(a.gbar, v[0] * a.v1.inv_eps);
      atomicAdd(a.gbar + nt2, v[1] * a.v1.inv_sigma);
    }
  } else {
    // thread k of the block sums table entry k (eps entries, then sigma)
    // over the block's threads: one atomic per entry and block
    __shared__ int stype[MD_BLOCK];
    stype[threadIdx.x] = active ? ti : -1;
    __syncthreads();
    const int k = threadIdx.x;
    if (k < 2 * nt2) {
      const int w = k / nt2, e = k % nt2, ea = e / a.nt, eb = e % a.nt;
      if (ea <= eb) {
        double sum = 0.0;
        for (int q = 0; q < MD_BLOCK; q++) {
          const int tq = stype[q];
          if (tq == ea) sum += sg[q][w * MD_MAX_TYPES + eb];
          else if (tq == eb) sum += sg[q][w * MD_MAX_TYPES + ea];
        }
        const VjpCoef& vc = sv[ea * a.nt + eb];
        if (sum != 0.0)
          atomicAdd(a.gbar + w * nt2 + ea * a.nt + eb, sum * (w ? vc.inv_sigma : vc.inv_eps));
      }
    }
  }
}

template <int PREC, bool HALF, bool SINGLE>
cudaError_t md_vjp_launch_tpa(const VjpArgs& a, int tpa, unsigned blocks, cudaStream_t s) {
  switch (tpa) {
    case 1: k_vjp<PREC, HALF, 1, SINGLE><<<blocks, MD_BLOCK, 0, s>>>(a); break;
    case 2: k_vjp<PREC, HALF, 2, SINGLE><<<blocks, MD_BLOCK, 0, s>>>(a); break;
    case 4: k_vjp<PREC, HALF, 4, SINGLE><<<blocks, MD_BLOCK, 0, s>>>(a); break;
    case 8: k_vjp<PREC, HALF, 8, SINGLE><<<blocks, MD_BLOCK, 0, s>>>(a); break;
    case 16: k_vjp<PREC, HALF, 16, SINGLE><<<blocks, MD_BLOCK, 0, s>>>(a); break;
    case 32: k_vjp<PREC, HALF, 32, SINGLE><<<blocks, MD_BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int PREC>
cudaError_t md_vjp_launch_prec(const VjpArgs& a, bool half, bool single, int tpa,
                               unsigned blocks, cudaStream_t s) {
  if (half)
    return single ? md_vjp_launch_tpa<PREC, true, true>(a, tpa, blocks, s)
                  : md_vjp_launch_tpa<PREC, true, false>(a, tpa, blocks, s);
  return single ? md_vjp_launch_tpa<PREC, false, true>(a, tpa, blocks, s)
                : md_vjp_launch_tpa<PREC, false, false>(a, tpa, blocks, s);
}

cudaError_t md_vjp_launch_fp64(const VjpArgs& a, bool half, bool single, int tpa,
                               unsigned blocks, cudaStream_t s);
cudaError_t md_vjp_launch_mixed(const VjpArgs& a, bool half, bool single, int tpa,
                                unsigned blocks, cudaStream_t s);
