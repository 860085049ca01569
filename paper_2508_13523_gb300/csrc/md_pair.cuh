// md_pair.cuh -- the Lennard-Jones pair kernel over the tiled neighbor list
// (arXiv 2508.13523, Eq. 1 and Sec. 4: forces are the pairwise derivative of
// E; Sec. 4.1: half list with atomics vs full list computing every pair
// twice, one atom per thread vs threads cooperating on one atom's neighbors,
// and the GPU list layout that interleaves consecutive atoms' lists).
//
// One template covers both precisions, both list kinds, T threads per atom
// (T | 32: the T lanes of an atom take neighbors k = t, t+T, ...; a warp
// covers 32/T consecutive atoms, so a warp-wide row read of the tiled list is
// T sector-aligned runs of 32/T indices), energy/virial on demand, and a
// single-type fast path (coefficients in kernel parameters instead of a
// shared-memory table).  With energy and virial the pair loop adds only the
// energy, a pair count and, for pairs taken through a periodic image, the
// virial's image terms; the rest of the virial is summed over atoms from the
// final forces (k_virial_atoms), which costs one pass over x and f instead
// of six FMAs per pair.
//
// FP64 form: separations, r^2, the cutoff test and all force arithmetic in
// FP64; the reciprocal is a hardware seed plus one cubic series round
// (md_rcp); cutoff and minimum-image tests are integer compares of bit
// patterns, so the FP64 pipe (the binding resource on GB300) only sees the
// arithmetic.
//
// Mixed form: no FP64 instruction per pair outside the cutoff bands.
// Positions are read as a double-float split (md_split: hi on a power-of-two
// grid, lo the rest; refreshed by the integrator), the separation is formed
// as (hi_j - hi_i) + (lo_j - lo_i) in FP32 (the hi difference and its image
// shift are exact, so the result is within an FP32 ulp of the FP64
// separation), and r^2 and the force are FP32.  The force is accumulated
// exactly: each FP32 contribution g = fpair d is converted, with integer
// instructions, to a 64-bit fixed-point count of 2^-44 units (md_fix32:
// exact for |g| >= 2^-21), and the counts are summed in 64-bit integers --
// the owner's share in registers, f_j's share (half list) by global integer
// reductions into fix -- and folded into the FP64 forces once per atom (the
// integrator, or md_launch_fix_finalize).  The sum does not depend on the
// order of the additions and lies within (contributions) x 2^-44 of the
// exact sum of the FP32 contributions, i.e. FP64-class accumulation; a
// contribution too large for the accumulators' range goes to f by FP64
// reductions.  The cutoff test is FP32 except within 2^-18 (relative) of a
// cutoff, where an FP64 r^2 decides after the loop.
#pragma once

#include <climits>
#include <type_traits>

#include "md_device.cuh"
#include "md_internal.cuh"

struct PairArgs {
  const double4_32a* x4;
  const XSplit* xs;
  const XFix* xq;        // fixed-point positions (compacted FP64 kernel's integer path)
  const int32_t* numneigh;
  const int32_t* nbr;
  double* f;            // SoA fx[n], fy[n], fz[n]
  unsigned long long* fix;   // SoA fixed-point accumulators (k_pair_q<FIX>, mixed
                             // k_pair); zero at entry of a half-list launch
  const unsigned int* kmax;  // bound on the contributions one atom receives
  const PairCoef* coef;  // nt*nt table (multi-type)
  PairCoef c1;           // the only coefficients when nt == 1
  const RepGeo* rep;     // box of each replica
  double* ev;            // per-replica accumulators: ev_spread rows of MD_EV_STRIDE
                         // doubles each (md_warp_add_rep)
  int ev_spread;
  int* tile_ctr;         // per-SM tile counters (zeroed before each launch), or
                         // NULL: one tile per block
  int nslots;            // counters (= SMs)
  int64_t n;
  int nt;
  int maxneigh;
};

// Persistent scheduling: the tiles (consecutive atoms, cell-sorted) are cut
// into one contiguous range per SM; a block takes the next tile of the range
// of the SM it runs on, and of the following SMs' ranges once its own is
// done.  Blocks on one SM then work on neighboring atoms, whose neighbor
// positions stay in that SM's L1.  Returns -1 when every range is done.
__device__ __forceinline__ int md_next_tile(int* ctr, int nslots, int ntiles) {
  unsigned sm;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
  const int s0 = (int)(sm % (unsigned)nslots);
  for (int k = 0; k < nslots; k++) {
    int s = s0 + k;
    if (s >= nslots) s -= nslots;
    const int lo = (int)((int64_t)s * ntiles / nslots);
    const int len = (int)((int64_t)(s + 1) * ntiles / nslots) - lo;
    if (len <= 0 || *(volatile int*)(ctr + s) >= len) continue;
    const int t = atomicAdd(ctr + s, 1);
    if (t < len) return lo + t;
  }
  return -1;
}

// Resident blocks per SM the register allocation must allow.  The mixed
// kernels are bound by the latency of their position loads: registers buy
// loads in flight (two entries a round), resident warps hide them.
// Mixed half-list energy/virial launches: at 4M atoms 7, 8, 9 and 10 blocks
// measured 2.00, 1.89, 1.82 and 1.97 ms (TPA 2).
// Mixed force-only launches walk their rows two entries a round (MD_PAIR_U),
// both gathers in flight: at 4M atoms (TPA 2) against one entry at 10
// blocks, 1.469 -> 1.440 ms (half list, 9 blocks: 56 registers) and 1.717 ->
// 1.408 ms (full list, 10 blocks); the half list at 10 blocks spills (1.60
// ms), the full list at 9 blocks measured 1.437 ms.
#ifndef MD_PAIR_U
#define MD_PAIR_U 2
#endif
// Mixed full-list energy/virial launches: two entries a round at 8 blocks
// measured 2.13 ms at 4M atoms, one at 10 (spills) 2.26 ms, one at 9
// 2.37 ms, two at 7 2.24 ms; the half-list ones keep one entry at 9 blocks
// (two spill).
#ifndef MD_PAIR_U_EV_FULL
#define MD_PAIR_U_EV_FULL 2
#endif
#ifndef MD_PAIR_MINB_EV_FULL
#define MD_PAIR_MINB_EV_FULL 8
#endif
constexpr int md_pair_minb(int prec, bool half, bool ev) {
  return prec == MD_PREC_MIXED ? (ev ? (half ? 9 : MD_PAIR_MINB_EV_FULL) : (half ? 9 : 10))
                               : (ev ? 6 : 8);
}

// COUL (mixed precision only): the lj/cut/coul/cut style, Eq. 1 plus the
// cut Coulomb term qq / r.
template <int PREC, bool HALF, int TPA, bool EV, bool SINGLE, bool COUL = false>
__global__ void __launch_bounds__(MD_BLOCK, md_pair_minb(PREC, HALF, EV)) k_pair(const PairArgs a) {
  static_assert(!COUL || PREC == MD_PREC_MIXED, "the FP64 Coulomb form is k_pair_q");
  __shared__ PairCoef sc[SINGLE ? 1 : MD_MAX_TYPES * MD_MAX_TYPES];
  if (!SINGLE) {
    for (int k = threadIdx.x; k < a.nt * a.nt; k += blockDim.x) sc[k] = a.coef[k];
    __syncthreads();
  }
  __shared__ int s_tile;
  // the virial's image terms (rare) of each thread: its own column
  __shared__ double simg[EV ? 6 : 1][MD_BLOCK];
  if (EV) {
  #pragma unroll
    for (int k = 0; k < 6; k++) simg[k][threadIdx.x] = 0.0;
  }
  const int ntiles = (int)((a.n * TPA + MD_BLOCK - 1) / MD_BLOCK);
  for (int it = 0;; it++) {
    if (threadIdx.x == 0)
      s_tile = a.tile_ctr ? md_next_tile(a.tile_ctr, a.nslots, ntiles)
                          : (it == 0 ? (int)blockIdx.x : -1);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile < 0) break;
    const int64_t gid = tile * MD_BLOCK + threadIdx.x;
    const int64_t i = gid / TPA;
    const int t = (int)(gid % TPA);
    const bool active = i < a.n;
    const int64_t ia = active ? i : 0;
    const int64_t n = a.n;
    const int nin = active ? __ldg(a.numneigh + ia) : 0;
    const int nsk = active ? __ldg(a.numneigh + n + ia) : 0;
    const int32_t* row = a.nbr + (ia >> 5) * (int64_t)a.maxneigh * 32 + (ia & 31);
    // inner entries at k = 0..nin-1, skin entries at k = maxneigh-1-s
    const int32_t* skin = row + (int64_t)(a.maxneigh - 1) * 32;

    double fx = 0.0, fy = 0.0, fz = 0.0;
    double e0 = 0.0;  // energy (FP64, several types)
    int npair = 0;    // pairs within rc
    // the energy's partial sums: FP64, one type -- sum r^-6 alone, the
    // energy being trace(W) / 12 - (lj4 / 2) sum r^-6 (lj1 = 12 lj3, lj2 =
    // 6 lj4: a pair's energy is fpair r^2 / 12 - (lj4 / 2) r^-6), with the
    // virial's trace added where the energy is read; mixed -- an FP32 sum
    // with its rounding errors (TwoSum), folded into FP64 after the loop
    double s6 = 0.0;
    float es = 0.f, ec = 0.f;
    const double evw = HALF ? 1.0 : 0.5;  // a full list visits each pair twice
    int rep_i = 0;

    if (PREC == MD_PREC_FP64) {
      const double4_32a xi = md_ld4(a.x4 + ia);
      const int tag_i = md_tag_of(xi);
      const int ti = MD_TAG_TYPE(tag_i);
      rep_i = MD_TAG_REP(tag_i);
      const RepGeo* g = a.rep + rep_i;
      const double L0 = g->L[0], L1 = g->L[1], L2 = g->L[2];
      const long long h0 = g->halfL_bits[0], h1 = g->halfL_bits[1], h2 = g->halfL_bits[2];
      for (int q = t; q < nin + nsk; q += TPA) {
        const int j = __ldcs(q < nin ? row + (int64_t)q * 32 : skin - (int64_t)(q - nin) * 32);
        const double4_32a xj = md_ld4(a.x4 + j);
        double dx = __dsub_rn(xj.x, xi.x);
        double dy = __dsub_rn(xj.y, xi.y);
        double dz = __dsub_rn(xj.z, xi.z);
        double shx = 0.0, shy = 0.0, shz = 0.0;  // EV: the image shift s L taken off d
        if (md_abs_gt(dx, h0) | md_abs_gt(dy, h1) | md_abs_gt(dz, h2)) {
          if (EV) {
            shx = md_abs_gt(dx, h0) ? copysign(L0, dx) : 0.0;
            shy = md_abs_gt(dy, h1) ? copysign(L1, dy) : 0.0;
            shz = md_abs_gt(dz, h2) ? copysign(L2, dz) : 0.0;
          }
          dx = md_min_image(dx, L0, h0);
          dy = md_min_image(dy, L1, h1);
          dz = md_min_image(dz, L2, h2);
        }
        const double r2 = md_r2(dx, dy, dz);
        const PairCoef& c = SINGLE ? a.c1 : sc[ti * a.nt + md_type_of(xj)];
        if (md_lt_pos(r2, c.cutsq_bits)) {
          const double r2inv = md_rcp(r2);
          const double r6inv = r2inv * r2inv * r2inv;
          const double fpair = r6inv * (c.lj1 * r6inv - c.lj2) * r2inv;
          // d = x_j - x_i: F_i -= fpair d, F_j += fpair d
          if (HALF) {
            const double gx = fpair * dx, gy = fpair * dy, gz = fpair * dz;
            fx -= gx;
            fy -= gy;
            fz -= gz;
            atomicAdd(a.f + j, gx);
            atomicAdd(a.f + n + j, gy);
            atomicAdd(a.f + 2 * n + j, gz);
          } else {
            fx = __fma_rn(-fpair, dx, fx);
            fy = __fma_rn(-fpair, dy, fy);
            fz = __fma_rn(-fpair, dz, fz);
          }
          if (EV) {  // weighted once after the loop; the virial is x (x) F per
                     // atom afterwards, less the image terms
            if (SINGLE) {
              s6 += r6inv;
            } else {
              e0 += r6inv * (c.lj3 * r6inv - c.lj4);
            }
            npair++;
            if ((shx != 0.0) | (shy != 0.0) | (shz != 0.0)) {
              const double gx = fpair * dx, gy = fpair * dy, gz = fpair * dz;
              double* m = &simg[0][threadIdx.x];
              m[0 * MD_BLOCK] = __fma_rn(-shx, gx, m[0 * MD_BLOCK]);
              m[1 * MD_BLOCK] = __fma_rn(-shy, gy, m[1 * MD_BLOCK]);
              m[2 * MD_BLOCK] = __fma_rn(-shz, gz, m[2 * MD_BLOCK]);
              m[3 * MD_BLOCK] = __fma_rn(-shx, gy, m[3 * MD_BLOCK]);
              m[4 * MD_BLOCK] = __fma_rn(-shx, gz, m[4 * MD_BLOCK]);
              m[5 * MD_BLOCK] = __fma_rn(-shy, gz, m[5 * MD_BLOCK]);
            }
          }
        }
      }
    } else {
      const XSplit si = md_ld_split(a.xs + ia);
      const int tag_i = __float_as_int(si.hi.w);
      const int ti = MD_TAG_TYPE(tag_i);
      rep_i = MD_TAG_REP(tag_i);
      const RepGeo* g = a.rep + rep_i;
      const float hf0 = g->halfLf[0], hf1 = g->halfLf[1], hf2 = g->halfLf[2];
      // the box edges are read where a pair needs an image (volatile: the
      // loads stay there instead of holding six registers across the loop)
      auto edge = [&](int k, float& Lf, float& Ll) {
        asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(Lf) : "l"(g->Lf + k));
        asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(Ll) : "l"(g->Llo + k));
      };
      // exact fixed-point force sums (md_fix32); a contribution goes there
      // only if its FP32 exponent is below ex_lim, so that |q| < 2^52 and
      // the at most kmax < 2^kb contributions to one atom sum below 2^63
      long long ax = 0, ay = 0, az = 0;
      const int kb = 32 - __clz((int)min(*a.kmax, 0x7fffffffu));
      const int ex_lim = min(127 + MD_FIX_EMAX + 1, 127 + 63 - MD_FIX_BITS - kb);
      // Cutoff decisions.  Outside a relative band of 2^-18 around rc^2 (and
      // rc_coul^2) the FP32 r^2 decides: its error, ~7 2^-24 relative, cannot
      // carry it across.  A pair inside a band is decided on an FP64 r^2
      // (md_r2_split), so that the mixed kernels sum over the pairs the FP64
      // kernels do: lj/cut jumps by |F(rc)| at the cutoff, and a pair decided
      // the other way would cost that whole force.  The loop only notes such
      // a pair in one pending slot (its row position; skin entries nin + s;
      // -1 none, INT_MAX more than one), updated without a branch, and the
      // slot is worked off after the loop; two or more send the thread over
      // its share of the row again, deciding only band pairs.
      int pend = -1;
      auto pair = [&](int j, const XSplit& sj, int pos, auto second) {
        constexpr bool SECOND = decltype(second)::value;
        float hx = sj.hi.x - si.hi.x, lx = sj.lo.x - si.lo.x;
        float hy = sj.hi.y - si.hi.y, ly = sj.lo.y - si.lo.y;
        float hz = sj.hi.z - si.hi.z, lz = sj.lo.z - si.lo.z;
        int shf = 0;  // EV: image shifts taken off d, 2 bits per axis (+L: 1, -L: 2)
        if ((fabsf(hx) > hf0) | (fabsf(hy) > hf1) | (fabsf(hz) > hf2)) {  // rare
          float Lf, Ll;
          if (fabsf(hx) > hf0) {
            edge(0, Lf, Ll);
            const float sg = copysignf(1.f, hx);
            if (EV) shf |= sg > 0.f ? 1 : 2;
            hx -= sg * Lf;
            lx -= sg * Ll;
          }
          if (fabsf(hy) > hf1) {
            edge(1, Lf, Ll);
            const float sg = copysignf(1.f, hy);
            if (EV) shf |= sg > 0.f ? 4 : 8;
            hy -= sg * Lf;
            ly -= sg * Ll;
          }
          if (fabsf(hz) > hf2) {
            edge(2, Lf, Ll);
            const float sg = copysignf(1.f, hz);
            if (EV) shf |= sg > 0.f ? 16 : 32;
            hz -= sg * Lf;
            lz -= sg * Ll;
          }
        }
        const float dx = hx + lx, dy = hy + ly, dz = hz + lz;
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
        const PairCoef& c = SINGLE ? a.c1 : sc[ti * a.nt + MD_TAG_TYPE(__float_as_int(sj.hi.w))];
        const bool band = ((r2 > c.cut_lof) & (r2 < c.cut_hif)) |
                          (COUL && ((r2 > c.coul_lof) & (r2 < c.coul_hif)));
        bool in_lj = r2 < c.cutsqf, in_co = COUL && r2 < c.cutsq_coulf;
        if (!SECOND) {
          pend = band ? (pend < 0 ? pos : INT_MAX) : pend;
          if (band) return;
        } else {
          if (!band) return;  // decided in FP32 by the main loop
          const double r2d =
              md_r2_split(a.xs + j, si, hf0, hf1, hf2, g->Lf[0], g->Lf[1], g->Lf[2],
                          g->Llo[0], g->Llo[1], g->Llo[2]);
          in_lj = md_lt_pos(r2d, c.cutsq_bits);
          in_co = COUL && md_lt_pos(r2d, c.cutsq_coul_bits);
        }
        if (in_lj | in_co) {
          float r2inv, r6inv, fpair, qr = 0.f;
          if (COUL) {
            float rinv;
            asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv) : "f"(r2));
            r2inv = rinv * rinv;
            r6inv = r2inv * r2inv * r2inv;
            const float flj = in_lj ? r6inv * (c.lj1f * r6inv - c.lj2f) * r2inv : 0.f;
            qr = in_co ? c.qqf * rinv : 0.f;
            fpair = __fmaf_rn(qr, r2inv, flj);
          } else {
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r2inv) : "f"(r2));
            r6inv = r2inv * r2inv * r2inv;
            fpair = r6inv * (c.lj1f * r6inv - c.lj2f) * r2inv;
          }
          const float gx = fpair * dx, gy = fpair * dy, gz = fpair * dz;
          if (md_fix32_fits(gx, gy, gz, ex_lim)) {
            const long long qx = md_fix32(gx);
            ax -= qx;
            if (HALF) atomicAdd(a.fix + j, (unsigned long long)qx);  // f_j's share, in L2
            const long long qy = md_fix32(gy);
            ay -= qy;
            if (HALF) atomicAdd(a.fix + n + j, (unsigned long long)qy);
            const long long qz = md_fix32(gz);
            az -= qz;
            if (HALF) atomicAdd(a.fix + 2 * n + j, (unsigned long long)qz);
          } else {  // beyond the fixed-point range (rare): FP64 reductions into f
            atomicAdd(a.f + ia, -(double)gx);
            atomicAdd(a.f + n + ia, -(double)gy);
            atomicAdd(a.f + 2 * n + ia, -(double)gz);
            if (HALF) {
              atomicAdd(a.f + j, (double)gx);
              atomicAdd(a.f + n + j, (double)gy);
              atomicAdd(a.f + 2 * n + j, (double)gz);
            }
          }
          if (EV) {  // weighted once after the loop; the virial is x (x) F per
                     // atom afterwards, less these image terms
            float en = r6inv * (c.lj3f * r6inv - c.lj4f);
            if (COUL) en = (in_lj ? en : 0.f) + qr;
            {  // TwoSum: es + en = t + the error, exactly
              const float t = __fadd_rn(es, en);
              const float bp = __fsub_rn(t, es);
              const float ap = __fsub_rn(t, bp);
              ec = __fadd_rn(ec, __fadd_rn(__fsub_rn(es, ap), __fsub_rn(en, bp)));
              es = t;
            }
            npair++;
            if (shf) {  // rare
              auto sh = [&](int k) {
                const int b = (shf >> (2 * k)) & 3;
                return b == 1 ? g->L[k] : (b == 2 ? -g->L[k] : 0.0);
              };
              const double sx = sh(0), sy = sh(1), sz = sh(2);
              const double wx = md_widen(gx), wy = md_widen(gy), wz = md_widen(gz);
              double* m = &simg[0][threadIdx.x];
              m[0 * MD_BLOCK] = __fma_rn(-sx, wx, m[0 * MD_BLOCK]);
              m[1 * MD_BLOCK] = __fma_rn(-sy, wy, m[1 * MD_BLOCK]);
              m[2 * MD_BLOCK] = __fma_rn(-sz, wz, m[2 * MD_BLOCK]);
              m[3 * MD_BLOCK] = __fma_rn(-sx, wy, m[3 * MD_BLOCK]);
              m[4 * MD_BLOCK] = __fma_rn(-sx, wz, m[4 * MD_BLOCK]);
              m[5 * MD_BLOCK] = __fma_rn(-sy, wz, m[5 * MD_BLOCK]);
            }
          }
        }
      };
      // inner entries from the front of the row, skin entries from the back
      // (force-only launches: PU entries a round, their gathers in flight
      // together)
      constexpr int PU = EV ? (HALF ? 1 : MD_PAIR_U_EV_FULL) : MD_PAIR_U;
      auto walk = [&](auto second) {
        const int32_t* p = row + (int64_t)t * 32;
        int q = t;
        if (PU == 2) {
          for (; q + TPA < nin; q += 2 * TPA, p += 2 * TPA * 32) {
            const int j0 = __ldcs(p), j1 = __ldcs(p + TPA * 32);
            const XSplit s0 = md_ld_split(a.xs + j0), s1 = md_ld_split(a.xs + j1);
            pair(j0, s0, q, second);
            pair(j1, s1, q + TPA, second);
          }
        }
        for (; q < nin; q += TPA, p += TPA * 32) {
          const int j = __ldcs(p);
          pair(j, md_ld_split(a.xs + j), q, second);
        }
        const int32_t* ps = skin - (int64_t)t * 32;
        q = t;
        if (PU == 2) {
          for (; q + TPA < nsk; q += 2 * TPA, ps -= 2 * TPA * 32) {
            const int j0 = __ldcs(ps), j1 = __ldcs(ps - TPA * 32);
            const XSplit s0 = md_ld_split(a.xs + j0), s1 = md_ld_split(a.xs + j1);
            pair(j0, s0, nin + q, second);
            pair(j1, s1, nin + q + TPA, second);
          }
        }
        for (; q < nsk; q += TPA, ps -= TPA * 32) {
          const int j = __ldcs(ps);
          pair(j, md_ld_split(a.xs + j), nin + q, second);
        }
      };
      walk(std::false_type{});
      if (pend == INT_MAX) {
        walk(std::true_type{});
      } else if (pend >= 0) {
        const int32_t* p = pend < nin ? row + (int64_t)pend * 32 : skin - (int64_t)(pend - nin) * 32;
        const int j = __ldcs(p);
        pair(j, md_ld_split(a.xs + j), pend, std::true_type{});
      }
      if (TPA > 1) {
  #pragma unroll
        for (int off = TPA / 2; off > 0; off >>= 1) {
          ax += __shfl_xor_sync(0xffffffffu, ax, off);
          ay += __shfl_xor_sync(0xffffffffu, ay, off);
          az += __shfl_xor_sync(0xffffffffu, az, off);
        }
      }
      if (active && t == 0) {
        if (HALF) {  // f_i also receives f_j shares from other owners
          atomicAdd(a.fix + i, (unsigned long long)ax);
          atomicAdd(a.fix + n + i, (unsigned long long)ay);
          atomicAdd(a.fix + 2 * n + i, (unsigned long long)az);
        } else {  // full list: the owner's sum is the whole count
          a.fix[i] = (unsigned long long)ax;
          a.fix[n + i] = (unsigned long long)ay;
          a.fix[2 * n + i] = (unsigned long long)az;
        }
      }
    }

    if (PREC == MD_PREC_FP64 && TPA > 1) {
  #pragma unroll
      for (int off = TPA / 2; off > 0; off >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, off);
        fy += __shfl_xor_sync(0xffffffffu, fy, off);
        fz += __shfl_xor_sync(0xffffffffu, fz, off);
      }
    }
    if (PREC == MD_PREC_FP64 && active && t == 0) {
      if (HALF) {
        atomicAdd(a.f + i, fx);
        atomicAdd(a.f + n + i, fy);
        atomicAdd(a.f + 2 * n + i, fz);
      } else {
        a.f[i] = fx;
        a.f[n + i] = fy;
        a.f[2 * n + i] = fz;
      }
    }
    if (EV) {
      double ev[8];
      ev[0] = PREC == MD_PREC_MIXED ? md_widen(es) + md_widen(ec)
                                    : (SINGLE ? -0.5 * a.c1.lj4 * s6 : e0);
  #pragma unroll
      for (int k = 1; k < 7; k++) {
        ev[k] = simg[k - 1][threadIdx.x];
        simg[k - 1][threadIdx.x] = 0.0;
      }
  #pragma unroll
      for (int k = 0; k < 7; k++) ev[k] *= evw;
      ev[7] = evw * (double)npair;
      md_warp_add_rep<8>(ev, active ? rep_i : -1, a.ev, a.ev_spread,
                         (int)(((int64_t)blockIdx.x * MD_BLOCK + threadIdx.x) >> 5) % a.ev_spread);
    }
  }
}

// Applies the preferred shared-memory carveout (percent; -1 leaves the
// driver default) to a kernel on the current device, once per (kernel,
// device, carveout), and returns in *occ its resident blocks per SM of
// MD_BLOCK threads at that carveout.  Thread safe (md_capi.cu).
cudaError_t md_prepare_kernel(const void* kernel, int carve, int* occ);

// Launch one instantiation; carve is the preferred shared-memory carveout in
// percent (0: largest L1, the LJ kernel's cache -- Sec. 4.4 -- uses almost no
// shared memory).  Returns cudaGetLastError().
template <typename K>
cudaError_t md_launch_carved(K kernel, const PairArgs& a, unsigned blocks, cudaStream_t s,
                             int carve) {
  int occ = 1;
  cudaError_t e = md_prepare_kernel((const void*)kernel, carve, &occ);
  if (e != cudaSuccess) return e;
  // persistent: as many blocks as can be resident at once
  if (a.tile_ctr) {
    const unsigned cap = (unsigned)(a.nslots * occ);
    if (blocks > cap) blocks = cap;
  }
  kernel<<<blocks, MD_BLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

template <int PREC, bool HALF, bool EV, bool SINGLE>
cudaError_t md_pair_launch_tpa(const PairArgs& a, int tpa, unsigned blocks, cudaStream_t s,
                               int carve) {
  switch (tpa) {
    case 1: return md_launch_carved(k_pair<PREC, HALF, 1, EV, SINGLE>, a, blocks, s, carve);
    case 2: return md_launch_carved(k_pair<PREC, HALF, 2, EV, SINGLE>, a, blocks, s, carve);
    case 4: return md_launch_carved(k_pair<PREC, HALF, 4, EV, SINGLE>, a, blocks, s, carve);
    case 8: return md_launch_carved(k_pair<PREC, HALF, 8, EV, SINGLE>, a, blocks, s, carve);
    case 16: return md_launch_carved(k_pair<PREC, HALF, 16, EV, SINGLE>, a, blocks, s, carve);
    case 32: return md_launch_carved(k_pair<PREC, HALF, 32, EV, SINGLE>, a, blocks, s, carve);
    default: return cudaErrorInvalidValue;
  }
}

template <int PREC>
cudaError_t md_pair_launch_prec(const PairArgs& a, bool half, bool ev, bool single, int tpa,
                                unsigned blocks, cudaStream_t s, int carve) {
  if (half) {
    if (ev) return single ? md_pair_launch_tpa<PREC, true, true, true>(a, tpa, blocks, s, carve)
                          : md_pair_launch_tpa<PREC, true, true, false>(a, tpa, blocks, s, carve);
    return single ? md_pair_launch_tpa<PREC, true, false, true>(a, tpa, blocks, s, carve)
                  : md_pair_launch_tpa<PREC, true, false, false>(a, tpa, blocks, s, carve);
  }
  if (ev) return single ? md_pair_launch_tpa<PREC, false, true, true>(a, tpa, blocks, s, carve)
                        : md_pair_launch_tpa<PREC, false, true, false>(a, tpa, blocks, s, carve);
  return single ? md_pair_launch_tpa<PREC, false, false, true>(a, tpa, blocks, s, carve)
                : md_pair_launch_tpa<PREC, false, false, false>(a, tpa, blocks, s, carve);
}

cudaError_t md_pair_launch_fp64(const PairArgs& a, bool half, bool ev, bool single, int tpa,
                                unsigned blocks, cudaStream_t s, int carve);
cudaError_t md_pair_launch_mixed(const PairArgs& a, bool half, bool ev, bool single, int tpa,
                                 unsigned blocks, cudaStream_t s, int carve);
// lj/cut/coul/cut, mixed precision, threads per atom 1, 2 or 4 (md_pair_coul.cu)
cudaError_t md_pair_launch_mixed_coul(const PairArgs& a, bool half, bool ev, bool single,
                                      int tpa, unsigned blocks, cudaStream_t s, int carve);
