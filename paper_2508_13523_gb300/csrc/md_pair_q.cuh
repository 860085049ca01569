// md_pair_q.cuh -- FP64 pair kernel with warp-level compaction of in-range
// pairs (arXiv 2508.13523, Eq. 1 and Sec. 4; Sec. 4.1 names the two sources
// of GPU divergence this removes: rows of different length and the cutoff
// branch).
//
// On GB300 the FP64 pipe is the bottleneck of the FP64 form, and in a
// one-thread-per-atom loop a warp issues every FP64 instruction for all 32
// lanes even when only some lanes have a pair inside rc (rows end at
// different lengths; skin pairs are mostly outside rc).  Here each warp
//   phase 1: takes one list entry per lane and tests it in FP32 against a
//            certified upper bound of rc^2 (positions' FP32 split and the FP32
//            arithmetic bounded as in the list build); entries that are
//            certainly outside rc are dropped, the rest are appended to one
//            of two per-warp queues in shared memory (ballot + popc): queue
//            1 if the FP32 separation along some axis is close to or above
//            half the box (a periodic image may be nearer), queue 0 if
//            certainly not;
//   phase 2: whenever 32 entries are queued, all 32 lanes take one each and
//            do the exact FP64 work: separation, minimum image (queue 1
//            only), r^2, the exact cutoff test, the force, and global
//            reductions into the owner's force and (half list) f_j, which
//            start from zero.
// The two queues keep the minimum image, which the compiler turns into
// three unconditional FP64 subtractions, off the ~98 % of pairs (in a large
// box) that never cross the boundary.
// The FP64 decisions and arithmetic per pair are those of k_pair; only the
// summation of the contributions into f_i differs:
//   FIX = false: FP64 reductions into f (order-dependent rounding);
//   FIX = true:  each contribution is rounded to a multiple of 2^-44 and
//                summed exactly in 64-bit integers: the owner's share in a
//                shared-memory accumulator of its warp (added to fix once
//                per atom), f_j's by a global reduction into fix;
//                contributions too large for the accumulators' range go to
//                f by FP64 reductions; md_launch_fix_finalize then adds fix
//                to f.  The sum is independent of the order, within
//                (contributions) x 2^-45 of the exact sum, needs no FP64
//                instruction (shared-memory FP64 atomics would run on the
//                FP64 pipe, and the owner's -g costs an FP64 negation when
//                it feeds an FP64 reduction) and sends one global reduction
//                per pair to L2 instead of two.
// Integer path (FIX, force-only, Eq. 1 alone): positions are also kept as
// fixed-point integers X = x 2^F (XFix; F per box, 53 for a 168-wide box),
// exact for every coordinate from 2^(52 - F) up and flagged otherwise.  Queue 0 then holds only pairs of
// unflagged atoms, whose separation D = X_j - X_i is the exact x_j - x_i.
// r^2 is formed from D with 64-bit high products (md_sep_r2: within 1.1
// ulps below the exact r^2), and each force contribution fpair d is the
// product of fpair's significand and |D|, rounded to a fixed-point count
// (md_fix_prod: within one count of the exact value).  That leaves 8 FP64
// operations per pair (the reciprocal's 3, r^-6's 2, fpair's 3) instead of
// 17.  The cutoff is decided on that r^2 except within 4 ulps of rc^2,
// where the oracle's rounded fma(dz,dz, fma(dy,dy, dx*dx)) decides (that
// expression lies within 1.5 ulps of the exact value, so
// outside the band both agree).  Pairs with a flagged atom go to queue 1.
// COUL adds the second pair style's cut Coulomb term qq / r (1/r from the
// rsqrt seed and one series round; r^-2 = (1/r)^2 instead of md_rcp).
#pragma once

#include <type_traits>

#include "md_device.cuh"
#include "md_internal.cuh"
#include "md_pair.cuh"

#define MD_Q_CAP 64  // queue entries per warp (a ring; at most 63 in use)
// U: list entries per lane per round of phase 1 (their loads in flight
// together), 1 or 2; 2 only in force-only fixed-point launches, where the
// tuner picks it per workload.  At 4M atoms (one box), 2 entries with 9
// blocks per SM against 1 with 10: 2.545 vs 2.577 ms (half list), 4.216 vs
// 4.340 ms (full); 2 with 10 blocks (spills) 2.61 ms, 3 or 4 with 8 blocks
// 3.3-3.9 ms.  The 512-replica batch (4.96M atoms) ran 7 % slower with 2.
// Resident blocks per SM the register allocation must allow (force-only
// launches): 10 x 128 threads caps the kernel at 48 registers, which it
// fits without spills.
#define MD_Q_MINB 10
// The same for the fixed-point launches, whose queue-0 drain takes the
// integer path: at 4M atoms with one list entry per round, 10 blocks (48
// registers) measured 2.58 ms per launch, 9 (56) 2.64 ms and 8 (64)
// 2.78 ms; with two entries a filter round the best is 9 blocks.
#define MD_Q_MINB_INT 10
#define MD_Q_MINB_INT2 9

// The tile loop of the compacted kernel: every block of the launch runs it
// (k_pair_q, and the pair phase of k_step_fused).  All threads of the block
// must call it.
template <bool HALF, bool EV, bool SINGLE, bool FIX, bool COUL, int U>
__device__ __forceinline__ void md_pair_q_tiles(const PairArgs& a, const float cut_hi1,
                                                const float* __restrict__ cut_hi_tab) {
  constexpr int W = MD_BLOCK / 32;
  // queue 0 takes the integer path: separations, r^2 and the fixed-point
  // contributions from the XFix positions (Eq. 1 launches)
  constexpr bool INTX = FIX && !COUL;
  // range of the fixed-point accumulators: a contribution goes there only if
  // its biased exponent is below ex_lim, so that |q| <= 2^(ex_lim - 1023 + 44)
  // and the at most kmax < 2^kb contributions to one atom sum below 2^63
  int ex_lim = 0, qbits = 0;
  if (FIX) {
    const int kb = 32 - __clz((int)min(*a.kmax, 0x7fffffffu));
    ex_lim = min(1023 + MD_FIX_EMAX + 1, 1023 + 63 - MD_FIX_BITS - kb);
    qbits = ex_lim - 1023 + MD_FIX_BITS;  // |count| < 2^qbits: the same range
  }
  __shared__ PairCoef sc[SINGLE ? 1 : MD_MAX_TYPES * MD_MAX_TYPES];
  __shared__ float scut[SINGLE ? 1 : MD_MAX_TYPES * MD_MAX_TYPES];
  __shared__ int qj[2][W][MD_Q_CAP];            // queue 0: no image, 1: may wrap
  __shared__ unsigned char qo[2][W][MD_Q_CAP];
  __shared__ double4_32a xown[W][32];      // owner positions (x, y, z, tag)
  __shared__ XFix xownq[INTX ? W : 1][32];  // owner fixed-point positions
  __shared__ double sev[EV ? W : 1][8][32];  // owner energy/virial accumulators
  __shared__ unsigned long long sown[FIX ? W : 1][3][32];  // owner fixed-point forces
  if (!SINGLE) {
    for (int k = threadIdx.x; k < a.nt * a.nt; k += blockDim.x) {
      sc[k] = a.coef[k];
      scut[k] = cut_hi_tab[k];
    }
  }
  if (!SINGLE) __syncthreads();
  __shared__ int s_tile;
  const int ntiles = (int)((a.n + MD_BLOCK - 1) / MD_BLOCK);
  for (int it = 0;; it++) {
    if (threadIdx.x == 0)
      s_tile = a.tile_ctr ? md_next_tile(a.tile_ctr, a.nslots, ntiles)
                          : (it == 0 ? (int)blockIdx.x : -1);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile < 0) break;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = tile * MD_BLOCK + threadIdx.x;
    const bool active = i < a.n;
    const int64_t ia = active ? i : 0;
    const int64_t n = a.n;
    const int nin = active ? __ldg(a.numneigh + ia) : 0;
    const int nsk = active ? __ldg(a.numneigh + n + ia) : 0;
    const int cnt = nin + nsk;
    const int32_t* row = a.nbr + (ia >> 5) * (int64_t)a.maxneigh * 32 + (ia & 31);
    const int32_t* skin = row + (int64_t)(a.maxneigh - 1) * 32;
    const double4_32a xi = md_ld4(a.x4 + ia);
    const int tag_i = md_tag_of(xi);
    const int ti = MD_TAG_TYPE(tag_i);
    const RepGeo* g = a.rep + MD_TAG_REP(tag_i);
    // FP32 view of the own position (phase 1)
    const float4 hi = __ldg(&a.xs[ia].hi);
    const float Lf0 = g->Lf[0], Lf1 = g->Lf[1], Lf2 = g->Lf[2];
    const float hf0 = g->halfLf[0], hf1 = g->halfLf[1], hf2 = g->halfLf[2];
    // routing bound (1 - 2^-12) L/2: the FP32 separation of the hi parts is
    // within 3 * 2^-24 L of the FP64 one, so |d32| <= this bound on every
    // axis means |d| < L/2 in FP64 (no periodic image is nearer)
    const float hm0 = hf0 * (1.f - 0x1p-12f), hm1 = hf1 * (1.f - 0x1p-12f),
                hm2 = hf2 * (1.f - 0x1p-12f);
    xown[w][lane] = xi;
    // an owner with some coordinate off the fixed-point grid sends all its
    // pairs to queue 1 (FP64 separations)
    const bool own_off = INTX && (__float_as_int(hi.w) & MD_TAG_OFFGRID);
    if (INTX) xownq[INTX ? w : 0][lane] = md_ld_xfix(a.xq + ia);
    if (FIX) {
  #pragma unroll
      for (int k = 0; k < 3; k++) sown[w][k][lane] = 0ULL;
    }
    if (EV) {
  #pragma unroll
      for (int k = 0; k < 8; k++) sev[w][k][lane] = 0.0;
    }
    __syncthreads();

    // Energy and virial: when every active atom of the warp lies in one box
    // (always for a single box), each lane sums the pairs it drains in
    // registers -- E, a pair count, and for the rare pairs taken through a
    // periodic image (queue 1 only) the virial's image terms -s_a g_b (s the
    // shift taken off d, g = fpair d) -- and the warp reduces them once;
    // otherwise they go to per-owner shared accumulators and then to the
    // owners' boxes.  The rest of the virial, sum_a x_a (x) F_a, is summed
    // per atom after the forces are complete.  The shuffle and vote run on
    // every lane.
    const int rep_i = MD_TAG_REP(tag_i);
    bool uni = false;
    int rep0 = -1;
    if (EV) {
      const int r0 = __shfl_sync(0xffffffffu, rep_i, 0);
      uni = __all_sync(0xffffffffu, !active || rep_i == r0);
      rep0 = __any_sync(0xffffffffu, active) ? r0 : -1;
    }
    double e0 = 0.0;  // this lane's energy sum (uniform warps; the virial's image
                      // terms, rare, go to the lane's own column of sev)
    int npair = 0;
    // one type, Eq. 1 alone: with lj1 = 12 lj3 and lj2 = 6 lj4 a pair's
    // energy is fpair r^2 / 12 - (lj4 / 2) r^-6, and the sum of fpair r^2 is
    // the trace of the virial, which the sum over atoms gives; so the loop
    // sums r^-6 alone (one FP64 add a pair) and the trace's share is added
    // where the energy is read (md_capi.cu, fill_thermo).  All pairs of the
    // box take this form, the shared-accumulator path too.
    constexpr bool S2 = SINGLE && !COUL;
    double s6 = 0.0;
    const double evw = HALF ? 1.0 : 0.5;
    int q = 0;            // this lane's next list entry
    unsigned head[2] = {0, 0}, tail[2] = {0, 0};  // warp-uniform ring counters

    // phase 2: one queued pair per lane, exact FP64
    auto drain = [&](auto queue, unsigned take) {
      constexpr int Q = decltype(queue)::value;
      const unsigned e = head[Q] + lane;
      if (INTX && Q == 0 && lane < take) {
        const int j = qj[Q][w][e % MD_Q_CAP];
        const int o = qo[Q][w][e % MD_Q_CAP];
        const XFix po = xownq[INTX ? w : 0][o];
        const XFix pj = md_ld_xfix(a.xq + j);
        // separations in units of 2^-F (F of the pair's box): exact, as is
        // x_j - x_i in FP64 here
        const long long Dx = pj.x - po.x, Dy = pj.y - po.y, Dz = pj.z - po.z;
        const int F = (int)(po.w >> 32);
        unsigned long long Ax, Ay, Az;
        int sh;
        double r2 = md_sep_r2(Dx, Dy, Dz, F, Ax, Ay, Az, sh);
        const int to = MD_TAG_TYPE((int)po.w);
        const PairCoef& c = SINGLE ? a.c1 : sc[to * a.nt + MD_TAG_TYPE((int)pj.w)];
        // r^2 from the exact separations (within 1.1 ulps below the exact
        // value) decides unless it lies within 4 ulps of rc^2, where
        // fma(dz,dz, fma(dy,dy, dx*dx)) -- within 1.5 ulps of the exact
        // value -- could fall on the other side: those pairs are decided on
        // that FP64 r^2, the definition the oracle uses
        const long long rb = __double_as_longlong(r2);
        bool in = rb < c.cutsq_bits - 4;
        if (!in && rb <= c.cutsq_bits + 4) {
          const double sc = __longlong_as_double((long long)(1023 - F) << 52);  // 2^-F
          r2 = md_r2(__dmul_rn(__ll2double_rn(Dx), sc), __dmul_rn(__ll2double_rn(Dy), sc),
                     __dmul_rn(__ll2double_rn(Dz), sc));
          in = md_lt_pos(r2, c.cutsq_bits);
        }
        if (in) {
          const double r2inv = md_rcp(r2);
          const double r6inv = r2inv * r2inv * r2inv;
          const double fpair = r6inv * (c.lj1 * r6inv - c.lj2) * r2inv;
          const int64_t io = tile * MD_BLOCK + w * 32 + o;
          // each component on its own: its exact fixed-point count, or --
          // beyond the accumulators' range (rare) -- FP64 reductions of
          // g = fpair d; either way the owner's and j's shares match
          auto comp = [&](long long D, unsigned long long A, int k) {
            long long q;
            if (md_fix_prod(fpair, A, D < 0, sh, F, qbits, q)) {
              atomicAdd(&sown[FIX ? w : 0][k][o], (unsigned long long)(-q));
              if (HALF) atomicAdd(a.fix + k * n + j, (unsigned long long)q);
            } else {
              const double g =
                  fpair * __dmul_rn(__ll2double_rn(D),
                                    __longlong_as_double((long long)(1023 - F) << 52));
              atomicAdd(a.f + k * n + io, md_neg(g));
              if (HALF) atomicAdd(a.f + k * n + j, g);
            }
          };
          comp(Dx, Ax, 0);
          comp(Dy, Ay, 1);
          comp(Dz, Az, 2);
          if (EV) {  // queue 0 never crosses the boundary: no image term of the virial
            if (uni) {
              if (S2)
                s6 += r6inv;
              else
                e0 += r6inv * (c.lj3 * r6inv - c.lj4);
              npair++;
            } else {
              atomicAdd(&sev[w][0][o], evw * (S2 ? -0.5 * c.lj4 * r6inv
                                                 : r6inv * (c.lj3 * r6inv - c.lj4)));
              atomicAdd(&sev[w][7][o], evw);
            }
          }
        }
      } else if (lane < take) {
        const int j = qj[Q][w][e % MD_Q_CAP];
        const int o = qo[Q][w][e % MD_Q_CAP];
        const double4_32a xo = xown[w][o];
        const double4_32a xj = md_ld4(a.x4 + j);
        double dx = __dsub_rn(xj.x, xo.x);
        double dy = __dsub_rn(xj.y, xo.y);
        double dz = __dsub_rn(xj.z, xo.z);
        double shx = 0.0, shy = 0.0, shz = 0.0;  // EV: the image shift s L taken off d
        if (Q == 1) {
          const RepGeo* go = a.rep + MD_TAG_REP(md_tag_of(xo));
          const long long h0 = go->halfL_bits[0], h1 = go->halfL_bits[1],
                          h2 = go->halfL_bits[2];
          if (EV) {
            shx = md_abs_gt(dx, h0) ? copysign(go->L[0], dx) : 0.0;
            shy = md_abs_gt(dy, h1) ? copysign(go->L[1], dy) : 0.0;
            shz = md_abs_gt(dz, h2) ? copysign(go->L[2], dz) : 0.0;
          }
          dx = md_min_image(dx, go->L[0], h0);
          dy = md_min_image(dy, go->L[1], h1);
          dz = md_min_image(dz, go->L[2], h2);
        }
        const double r2 = md_r2(dx, dy, dz);
        const int to = MD_TAG_TYPE(md_tag_of(xo));
        const PairCoef& c = SINGLE ? a.c1 : sc[to * a.nt + md_type_of(xj)];
        if (md_lt_pos(r2, COUL ? c.cutmax_bits : c.cutsq_bits)) {
          double r2inv, r6inv, fpair, qr = 0.0;
          if (COUL) {  // Eq. 1 below rc, plus qq / r below rc_coul (selects, no branch)
            const double rinv = md_rsqrt(r2);
            r2inv = rinv * rinv;
            r6inv = r2inv * r2inv * r2inv;
            const double flj = r6inv * (c.lj1 * r6inv - c.lj2) * r2inv;
            qr = c.qq * rinv;
            qr = md_lt_pos(r2, c.cutsq_coul_bits) ? qr : 0.0;
            fpair = __fma_rn(qr, r2inv, md_lt_pos(r2, c.cutsq_bits) ? flj : 0.0);
          } else {
            r2inv = md_rcp(r2);
            r6inv = r2inv * r2inv * r2inv;
            fpair = r6inv * (c.lj1 * r6inv - c.lj2) * r2inv;
          }
          const double gx = fpair * dx, gy = fpair * dy, gz = fpair * dz;
          const int64_t io = tile * MD_BLOCK + w * 32 + o;
          long long qx = 0, qy = 0, qz = 0;
          if (FIX && (md_fix(gx, ex_lim, qx) & md_fix(gy, ex_lim, qy) &
                      md_fix(gz, ex_lim, qz))) {
            atomicAdd(&sown[FIX ? w : 0][0][o], (unsigned long long)(-qx));
            atomicAdd(&sown[FIX ? w : 0][1][o], (unsigned long long)(-qy));
            atomicAdd(&sown[FIX ? w : 0][2][o], (unsigned long long)(-qz));
            if (HALF) {
              atomicAdd(a.fix + j, (unsigned long long)qx);
              atomicAdd(a.fix + n + j, (unsigned long long)qy);
              atomicAdd(a.fix + 2 * n + j, (unsigned long long)qz);
            }
          } else {
            atomicAdd(a.f + io, md_neg(gx));
            atomicAdd(a.f + n + io, md_neg(gy));
            atomicAdd(a.f + 2 * n + io, md_neg(gz));
            if (HALF) {
              atomicAdd(a.f + j, gx);
              atomicAdd(a.f + n + j, gy);
              atomicAdd(a.f + 2 * n + j, gz);
            }
          }
          if (EV) {  // the virial is x (x) F per atom afterwards, less the image terms
            const bool img = (shx != 0.0) | (shy != 0.0) | (shz != 0.0);
            auto energy = [&]() {
              if (S2) return -0.5 * c.lj4 * r6inv;
              double en = r6inv * (c.lj3 * r6inv - c.lj4);
              if (COUL) en = (md_lt_pos(r2, c.cutsq_bits) ? en : 0.0) + qr;
              return en;
            };
            if (uni) {
              if (S2)
                s6 += r6inv;
              else
                e0 += energy();
              npair++;
              if (img) {  // this lane's column: no other lane writes it
                double* m = &sev[w][0][lane];
                m[1 * 32] = __fma_rn(-shx, gx, m[1 * 32]);
                m[2 * 32] = __fma_rn(-shy, gy, m[2 * 32]);
                m[3 * 32] = __fma_rn(-shz, gz, m[3 * 32]);
                m[4 * 32] = __fma_rn(-shx, gy, m[4 * 32]);
                m[5 * 32] = __fma_rn(-shx, gz, m[5 * 32]);
                m[6 * 32] = __fma_rn(-shy, gz, m[6 * 32]);
              }
            } else {
              atomicAdd(&sev[w][0][o], evw * energy());
              atomicAdd(&sev[w][7][o], evw);
              if (img) {
                atomicAdd(&sev[w][1][o], -evw * shx * gx);
                atomicAdd(&sev[w][2][o], -evw * shy * gy);
                atomicAdd(&sev[w][3][o], -evw * shz * gz);
                atomicAdd(&sev[w][4][o], -evw * shx * gy);
                atomicAdd(&sev[w][5][o], -evw * shx * gz);
                atomicAdd(&sev[w][6][o], -evw * shy * gz);
              }
            }
          }
        }
      }
      head[Q] += take;
      __syncwarp();
    };
    const std::integral_constant<int, 0> q0{};
    const std::integral_constant<int, 1> q1{};

    // phase 1: U list entries per lane per round, their loads in
    // flight together; each entry's survivors are pushed (and full queues
    // drained) in turn, so fewer than 32 entries wait before each push
    static_assert(U == 1 || (U == 2 && FIX && !EV && !COUL), "two entries: force-only, fixed point");
    for (;;) {
      if (!__any_sync(0xffffffffu, q < cnt)) break;
      int jv[U];
      float4 hv[U];
  #pragma unroll
      for (int u = 0; u < U; u++) {
        jv[u] = 0;
        if (q + u < cnt)
          jv[u] = __ldcs(q + u < nin ? row + (int64_t)(q + u) * 32
                                     : skin - (int64_t)(q + u - nin) * 32);
      }
  #pragma unroll
      for (int u = 0; u < U; u++)
        hv[u] = q + u < cnt ? __ldg(&a.xs[jv[u]].hi) : make_float4(0.f, 0.f, 0.f, 0.f);
  #pragma unroll
      for (int u = 0; u < U; u++) {
        const bool has = q + u < cnt;
        const int j = jv[u];
        const float4 hj = hv[u];
        bool cand = false, wrap = false;
        if (has) {
          float dx = hj.x - hi.x, dy = hj.y - hi.y, dz = hj.z - hi.z;
          wrap = (fabsf(dx) > hm0) | (fabsf(dy) > hm1) | (fabsf(dz) > hm2);
          if (INTX) wrap |= own_off | ((__float_as_int(hj.w) & MD_TAG_OFFGRID) != 0);
          dx = fabsf(dx) > hf0 ? dx - copysignf(Lf0, dx) : dx;
          dy = fabsf(dy) > hf1 ? dy - copysignf(Lf1, dy) : dy;
          dz = fabsf(dz) > hf2 ? dz - copysignf(Lf2, dz) : dz;
          const float r2f = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
          const float cut =
              SINGLE ? cut_hi1 : scut[ti * a.nt + MD_TAG_TYPE(__float_as_int(hj.w))];
          cand = r2f <= cut;
        }
        const unsigned lt = (1u << lane) - 1u;
        const unsigned b0 = __ballot_sync(0xffffffffu, cand && !wrap);
        const unsigned b1 = __ballot_sync(0xffffffffu, cand && wrap);
        if (cand) {
          const int Q = wrap ? 1 : 0;
          const unsigned slot = tail[Q] + __popc((wrap ? b1 : b0) & lt);
          qj[Q][w][slot % MD_Q_CAP] = j;
          qo[Q][w][slot % MD_Q_CAP] = (unsigned char)lane;
        }
        tail[0] += __popc(b0);
        tail[1] += __popc(b1);
        __syncwarp();
        if (tail[0] - head[0] >= 32) drain(q0, 32);
        if (tail[1] - head[1] >= 32) drain(q1, 32);
      }
      q += U;
    }
    while (tail[0] != head[0]) drain(q0, tail[0] - head[0] < 32 ? tail[0] - head[0] : 32);
    while (tail[1] != head[1]) drain(q1, tail[1] - head[1] < 32 ? tail[1] - head[1] : 32);
    __syncwarp();
    if (FIX && active) {  // the owner's share: one reduction per component
  #pragma unroll
      for (int k = 0; k < 3; k++) {
        const unsigned long long q = sown[FIX ? w : 0][k][lane];
        if (q) atomicAdd(a.fix + k * n + i, q);
      }
    }

    if (EV) {
      const int slot = (int)(((int64_t)tile * (MD_BLOCK / 32) + w) % a.ev_spread);
      double ev[8];
      if (uni) {  // every lane's sums belong to box rep0
        ev[0] = S2 ? -0.5 * a.c1.lj4 * s6 : e0;
  #pragma unroll
        for (int k = 1; k < 7; k++) ev[k] = sev[w][k][lane];
  #pragma unroll
        for (int k = 0; k < 7; k++) ev[k] *= evw;
        ev[7] = evw * (double)npair;
        md_warp_add_rep<8>(ev, rep0, a.ev, a.ev_spread, slot);
      } else {
  #pragma unroll
        for (int k = 0; k < 8; k++) ev[k] = sev[w][k][lane];
        md_warp_add_rep<8>(ev, active ? rep_i : -1, a.ev, a.ev_spread, slot);
      }
    }
  }
}

// Resident blocks per SM the register allocation must allow.
// The energy/virial launches: at 4M atoms (fcc liquid) 7, 8 and 10 blocks
// (72, 64 and 48 registers; 48 spills a few words) measured 3.49, 3.37 and
// 3.60 ms per half-list launch and 5.80, 5.60 and 5.38 ms per full-list one.
constexpr int md_pair_q_minb(bool half, bool ev, bool fix, bool coul, int u) {
  return ev ? (half ? 8 : 10)
            : ((fix && !coul) ? (u == 2 ? MD_Q_MINB_INT2 : MD_Q_MINB_INT) : MD_Q_MINB);
}

template <bool HALF, bool EV, bool SINGLE, bool FIX, bool COUL, int U>
__global__ void __launch_bounds__(MD_BLOCK, md_pair_q_minb(HALF, EV, FIX, COUL, U))
    k_pair_q(const PairArgs a, const float cut_hi1, const float* __restrict__ cut_hi_tab) {
  md_pair_q_tiles<HALF, EV, SINGLE, FIX, COUL, U>(a, cut_hi1, cut_hi_tab);
}

template <bool HALF, bool EV, bool SINGLE, bool FIX, bool COUL, int U = 1>
cudaError_t md_pair_q_launch5(const PairArgs& a, float cut1, const float* cut_tab,
                              unsigned blocks, cudaStream_t s, int carve) {
  int occ = 1;
  cudaError_t e =
      md_prepare_kernel((const void*)k_pair_q<HALF, EV, SINGLE, FIX, COUL, U>, carve, &occ);
  if (e != cudaSuccess) return e;
  if (a.tile_ctr) {
    const unsigned cap = (unsigned)(a.nslots * occ);
    if (blocks > cap) blocks = cap;
  }
  k_pair_q<HALF, EV, SINGLE, FIX, COUL, U><<<blocks, MD_BLOCK, 0, s>>>(a, cut1, cut_tab);
  return cudaGetLastError();
}

// qu: list entries per phase-1 round (2 only in force-only fixed-point
// launches; 1 otherwise)
template <bool FIX, bool COUL>
cudaError_t md_pair_q_launch_t(const PairArgs& a, bool half, bool ev, bool single, float cut1,
                               const float* cut_tab, unsigned blocks, cudaStream_t s,
                               int carve, int qu = 1) {
  if constexpr (FIX && !COUL) {
    if (!ev && qu == 2) {
      if (half)
        return single ? md_pair_q_launch5<true, false, true, FIX, COUL, 2>(a, cut1, cut_tab, blocks, s, carve)
                      : md_pair_q_launch5<true, false, false, FIX, COUL, 2>(a, cut1, cut_tab, blocks, s, carve);
      return single ? md_pair_q_launch5<false, false, true, FIX, COUL, 2>(a, cut1, cut_tab, blocks, s, carve)
                    : md_pair_q_launch5<false, false, false, FIX, COUL, 2>(a, cut1, cut_tab, blocks, s, carve);
    }
  }
  if (half) {
    if (ev)
      return single ? md_pair_q_launch5<true, true, true, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve)
                    : md_pair_q_launch5<true, true, false, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve);
    return single ? md_pair_q_launch5<true, false, true, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve)
                  : md_pair_q_launch5<true, false, false, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve);
  }
  if (ev)
    return single ? md_pair_q_launch5<false, true, true, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve)
                  : md_pair_q_launch5<false, true, false, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve);
  return single ? md_pair_q_launch5<false, false, true, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve)
                : md_pair_q_launch5<false, false, false, FIX, COUL>(a, cut1, cut_tab, blocks, s, carve);
}

// FP64 reductions (md_pair_fp64.cu), fixed-point reductions (md_pair_fix.cu),
// and the lj/cut/coul/cut style with either (md_pair_coul.cu)
cudaError_t md_pair_q_launch(const PairArgs& a, bool half, bool ev, bool single, float cut1,
                             const float* cut_tab, unsigned blocks, cudaStream_t s, int carve);
cudaError_t md_pair_q_fix_launch(const PairArgs& a, bool half, bool ev, bool single, float cut1,
                                 const float* cut_tab, unsigned blocks, cudaStream_t s,
                                 int carve, int qu);
cudaError_t md_pair_q_coul_launch(const PairArgs& a, bool fix, bool half, bool ev, bool single,
                                  float cut1, const float* cut_tab, unsigned blocks,
                                  cudaStream_t s, int carve);
