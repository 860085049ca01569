// md_neigh.cu -- cell binning by counting sort and prefix scan, and the
// neighbor-list build with skin (arXiv 2508.13523, Sec. 4: a list built and
// periodically updated; Sec. 4.1: half lists with each pair once, full lists
// with each pair in both atoms' lists; App. B: 64-bit row offsets with
// 32-bit column indices).
//
// Rebuild pipeline, all on the context's stream:
//   k_wrap_bin    wrap x into [0,L) (x - L*floor(x/L), L -> 0), cell index,
//                 histogram with atomics (rank of each atom in its cell)
//   scan          exclusive prefix sum of the histogram -> cell starts
//   k_scatter     perm[start[c] + rank] = atom
//   k_cell_sort   sort each cell's slice of perm ascending: a stable,
//                 deterministic counting sort
//   k_gather      permuted copies of x, v, f, id, cell; copied back so that
//                 every pointer stays fixed (CUDA graphs capture them)
//   k_split_snapshot  double-float split of x (xs, md_split) and the build
//                 snapshot (xb)
//   k_build       27-cell stencil (one cell along an axis with < 3 cells);
//                 FP32 test with certified bounds, FP64 only inside the
//                 band where FP32 cannot decide; writes tiled lists
// The host then reads the largest count; if it exceeds the capacity the
// list storage grows and k_build runs again.
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_device.cuh"
#include "md_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// x - L*floor(x/L) with correctly rounded division and product (no
// contraction); a result equal to L becomes 0.
__device__ __forceinline__ double wrap1(double x, double L) {
  double q = floor(__ddiv_rn(x, L));
  double w = __dsub_rn(x, __dmul_rn(L, q));
  return (w == L) ? 0.0 : w;
}

__device__ __forceinline__ int cell_coord(double x, double cinv, int nc) {
  int c = (int)(x * cinv);  // x >= 0 after the wrap: truncation is floor
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_wrap_bin(double4_32a* __restrict__ x4, int64_t n,
                           const RepGeo* __restrict__ rep, int32_t* __restrict__ cell,
                           int32_t* __restrict__ cnt, int32_t* __restrict__ rank) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4_32a p = x4[i];
  const RepGeo& g = rep[MD_TAG_REP(md_tag_of(p))];
  p.x = wrap1(p.x, g.L[0]);
  p.y = wrap1(p.y, g.L[1]);
  p.z = wrap1(p.z, g.L[2]);
  x4[i] = p;
  int cx = cell_coord(p.x, g.cinv[0], g.nc[0]);
  int cy = cell_coord(p.y, g.cinv[1], g.nc[1]);
  int cz = cell_coord(p.z, g.cinv[2], g.nc[2]);
  int c = md_cell_index(g, cx, cy, cz);
  cell[i] = c;
  rank[i] = atomicAdd(&cnt[c], 1);
}

// ---- exclusive scan (three passes, block sums kept in int64) ---------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += u;
  }
  return v;
}

// Exclusive scan of the SCAN_TILE items owned by this block; returns the
// block total to thread 0 via *total.
template <typename TIN, typename TOUT>
__device__ void block_scan_tile(const TIN* in, TOUT* out, int64_t n, int64_t base,
                                TOUT carry, int64_t* total) {
  __shared__ int64_t wsum[SCAN_THREADS / 32];
  TOUT v[SCAN_ITEMS];
  TOUT s = 0;
  int64_t first = base + (int64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t idx = first + k;
    v[k] = idx < n ? (TOUT)in[idx] : (TOUT)0;
    s += v[k];
  }
  int64_t incl = warp_incl_scan<int64_t>((int64_t)s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int64_t woff = 0, btot = 0;
#pragma unroll
  for (int w = 0; w < SCAN_THREADS / 32; w++) {
    if (w < warp) woff += wsum[w];
    btot += wsum[w];
  }
  TOUT run = carry + (TOUT)(woff + incl - (int64_t)s);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t idx = first + k;
    if (idx < n) out[idx] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) *total = btot;
  __syncthreads();
}

template <typename TOUT>
__global__ void k_scan_tiles(const int32_t* __restrict__ in, TOUT* __restrict__ out,
                             int64_t n, int64_t* __restrict__ tile_sums) {
  int64_t t;
  block_scan_tile<int32_t, TOUT>(in, out, n, (int64_t)blockIdx.x * SCAN_TILE, (TOUT)0, &t);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
}

// One block: exclusive scan of the tile sums in place, any count.
__global__ void k_scan_top(int64_t* __restrict__ sums, int64_t m) {
  __shared__ int64_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < m; base += SCAN_TILE) {
    int64_t t;
    int64_t carry = carry_s;
    block_scan_tile<int64_t, int64_t>(sums, sums, m, base, carry, &t);
    if (threadIdx.x == 0) carry_s = carry + t;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[m] = carry_s;
}

template <typename TOUT>
__global__ void k_scan_add(TOUT* __restrict__ out, int64_t n,
                           const int64_t* __restrict__ tile_off) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += (TOUT)tile_off[i / SCAN_TILE];
  if (i == 0) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    out[n] = (TOUT)tile_off[tiles];
  }
}

__global__ void k_scatter(const int32_t* __restrict__ cell, const int32_t* __restrict__ rank,
                          const int32_t* __restrict__ start, int32_t* __restrict__ perm,
                          int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  perm[start[cell[i]] + rank[i]] = (int32_t)i;
}

// Insertion sort of each cell's slice (cells hold tens of atoms).
__global__ void k_cell_sort(int32_t* __restrict__ perm, const int32_t* __restrict__ start,
                            int64_t ncell) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  int b = start[c], e = start[c + 1];
  for (int k = b + 1; k < e; k++) {
    int32_t key = perm[k];
    int q = k - 1;
    while (q >= b && perm[q] > key) {
      perm[q + 1] = perm[q];
      q--;
    }
    perm[q + 1] = key;
  }
}

__global__ void k_gather(const int32_t* __restrict__ perm, int64_t n,
                         const double4_32a* __restrict__ x4, const double* __restrict__ v,
                         const double* __restrict__ f, const int32_t* __restrict__ id,
                         const int32_t* __restrict__ cell, double4_32a* __restrict__ x4n,
                         double* __restrict__ vn, double* __restrict__ fn,
                         int32_t* __restrict__ idn, int32_t* __restrict__ celln) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t o = perm[p];
  x4n[p] = x4[o];
  vn[p] = v[o];
  vn[n + p] = v[n + o];
  vn[2 * n + p] = v[2 * n + o];
  fn[p] = f[o];
  fn[n + p] = f[n + o];
  fn[2 * n + p] = f[2 * n + o];
  idn[p] = id[o];
  celln[p] = cell[o];
}

__global__ void k_split_snapshot(const double4_32a* __restrict__ x4, XSplit* __restrict__ xs,
                                 XSplit* __restrict__ xb, XFix* __restrict__ xq, int64_t n,
                                 const XGrid gr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  md_store_pos(x4[i], gr, xs, xq, i, xb);
}

// FP32 minimum image of one component (float positions in [0, L]).
__device__ __forceinline__ float min_image_f(float d, float L, float halfL) {
  return fabsf(d) > halfL ? d - copysignf(L, d) : d;
}

// Neighbor build, one thread per atom (cell-sorted order).  Candidate j is
// kept iff its FP64 minimum-image r2 < rlist2, where
//   r2 = fma(dz,dz, fma(dy,dy, dx*dx)),  d = x_j - x_i - L*rint((x_j-x_i)/L).
// The FP32 distance of the hi parts decides whenever it is outside
// [lo2f, hi2f]; those bounds are certified on the host from the FP32
// rounding of positions and arithmetic, so the kept set is exactly the FP64
// one.  Half list: only the pairs i owns (md_owns), each pair once.
// Row order: pairs with r2f < rc^2 of their type pair ("inner") from the
// front, the rest ("skin") from the back, so that in the force kernel the
// inner loop is almost branch-free and the skin loop mostly skips the force.
template <bool HALF>
__global__ void __launch_bounds__(MD_BLOCK)
    k_build(const double4_32a* __restrict__ x4, const XSplit* __restrict__ xs,
            const int32_t* __restrict__ cell, const int32_t* __restrict__ start, int64_t n,
            Geo gg, const RepGeo* __restrict__ rep, int32_t* __restrict__ numneigh,
            int32_t* __restrict__ nbr, int maxneigh, unsigned int* __restrict__ maxcount) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 hi = xs[i].hi;
  const int tag = __float_as_int(hi.w);
  const int ti = MD_TAG_TYPE(tag);
  const RepGeo& g = rep[MD_TAG_REP(tag)];  // fields read on use (fewer registers)
  int cx, cy, cz;
  md_cell_coords(g, cell[i], cx, cy, cz);
  int32_t* out = nbr + (i >> 5) * (int64_t)maxneigh * 32 + (i & 31);
  int nin = 0, nsk = 0;  // entries written (nin + nsk <= maxneigh)
  int total = 0;         // entries found
  int cand = -1;         // atoms in the stencil's cells other than i
  double4_32a xi;
  bool have_xi = false;
  const int ii = (int)i;

  // candidate j at FP32 separation (dx, dy, dz) of the hi parts, nearest image
  auto consider = [&](int j, float dx, float dy, float dz, float wj) {
    const float r2f = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
    if (r2f > gg.hi2f) return;
    bool keep = true;
    if (r2f >= gg.lo2f) {  // undecided in FP32: the exact FP64 test
      if (!have_xi) {
        xi = x4[i];
        have_xi = true;
      }
      const double4_32a xj = x4[j];
      const double ex = md_min_image(__dsub_rn(xj.x, xi.x), g.L[0], g.halfL_bits[0]);
      const double ey = md_min_image(__dsub_rn(xj.y, xi.y), g.L[1], g.halfL_bits[1]);
      const double ez = md_min_image(__dsub_rn(xj.z, xi.z), g.L[2], g.halfL_bits[2]);
      keep = md_lt_pos(md_r2(ex, ey, ez), gg.rlist2_bits);
    }
    if (keep) {
      const bool inner = r2f < gg.cutsqf[ti * gg.nt + MD_TAG_TYPE(__float_as_int(wj))];
      if (nin + nsk < maxneigh) {
        if (inner)
          out[(int64_t)(nin++) * 32] = j;
        else
          out[(int64_t)(maxneigh - 1 - nsk++) * 32] = j;
      }
      total++;
    }
  };

  if (g.nc[0] >= 3 && g.nc[1] >= 3 && g.nc[2] >= 3) {
    // Every axis has >= 3 cells of side >= rlist: each stencil cell is one
    // periodic image, so the image shift (0 or -+L) is fixed per cell and
    // added to the separation exactly as the per-candidate minimum image
    // would (the same two FP32 roundings).  Cells along z that are adjacent
    // in the sorted order and share the shift are scanned as one run.
    // Half list: i owns j < i iff i + j is odd and j > i iff i + j is even
    // (md_owns), so each run is walked with stride 2 on the owned parity.
    auto run = [&](int b, int e, float sx, float sy, float sz) {
      auto visit = [&](int j) {
        const float4 hj = __ldg(&xs[j].hi);
        consider(j, __fadd_rn(__fsub_rn(hj.x, hi.x), sx), __fadd_rn(__fsub_rn(hj.y, hi.y), sy),
                 __fadd_rn(__fsub_rn(hj.z, hi.z), sz), hj.w);
      };
      // one loop per run, so that lanes of the same cell (same run, different
      // i) run the same number of iterations
      if (HALF) {
        const int le = min(e, ii);                   // owned j < i: parity of i + 1
        const int j0 = b + ((b ^ (ii + 1)) & 1);
        const int nlo = le > j0 ? (le - j0 + 1) >> 1 : 0;
        const int hb = max(b, ii + 1);               // owned j > i: parity of i
        const int j1 = hb + ((hb ^ ii) & 1);
        const int nhi = e > j1 ? (e - j1 + 1) >> 1 : 0;
        for (int t = 0; t < nlo + nhi; t++) visit(t < nlo ? j0 + 2 * t : j1 + 2 * (t - nlo));
      } else {
        const bool self = ii >= b && ii < e;
        const int cnt = e - b - (self ? 1 : 0);
        for (int t = 0; t < cnt; t++) visit(b + t + ((self && b + t >= ii) ? 1 : 0));
      }
    };
    for (int ox = -1; ox <= 1; ox++) {
      int qx = cx + ox;
      float sx = 0.f;
      if (qx < 0) { qx += g.nc[0]; sx = -g.Lf[0]; }
      else if (qx >= g.nc[0]) { qx -= g.nc[0]; sx = g.Lf[0]; }
      for (int oy = -1; oy <= 1; oy++) {
        int qy = cy + oy;
        float sy = 0.f;
        if (qy < 0) { qy += g.nc[1]; sy = -g.Lf[1]; }
        else if (qy >= g.nc[1]) { qy -= g.nc[1]; sy = g.Lf[1]; }
        int rb = 0, re = 0;
        float rs = 0.f;
        bool open = false;
        for (int oz = -1; oz <= 1; oz++) {
          int qz = cz + oz;
          float sz = 0.f;
          if (qz < 0) { qz += g.nc[2]; sz = -g.Lf[2]; }
          else if (qz >= g.nc[2]) { qz -= g.nc[2]; sz = g.Lf[2]; }
          const int q = md_cell_index(g, qx, qy, qz);
          const int b = start[q], e = start[q + 1];
          cand += e - b;
          if (open && b == re && sz == rs) {
            re = e;
          } else {
            if (open) run(rb, re, sx, sy, rs);
            rb = b;
            re = e;
            rs = sz;
            open = true;
          }
        }
        run(rb, re, sx, sy, rs);
      }
    }
  } else {
    // some axis has a single cell: per-candidate minimum image
    for (int ox = g.lo[0]; ox <= g.hi[0]; ox++) {
      int qx = cx + ox;
      qx = qx < 0 ? qx + g.nc[0] : (qx >= g.nc[0] ? qx - g.nc[0] : qx);
      for (int oy = g.lo[1]; oy <= g.hi[1]; oy++) {
        int qy = cy + oy;
        qy = qy < 0 ? qy + g.nc[1] : (qy >= g.nc[1] ? qy - g.nc[1] : qy);
        for (int oz = g.lo[2]; oz <= g.hi[2]; oz++) {
          int qz = cz + oz;
          qz = qz < 0 ? qz + g.nc[2] : (qz >= g.nc[2] ? qz - g.nc[2] : qz);
          const int q = md_cell_index(g, qx, qy, qz);
          const int b = start[q], e = start[q + 1];
          cand += e - b;
          for (int j = b; j < e; j++) {
            if (j == ii) continue;
            if (HALF && !md_owns(ii, j)) continue;
            const float4 hj = __ldg(&xs[j].hi);
            consider(j, min_image_f(hj.x - hi.x, g.Lf[0], g.halfLf[0]),
                     min_image_f(hj.y - hi.y, g.Lf[1], g.halfLf[1]),
                     min_image_f(hj.z - hi.z, g.Lf[2], g.halfLf[2]), hj.w);
          }
        }
      }
    }
  }
  // on overflow the rows are incomplete (but in bounds); the host sees
  // total > maxneigh, grows the list and rebuilds
  numneigh[i] = nin;
  numneigh[n + i] = nsk;
  atomicMax(maxcount, (unsigned int)total);
  // every pair of atom i in any list built now joins i to a stencil
  // candidate, so cand bounds the force contributions atom i receives in
  // one pair launch (the range of the fixed-point accumulators)
  atomicMax(maxcount + 1, (unsigned int)cand);
}

__global__ void k_sum_counts(const int32_t* __restrict__ numneigh, int64_t n,
                             unsigned long long* __restrict__ total) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = i < n ? (unsigned long long)numneigh[i] : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// Row length of each caller-order atom.
__global__ void k_csr_counts(const int32_t* __restrict__ numneigh, const int32_t* __restrict__ id,
                             int64_t n, int32_t* __restrict__ cnt_orig) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  cnt_orig[id[p]] = numneigh[p] + numneigh[n + p];
}

__global__ void k_csr_fill(const int32_t* __restrict__ numneigh, const int32_t* __restrict__ nbr,
                           const int32_t* __restrict__ id, int64_t n, int maxneigh,
                           const int64_t* __restrict__ offsets, int32_t* __restrict__ idx) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t* row = nbr + (p >> 5) * (int64_t)maxneigh * 32 + (p & 31);
  int64_t o = offsets[id[p]];
  const int nin = numneigh[p], nsk = numneigh[n + p];
  for (int k = 0; k < nin; k++) idx[o + k] = id[row[(int64_t)k * 32]];
  for (int k = 0; k < nsk; k++) idx[o + nin + k] = id[row[(int64_t)(maxneigh - 1 - k) * 32]];
}

}  // namespace

// ---- host side -----------------------------------------------------------------

static int scan_tmp_reserve(md_ctx* c, int64_t n) {
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE + 1;
  if (tiles <= c->scan_tmp_n) return MD_OK;
  if (c->scan_tmp) cudaFree(c->scan_tmp);
  c->scan_tmp = nullptr;
  c->scan_tmp_n = 0;
  if (cudaMalloc(&c->scan_tmp, sizeof(int64_t) * tiles) != cudaSuccess) return MD_ENOMEM;
  c->scan_tmp_n = tiles;
  return MD_OK;
}

template <typename TOUT>
static int scan_impl(md_ctx* c, const int32_t* in, TOUT* out, int64_t n) {
  MD_TRY(scan_tmp_reserve(c, n));
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles > 0) {
    k_scan_tiles<TOUT><<<(unsigned)tiles, SCAN_THREADS, 0, c->stream>>>(in, out, n, c->scan_tmp);
    c->launches++;
  }
  k_scan_top<<<1, SCAN_THREADS, 0, c->stream>>>(c->scan_tmp, tiles);
  k_scan_add<TOUT><<<(unsigned)md_blocks(n > 0 ? n : 1), MD_BLOCK, 0, c->stream>>>(out, n,
                                                                                   c->scan_tmp);
  c->launches += 2;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_scan_i32(md_ctx* c, const int32_t* in, int32_t* out, int64_t n) {
  return scan_impl<int32_t>(c, in, out, n);
}
int md_scan_i64(md_ctx* c, const int32_t* in, int64_t* out, int64_t n) {
  return scan_impl<int64_t>(c, in, out, n);
}

static int grow_list(md_ctx* c, int new_max) {
  int64_t tiles = (c->n + 31) / 32;
  int64_t need = tiles * 32 * (int64_t)new_max;
  if (need > c->nbr_alloc) {
    if (c->nbr) cudaFree(c->nbr);
    c->nbr = nullptr;
    c->nbr_alloc = 0;
    if (cudaMalloc(&c->nbr, sizeof(int32_t) * need) != cudaSuccess) return MD_ENOMEM;
    c->nbr_alloc = need;
  }
  c->maxneigh = new_max;
  md_drop_graphs(c);  // captured graphs hold the old pointer and capacity
  return MD_OK;
}

void md_drop_graphs(md_ctx* c) {
  if (!c->graphs) return;
  for (auto& kv : *c->graphs) cudaGraphExecDestroy(kv.second.first);
  c->graphs->clear();
}

static int launch_build(md_ctx* c) {
  MD_CUDA(cudaMemsetAsync(c->dmax + 1, 0, 2 * sizeof(unsigned int), c->stream));
  unsigned nb = (unsigned)md_blocks(c->n);
  if (c->list_kind == MD_LIST_HALF)
    k_build<true><<<nb, MD_BLOCK, 0, c->stream>>>(c->x4, c->xs, c->cell, c->start, c->n,
                                                  c->geo, c->rep, c->numneigh, c->nbr,
                                                  c->maxneigh, c->dmax + 1);
  else
    k_build<false><<<nb, MD_BLOCK, 0, c->stream>>>(c->x4, c->xs, c->cell, c->start, c->n,
                                                   c->geo, c->rep, c->numneigh, c->nbr,
                                                   c->maxneigh, c->dmax + 1);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}

int md_rebuild(md_ctx* c) {
  const int64_t n = c->n;
  const unsigned nb = (unsigned)md_blocks(n);
  cudaStream_t s = c->stream;
  // displacement since the previous build: dangerous if > skin/2
  MD_CUDA(cudaMemcpyAsync(c->h_pinned + 8, c->dmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  MD_CUDA(cudaMemcpyAsync(c->h_pinned + 14, c->dmax + 5, sizeof(unsigned int),
                          cudaMemcpyDeviceToHost, s));
  MD_CUDA(cudaMemsetAsync(c->cnt, 0, sizeof(int32_t) * c->ncell, s));
  k_wrap_bin<<<nb, MD_BLOCK, 0, s>>>(c->x4, n, c->rep, c->cell, c->cnt, c->rank);
  c->launches++;
  MD_TRY(md_scan_i32(c, c->cnt, c->start, c->ncell));
  k_scatter<<<nb, MD_BLOCK, 0, s>>>(c->cell, c->rank, c->start, c->perm, n);
  k_cell_sort<<<(unsigned)md_blocks(c->ncell), MD_BLOCK, 0, s>>>(c->perm, c->start, c->ncell);
  k_gather<<<nb, MD_BLOCK, 0, s>>>(c->perm, n, c->x4, c->v, c->f, c->id, c->cell, c->x4_alt,
                                   c->v_alt, c->f_alt, c->id_alt, c->cell_alt);
  c->launches += 3;
  MD_CUDA(cudaGetLastError());
  MD_CUDA(cudaMemcpyAsync(c->x4, c->x4_alt, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, s));
  MD_CUDA(cudaMemcpyAsync(c->v, c->v_alt, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
  MD_CUDA(cudaMemcpyAsync(c->f, c->f_alt, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
  MD_CUDA(cudaMemcpyAsync(c->id, c->id_alt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  MD_CUDA(cudaMemcpyAsync(c->cell, c->cell_alt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  k_split_snapshot<<<nb, MD_BLOCK, 0, s>>>(c->x4, c->xs, c->xb, c->xq, n, c->xgrid);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  MD_CUDA(cudaMemsetAsync(c->dmax, 0, sizeof(unsigned int), s));
  for (int attempt = 0; attempt < 4; attempt++) {
    MD_TRY(launch_build(c));
    MD_CUDA(cudaMemcpyAsync(c->h_pinned + 9, c->dmax + 1, sizeof(unsigned int),
                            cudaMemcpyDeviceToHost, s));
    MD_CUDA(cudaStreamSynchronize(s));
    MD_TRY(md_barrier_status(c));
    unsigned int mc;
    memcpy(&mc, (const char*)(c->h_pinned + 9), sizeof(mc));
    c->max_count = (int32_t)mc;
    if ((int)mc <= c->maxneigh) {
      unsigned int disp_bits;
      memcpy(&disp_bits, (const char*)(c->h_pinned + 8), sizeof(disp_bits));
      float disp2;
      memcpy(&disp2, &disp_bits, sizeof(disp2));
      double half = 0.5 * c->skin;
      // with check_disp the list is rebuilt before any force evaluation at
      // positions beyond skin/2, so no build is dangerous
      if (c->builds > 0 && !c->check_disp && (double)disp2 > half * half) c->dangerous++;
      c->builds++;
      return MD_OK;
    }
    int grown = (int)(mc + mc / 8 + 8);
    grown = (grown + 7) & ~7;
    MD_TRY(grow_list(c, grown));
  }
  return MD_ENEIGH;
}

int md_list_entries(md_ctx* c, int64_t* total) {
  unsigned long long* d = reinterpret_cast<unsigned long long*>(c->i64_tmp);
  MD_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), c->stream));
  k_sum_counts<<<(unsigned)md_blocks(2 * c->n), MD_BLOCK, 0, c->stream>>>(c->numneigh, 2 * c->n, d);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  MD_CUDA(cudaMemcpyAsync(c->h_pinned + 10, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  unsigned long long t;
  memcpy(&t, (const char*)(c->h_pinned + 10), sizeof(t));
  *total = (int64_t)t;
  return MD_OK;
}

int md_list_to_csr(md_ctx* c, int64_t* offsets, int32_t* idx) {
  const unsigned nb = (unsigned)md_blocks(c->n);
  int32_t* cnt_orig = c->rank;  // rebuild scratch, free between rebuilds
  k_csr_counts<<<nb, MD_BLOCK, 0, c->stream>>>(c->numneigh, c->id, c->n, cnt_orig);
  c->launches++;
  MD_TRY(md_scan_i64(c, cnt_orig, offsets, c->n));
  k_csr_fill<<<nb, MD_BLOCK, 0, c->stream>>>(c->numneigh, c->nbr, c->id, c->n, c->maxneigh,
                                             offsets, idx);
  c->launches++;
  MD_CUDA(cudaGetLastError());
  return MD_OK;
}
