// md_capi.cu -- the C ABI of libmd.so (declared in include/md.h): context
// lifetime for one box or a batch of replicas, parameter checks, the step
// driver with CUDA-graph segments, energies, statistics and the
// threads-per-atom tuner.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "md_device.cuh"
#include "md_integrate.cuh"
#include "md_internal.cuh"
#include "md_pair.cuh"
#include "md_pair_q.cuh"

// md_step_fused.cu
cudaError_t md_step_fused_launch(const IntArgs& ia, const PairArgs& a, int mode, bool half,
                                 bool single, float cut1, const float* cut_tab,
                                 unsigned int* bar, unsigned int* err, cudaStream_t s);

int md_cuda_fail(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? MD_ENOMEM : MD_ECUDA;
}

cudaError_t md_prepare_kernel(const void* kernel, int carve, int* occ) {
  // (kernel, device) -> (carveout applied, -1 none; resident blocks per SM)
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, std::pair<int, int>> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({kernel, dev});
  if (it == cache.end()) it = cache.emplace(std::make_pair(kernel, dev), std::make_pair(-1, 0)).first;
  std::pair<int, int>& st = it->second;
  if (carve >= 0 && carve != st.first) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    if (e != cudaSuccess) return e;
    st.first = carve;
    st.second = 0;
  }
  if (st.second == 0) {
    int o = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, MD_BLOCK, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      o = 1;
    }
    st.second = o < 1 ? 1 : o;
  }
  *occ = st.second;
  return cudaSuccess;
}

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

// Largest cell count along an axis with cell edge >= rlist, with a guard of
// 1e-9 L so that rounding in the cell index can never lose a pair; an axis
// with fewer than 3 cells gets 1 (the stencil then covers it once).
int cells_along(double L, double rlist) {
  int nc = (int)floor(L / rlist);
  if (nc > 0 && L / nc - rlist < 1e-9 * L) nc--;
  return nc < 3 ? 1 : nc;
}

float round_down_f(double x) {
  float f = (float)x;
  return ((double)f > x) ? nextafterf(f, -INFINITY) : f;
}
float round_up_f(double x) {
  float f = (float)x;
  return ((double)f < x) ? nextafterf(f, INFINITY) : f;
}

// Per-replica boxes and cell grids, and the FP32 build-filter bounds.
int setup_geometry(md_ctx* c, const double* boxes) {
  const double u = ldexp(1.0, -24);
  double e2max = 0.0;
  int64_t cells = 0;
  // grid of the split positions' hi parts: 2^24 steps span P, the smallest
  // power of two above 1.25 x the largest edge (room for atoms that drift
  // out of the box between rebuilds)
  double lmax = 0.0;
  for (int k = 0; k < 3 * c->nrep; k++) lmax = boxes[k] > lmax ? boxes[k] : lmax;
  int pe = 0;
  frexp(1.25 * lmax, &pe);
  const double P = ldexp(1.0, pe);
  c->xgrid.k = pe - 24;
  for (int r = 0; r < c->nrep; r++) {
    RepGeo& g = c->rep_host[r];
    memset(&g, 0, sizeof(g));
    double e2 = 0.0;
    int64_t ncr = 1;
    for (int a = 0; a < 3; a++) {
      const double L = boxes[3 * r + a];
      g.L[a] = L;
      const double half = 0.5 * L;
      memcpy(&g.halfL_bits[a], &half, 8);
      g.Lf[a] = (float)L;
      g.Llo[a] = (float)(L - (double)g.Lf[a]);
      g.halfLf[a] = (float)half;
      g.nc[a] = cells_along(L, c->rlist);
      g.cinv[a] = g.nc[a] / L;
      g.nb[a] = (g.nc[a] + 3) / 4;
      // fixed-point scale of the box's positions: 2^E >= 1.25 x its largest
      // edge bounds every position between rebuilds, and F = 61 - E keeps
      // |X| < 2^61 and separations below half the box under 2^60
      if (a == 2) {
        const double lm = 1.25 * fmax(boxes[3 * r], fmax(boxes[3 * r + 1], boxes[3 * r + 2]));
        int E = 0;
        frexp(lm, &E);  // lm < 2^E
        g.xfix = 61 - E;
      }
      g.lo[a] = g.nc[a] >= 3 ? -1 : 0;
      g.hi[a] = g.nc[a] >= 3 ? 1 : 0;
      ncr *= 4 * g.nb[a];  // brick order pads each axis to a multiple of 4
      // |(|d_f| - |d|)| per component: position rounding (|x - hi| <= u P
      // for each of the two atoms; the subtraction of hi parts and the image
      // shift are exact), and a different image choice near |d| = L/2
      // (<= 5 u L); u (2 P + 10 L) covers them.
      const double ea = u * (2.0 * P + 10.0 * L);
      e2 += ea * ea;
    }
    if (cells + ncr > (int64_t)INT32_MAX - 1) return MD_EINVAL;
    g.cell_base = (int)cells;
    cells += ncr;
    if (e2 > e2max) e2max = e2;
  }
  c->ncell = cells;
  Geo& gg = c->geo;
  gg.rlist2 = c->rlist * c->rlist;
  memcpy(&gg.rlist2_bits, &gg.rlist2, 8);
  const double e = sqrt(e2max);
  // r2f carries at most ~3u relative rounding; 4u margin
  const double lo = c->rlist - e;
  gg.lo2f = lo > 0 ? round_down_f(lo * lo * (1.0 - 4.0 * u)) : 0.0f;
  gg.hi2f = round_up_f((c->rlist + e) * (c->rlist + e) * (1.0 + 4.0 * u));
  gg.nt = c->nt;
  c->filt_e = e;
  return MD_OK;
}

}  // namespace

// The force cutoff of each type pair (the larger of rc and, with the
// Coulomb term, rc_coul): the build's inner/skin split and the compacted
// kernel's certified FP32 upper bound of it.
static void set_cut_bounds(md_ctx* c) {
  const double u = ldexp(1.0, -24), e = c->filt_e;
  Geo& gg = c->geo;
  for (int k = 0; k < MD_MAX_TYPES * MD_MAX_TYPES; k++) {
    if (k >= c->nt * c->nt) {
      gg.cutsqf[k] = 0.f;
      gg.cut_hi[k] = 0.f;
      continue;
    }
    const double rce = (c->coul && c->rc_coul > c->rc[k]) ? c->rc_coul : c->rc[k];
    gg.cutsqf[k] = (float)(rce * rce);
    gg.cut_hi[k] = round_up_f((rce + e) * (rce + e) * (1.0 + 4.0 * u));
  }
}

void md_set_coef(PairCoef& pc, double eps, double sigma, double rc, double qq,
                 double rc_coul) {
  const double s2 = sigma * sigma, s6 = s2 * s2 * s2, s12 = s6 * s6;
  pc.cutsq = rc * rc;
  memcpy(&pc.cutsq_bits, &pc.cutsq, 8);
  const double cc = rc_coul > 0.0 ? rc_coul * rc_coul : 0.0;
  memcpy(&pc.cutsq_coul_bits, &cc, 8);
  const double cm = cc > pc.cutsq ? cc : pc.cutsq;
  memcpy(&pc.cutmax_bits, &cm, 8);
  pc.qq = rc_coul > 0.0 ? qq : 0.0;
  pc.qqf = (float)pc.qq;
  pc.cutsq_coulf = (float)cc;
  pc.lj1 = 48.0 * eps * s12;
  pc.lj2 = 24.0 * eps * s6;
  pc.lj3 = 4.0 * eps * s12;
  pc.lj4 = 4.0 * eps * s6;
  pc.cutsqf = (float)pc.cutsq;
  const double band = ldexp(1.0, -18);
  pc.cut_lof = round_down_f(pc.cutsq * (1.0 - band));
  pc.cut_hif = round_up_f(pc.cutsq * (1.0 + band));
  pc.coul_lof = cc > 0.0 ? round_down_f(cc * (1.0 - band)) : 0.f;
  pc.coul_hif = cc > 0.0 ? round_up_f(cc * (1.0 + band)) : 0.f;
  pc.lj1f = (float)pc.lj1;
  pc.lj2f = (float)pc.lj2;
  pc.lj3f = (float)pc.lj3;
  pc.lj4f = (float)pc.lj4;
}

// Coefficient table (device), the single-type copy, and the FP32 cutoff
// bounds (device copy for the compacted kernel).  Synchronizes: the host
// table must outlive the copies.
int md_upload_coef(md_ctx* c) {
  const int nt = c->nt;
  set_cut_bounds(c);
  PairCoef tab[MD_MAX_TYPES * MD_MAX_TYPES];
  memset(tab, 0, sizeof(tab));
  for (int a = 0; a < nt; a++)
    for (int b = 0; b < nt; b++) {
      const int k = a * nt + b;
      const double qq = c->coul ? c->qqrd2e * c->qtype[a] * c->qtype[b] : 0.0;
      md_set_coef(tab[k], c->eps[k], c->sigma[k], c->rc[k], qq, c->coul ? c->rc_coul : 0.0);
    }
  c->coef1 = tab[0];
  MD_CUDA(cudaMemcpyAsync(c->coef, tab, sizeof(tab), cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaMemcpyAsync(c->cut_hi_dev, c->geo.cut_hi, sizeof(c->geo.cut_hi),
                          cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return MD_OK;
}

namespace {

// Checks of everything but the boxes; *rcmax_out receives max rc.
int check_params(const md_params* p, double* rcmax_out) {
  if (!p) return MD_EINVAL;
  if (p->n_atoms < 1 || p->n_atoms >= (int64_t)INT32_MAX) return MD_EINVAL;
  if (p->n_types < 1 || p->n_types > MD_MAX_TYPES) return MD_EINVAL;
  if (p->list_kind != MD_LIST_FULL && p->list_kind != MD_LIST_HALF) return MD_EINVAL;
  if (p->precision != MD_PREC_FP64 && p->precision != MD_PREC_MIXED) return MD_EINVAL;
  if (p->rebuild_every < 1) return MD_EINVAL;
  if (!(p->skin >= 0.0) || !(p->dt > 0.0) || !isfinite(p->dt) || !isfinite(p->skin))
    return MD_EINVAL;
  const int tpa = p->threads_per_atom;
  if (tpa != 0 && tpa != 1 && tpa != 2 && tpa != 4 && tpa != 8 && tpa != 16 && tpa != 32)
    return MD_EINVAL;
  if (p->max_neigh < 0) return MD_EINVAL;
  if (p->check_disp != 0 && p->check_disp != 1) return MD_EINVAL;
  if (!p->eps || !p->sigma || !p->rc || !p->mass) return MD_EINVAL;
  const int nt = p->n_types;
  double rcmax = 0.0;
  for (int a = 0; a < nt; a++) {
    if (!(p->mass[a] > 0.0) || !isfinite(p->mass[a])) return MD_EINVAL;
    for (int b = 0; b < nt; b++) {
      const double e = p->eps[a * nt + b], s = p->sigma[a * nt + b], r = p->rc[a * nt + b];
      if (!(e > 0.0) || !(s > 0.0) || !(r > 0.0) || !isfinite(e) || !isfinite(s) || !isfinite(r))
        return MD_EINVAL;
      if (e != p->eps[b * nt + a] || s != p->sigma[b * nt + a] || r != p->rc[b * nt + a])
        return MD_EINVAL;
      if (r > rcmax) rcmax = r;
    }
  }
  *rcmax_out = rcmax;
  return MD_OK;
}

// One periodic image within rc along every axis of every box.
int check_boxes(const double* boxes, int nrep, double rcmax) {
  for (int r = 0; r < nrep; r++)
    for (int a = 0; a < 3; a++) {
      const double L = boxes[3 * r + a];
      if (!(L > 0.0) || !isfinite(L) || !(rcmax < 0.5 * L)) return MD_EINVAL;
    }
  return MD_OK;
}

void free_ctx(md_ctx* c) {
  if (!c) return;
  if (c->graphs) {
    md_drop_graphs(c);
    delete c->graphs;
  }
  void* bufs[] = {c->x4,     c->v,      c->f,        c->id,       c->xs,      c->xb,
                  c->cell,   c->tag0,   c->coef,     c->x4_alt,   c->v_alt,   c->f_alt,
                  c->id_alt, c->cnt,    c->start,    c->rank,     c->perm,    c->cell_alt,
                  c->scan_tmp, c->numneigh, c->nbr,  c->ev,       c->dmax,    c->i64_tmp,
                  c->stage,  c->rep,     c->vcoef,    c->adj_c,    c->adj_xbar, c->adj_vbar,
                  c->adj_carry, c->seg_x, c->gbar,     c->fmax_bits, c->cut_hi_dev,
                  c->tile_ctr, c->fix,   c->xq,       c->evs};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->pair_ev) {
    for (int k = 0; k < 2 * MD_PAIR_TIMING_MAX; k++)
      if (c->pair_ev[k]) cudaEventDestroy(c->pair_ev[k]);
    delete[] c->pair_ev;
  }
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->ev_host) cudaFreeHost(c->ev_host);
  delete[] c->rep_host;
  delete[] c->rep_off_host;
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int initial_capacity(const md_ctx* c) {
  double expect = 0.0;
  for (int r = 0; r < c->nrep; r++) {
    const RepGeo& g = c->rep_host[r];
    const double nr = (double)(c->rep_off_host[r + 1] - c->rep_off_host[r]);
    const double rho = nr / (g.L[0] * g.L[1] * g.L[2]);
    double e = 4.0 / 3.0 * M_PI * c->rlist * c->rlist * c->rlist * rho;
    if (e > nr - 1) e = nr - 1;
    if (e > expect) expect = e;
  }
  int cap = (int)(expect * 1.3) + 16;
  return (cap + 7) & ~7;
}

}  // namespace

// The step driver runs one cooperative launch per step (md_step_fused.cu):
// persistent mode 2 on the compacted FP64 kernel with fixed-point sums.
int md_step_fused_ok(const md_ctx* c) {
  return c->persist == 2 && c->precision == MD_PREC_FP64 && c->compact == 2 && !c->coul;
}

// Build, then compute forces (no energy) -- the fresh-start sequence.
int md_fresh_start(md_ctx* c) {
  MD_TRY(md_rebuild(c));
  if (c->tpa == 0) MD_TRY(md_autotune(c));
  MD_TRY(md_launch_pair(c, 0, c->tpa));
  return MD_OK;
}

namespace {

// One cooperative launch: K21 (or K1) of every atom, a grid barrier, the
// forces (md_step_fused.cu).
int launch_fused(md_ctx* c, int mode) {
  const IntArgs ia = md_int_args(c, md_pair_fixed(c), md_pair_accumulates(c));
  PairArgs a;
  memset(&a, 0, sizeof(a));
  a.x4 = c->x4;
  a.xs = c->xs;
  a.xq = c->xq;
  a.numneigh = c->numneigh;
  a.nbr = c->nbr;
  a.f = c->f;
  a.fix = c->fix;
  a.kmax = c->dmax + 2;
  a.coef = c->coef;
  a.c1 = c->coef1;
  a.rep = c->rep;
  a.ev = c->evs;
  a.ev_spread = c->ev_spread;
  a.n = c->n;
  a.nt = c->nt;
  a.maxneigh = c->maxneigh;
  a.nslots = c->nsm;
  a.tile_ctr = c->tile_ctr;
  cudaError_t e = md_step_fused_launch(ia, a, mode, c->list_kind == MD_LIST_HALF, c->nt == 1,
                                       c->geo.cut_hi[0], c->cut_hi_dev, c->dmax + 6,
                                       c->dmax + 5, c->stream);
  c->launches++;
  MD_CUDA(e);
  return MD_OK;
}

// The kernels of a segment launched directly, with a CUDA event pair around
// every pair launch (md_time_pair_kernel): the same launches, in the same
// order, as the segment's graph.
int run_segment_timed(md_ctx* c, int m, int last_k2) {
  const int fold = md_pair_fixed(c), zero = md_pair_accumulates(c);
  auto timed = [&](auto&& launch) -> int {
    const int k = c->pair_ev_used;
    const bool rec = k < MD_PAIR_TIMING_MAX;
    if (rec) MD_CUDA(cudaEventRecord(c->pair_ev[2 * k], c->stream));
    MD_TRY(launch());
    if (rec) {
      MD_CUDA(cudaEventRecord(c->pair_ev[2 * k + 1], c->stream));
      c->pair_ev_used = k + 1;
    }
    return MD_OK;
  };
  if (md_step_fused_ok(c)) {
    MD_TRY(timed([&] { return md_launch_pair_step(c); }));
    for (int k = 1; k < m; k++) MD_TRY(timed([&] { return launch_fused(c, MD_K21); }));
    return md_launch_integrate(c, last_k2 ? MD_K2 : MD_K21, fold, last_k2 ? 0 : zero);
  }
  for (int k = 0; k < m; k++) {
    MD_TRY(timed([&] { return md_launch_pair_step(c); }));
    if (last_k2 && k == m - 1)
      MD_TRY(md_launch_integrate(c, MD_K2, fold, 0));
    else
      MD_TRY(md_launch_integrate(c, MD_K21, fold, zero));
  }
  return MD_OK;
}

int run_segment(md_ctx* c, int m, int last_k2) {
  if (c->time_pair) return run_segment_timed(c, m, last_k2);
  GraphKey key{m, last_k2};
  auto it = c->graphs->find(key);
  if (it == c->graphs->end()) {
    cudaGraph_t g = nullptr;
    MD_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = MD_OK;
    const int64_t saved = c->launches;
    const int fold = md_pair_fixed(c), zero = md_pair_accumulates(c);
    if (md_step_fused_ok(c)) {
      // P, then (K21 + P) as one launch per step, then the closing kick:
      // m + 1 launches for m steps
      rc = md_launch_pair_step(c);
      for (int k = 1; k < m && rc == MD_OK; k++) rc = launch_fused(c, MD_K21);
      if (rc == MD_OK) rc = md_launch_integrate(c, last_k2 ? MD_K2 : MD_K21, fold,
                                                last_k2 ? 0 : zero);
    }
    for (int k = 0; k < m && rc == MD_OK && !md_step_fused_ok(c); k++) {
      rc = md_launch_pair_step(c);
      if (rc != MD_OK) break;
      if (last_k2 && k == m - 1)
        rc = md_launch_integrate(c, MD_K2, fold, 0);
      else
        rc = md_launch_integrate(c, MD_K21, fold, zero);
    }
    const int kernels = (int)(c->launches - saved);
    c->launches = saved;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != MD_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    MD_CUDA(e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    MD_CUDA(e);
    it = c->graphs->emplace(key, std::make_pair(ex, kernels)).first;
  }
  MD_CUDA(cudaGraphLaunch(it->second.first, c->stream));
  c->launches += it->second.second;
  return MD_OK;
}

// Tags (type | replica << 8) in the caller's order; the replica of atom i is
// found by binary search in the atom offsets.
__global__ void k_make_tags(const int32_t* __restrict__ type, const int64_t* __restrict__ off,
                            int nrep, int64_t n, int32_t* __restrict__ tag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nrep - 1;  // off[lo] <= i < off[hi + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  tag[i] = MD_TAG(type[i], lo);
}

int create_impl(const md_params* p, int nrep, const int64_t* rep_off, const double* boxes,
                const double* x, const double* v, const int32_t* type, void* stream,
                md_ctx** out) {
  if (!out) return MD_EINVAL;
  *out = nullptr;
  double rcmax = 0.0;
  MD_TRY(check_params(p, &rcmax));
  if (nrep < 1 || nrep >= (1 << 23) || !rep_off || !boxes) return MD_EINVAL;
  if (rep_off[0] != 0 || rep_off[nrep] != p->n_atoms) return MD_EINVAL;
  for (int r = 0; r < nrep; r++)
    if (rep_off[r + 1] <= rep_off[r]) return MD_EINVAL;
  MD_TRY(check_boxes(boxes, nrep, rcmax));
  if (!x || !v || !type) return MD_EINVAL;
  md_ctx* c = new (std::nothrow) md_ctx();
  if (!c) return MD_ENOMEM;
  memset((void*)c, 0, sizeof(md_ctx));
  c->n = p->n_atoms;
  c->nt = p->n_types;
  c->list_kind = p->list_kind;
  c->precision = p->precision;
  c->rebuild_every = p->rebuild_every;
  c->check_disp = p->check_disp;
  c->tpa = p->threads_per_atom;
  c->carve = -1;
  c->skin = p->skin;
  c->dt = p->dt;
  c->nrep = nrep;
  const int nt = c->nt;
  for (int k = 0; k < nt * nt; k++) {
    c->eps[k] = p->eps[k];
    c->sigma[k] = p->sigma[k];
    c->rc[k] = p->rc[k];
  }
  for (int t = 0; t < nt; t++) {
    c->mass[t] = p->mass[t];
    c->dtf[t] = 0.5 * c->dt / c->mass[t];
  }
  c->rlist = rcmax + c->skin;
  c->rep_host = new (std::nothrow) RepGeo[nrep];
  c->rep_off_host = new (std::nothrow) int64_t[nrep + 1];
  c->graphs = new (std::nothrow) std::map<GraphKey, std::pair<cudaGraphExec_t, int>>();
  int rc = (c->rep_host && c->rep_off_host && c->graphs) ? MD_OK : MD_ENOMEM;
  if (rc == MD_OK) {
    memcpy(c->rep_off_host, rep_off, sizeof(int64_t) * (nrep + 1));
    rc = setup_geometry(c, boxes);
  }
  if (rc == MD_OK) {
    if (stream) {
      c->stream = (cudaStream_t)stream;
    } else {
      // a blocking stream: ordered after work the caller left on the legacy stream
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault) != cudaSuccess) rc = MD_ECUDA;
      c->own_stream = 1;
    }
  }
  const int64_t n = c->n;
  if (rc == MD_OK) rc = dalloc(&c->x4, n);
  if (rc == MD_OK) rc = dalloc(&c->v, 3 * n);
  if (rc == MD_OK) rc = dalloc(&c->f, 3 * n);
  if (rc == MD_OK) rc = dalloc(&c->fix, 3 * n);
  if (rc == MD_OK) rc = dalloc(&c->id, n);
  if (rc == MD_OK) rc = dalloc(&c->xs, n);
  if (rc == MD_OK) rc = dalloc(&c->xb, n);
  if (rc == MD_OK && c->precision == MD_PREC_FP64) rc = dalloc(&c->xq, n);
  if (rc == MD_OK) rc = dalloc(&c->cell, n);
  if (rc == MD_OK) rc = dalloc(&c->tag0, n);
  if (rc == MD_OK) rc = dalloc(&c->coef, MD_MAX_TYPES * MD_MAX_TYPES);
  if (rc == MD_OK) rc = dalloc(&c->cut_hi_dev, MD_MAX_TYPES * MD_MAX_TYPES);
  if (rc == MD_OK) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        c->nsm < 1)
      rc = MD_ECUDA;
    c->persist = 0;
    c->qu = 1;
  }
  if (rc == MD_OK) rc = dalloc(&c->tile_ctr, c->nsm);
  if (rc == MD_OK) rc = dalloc(&c->rep, nrep);
  c->xgrid.rep = c->rep;
  if (rc == MD_OK) rc = dalloc(&c->x4_alt, n);
  if (rc == MD_OK) rc = dalloc(&c->v_alt, 3 * n);
  if (rc == MD_OK) rc = dalloc(&c->f_alt, 3 * n);
  if (rc == MD_OK) rc = dalloc(&c->id_alt, n);
  if (rc == MD_OK) rc = dalloc(&c->cell_alt, n);
  if (rc == MD_OK) rc = dalloc(&c->rank, n);
  if (rc == MD_OK) rc = dalloc(&c->perm, n);
  if (rc == MD_OK) rc = dalloc(&c->cnt, c->ncell);
  if (rc == MD_OK) rc = dalloc(&c->start, c->ncell + 1);
  if (rc == MD_OK) rc = dalloc(&c->numneigh, 2 * n);
  if (rc == MD_OK) rc = dalloc(&c->ev, (int64_t)nrep * MD_EV_STRIDE);
  c->ev_spread = nrep < 128 ? 128 / nrep : 1;
  if (rc == MD_OK) rc = dalloc(&c->evs, (int64_t)nrep * c->ev_spread * MD_EV_STRIDE);
  if (rc == MD_OK &&
      cudaMemset(c->evs, 0, sizeof(double) * (size_t)nrep * c->ev_spread * MD_EV_STRIDE) !=
          cudaSuccess)
    rc = MD_ECUDA;
  if (rc == MD_OK) rc = dalloc(&c->dmax, 8);
  if (rc == MD_OK) rc = dalloc(&c->i64_tmp, 4);
  if (rc == MD_OK && cudaMallocHost((void**)&c->h_pinned, 16 * sizeof(double)) != cudaSuccess)
    rc = MD_ENOMEM;
  if (rc == MD_OK) memset(c->h_pinned, 0, 16 * sizeof(double));
  if (rc == MD_OK && cudaMallocHost((void**)&c->ev_host,
                                    sizeof(double) * (size_t)nrep * MD_EV_STRIDE) != cudaSuccess)
    rc = MD_ENOMEM;
  if (rc == MD_OK) {
    int cap = p->max_neigh > 0 ? ((p->max_neigh + 7) & ~7) : initial_capacity(c);
    int64_t tiles = (n + 31) / 32;
    rc = dalloc(&c->nbr, tiles * 32 * (int64_t)cap);
    c->nbr_alloc = tiles * 32 * (int64_t)cap;
    c->maxneigh = cap;
  }
  int64_t* off_dev = nullptr;
  if (rc == MD_OK) rc = dalloc(&off_dev, nrep + 1);
  if (rc == MD_OK) rc = md_upload_coef(c);
  if (rc == MD_OK) {
    cudaStream_t s = c->stream;
    bool ok =
        cudaMemcpyAsync(c->rep, c->rep_host, sizeof(RepGeo) * nrep, cudaMemcpyHostToDevice, s) ==
            cudaSuccess &&
        cudaMemcpyAsync(off_dev, rep_off, sizeof(int64_t) * (nrep + 1), cudaMemcpyHostToDevice,
                        s) == cudaSuccess &&
        cudaMemsetAsync(c->dmax, 0, 8 * sizeof(unsigned int), s) == cudaSuccess &&
        cudaMemsetAsync(c->f, 0, sizeof(double) * 3 * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->fix, 0, sizeof(unsigned long long) * 3 * n, s) == cudaSuccess;
    if (ok) {
      k_make_tags<<<(unsigned)md_blocks(n), MD_BLOCK, 0, s>>>(type, off_dev, nrep, n, c->tag0);
      c->launches++;
      ok = cudaGetLastError() == cudaSuccess;
    }
    // the host tables and the offsets must outlive the copies
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) rc = MD_ECUDA;
  }
  if (off_dev) cudaFree(off_dev);
  if (rc == MD_OK) rc = md_launch_load_state(c, x, v);
  if (rc == MD_OK) rc = md_fresh_start(c);
  if (rc == MD_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = MD_ECUDA;
  if (rc != MD_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return MD_OK;
}

// The FP64 kernels with one type and Eq. 1 alone sum a pair's energy as
// -(lj4 / 2) r^-6 and leave fpair r^2 / 12 (lj1 = 12 lj3, lj2 = 6 lj4) to
// the virial: the potential energy is then ev[0] + trace(W) / 12.
double md_ev_trace_share(const md_ctx* c) {
  return (c->precision == MD_PREC_FP64 && c->nt == 1 && !c->coul) ? 1.0 / 12.0 : 0.0;
}

// Pair energies/virials and kinetic energies per replica into ev_host.
int thermo_per_replica(md_ctx* c) {
  MD_TRY(md_launch_pair(c, 1, c->tpa));
  MD_TRY(md_launch_kinetic(c));
  MD_CUDA(cudaMemcpyAsync(c->ev_host, c->ev, sizeof(double) * (size_t)c->nrep * MD_EV_STRIDE,
                          cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  double pairs = 0.0;
  for (int r = 0; r < c->nrep; r++) pairs += c->ev_host[r * MD_EV_STRIDE + 7];
  c->pairs_in_range = (int64_t)llround(pairs);
  return MD_OK;
}

// MD_THERMO_N values from one accumulator block; dof = degrees of freedom.
// trc: the share of the virial's trace in the potential energy (1/12 where
// the FP64 kernels summed only the r^-6 part, md_ev_trace_share; else 0).
void fill_thermo(const double* e, double dof, double* out, double trc) {
  const double pe = trc != 0.0 ? e[0] + trc * (e[1] + e[2] + e[3]) : e[0];
  out[0] = pe;
  out[1] = e[8];
  out[2] = pe + e[8];
  out[3] = dof > 0 ? 2.0 * e[8] / dof : 0.0;
  for (int k = 0; k < 6; k++) out[4 + k] = e[1 + k];
}

}  // namespace

// ---- pair dispatch (used by the step driver and the tuner) -------------------

int md_pair_accumulates(const md_ctx* c) {
  // mixed: fixed-point sums in fix, contributions beyond their range in f
  if (c->precision != MD_PREC_FP64) return 1;
  return c->list_kind == MD_LIST_HALF || c->compact;
}

int md_pair_fixed(const md_ctx* c) {
  if (c->precision == MD_PREC_FP64) return c->compact == 2;
  return 1;
}

namespace {

// ev: energy and virial too; the virial's sum over atoms needs the final
// forces, so it is only asked for with the fold in this call.
int launch_pair_impl(md_ctx* c, int ev, int tpa, int prezeroed, int defer_fold) {
  if (ev && defer_fold) return MD_EINVAL;
  PairArgs a;
  a.x4 = c->x4;
  a.xs = c->xs;
  a.xq = c->xq;
  a.numneigh = c->numneigh;
  a.nbr = c->nbr;
  a.f = c->f;
  a.fix = c->fix;
  a.kmax = c->dmax + 2;
  a.coef = c->coef;
  a.c1 = c->coef1;
  a.rep = c->rep;
  a.ev = c->evs;
  a.ev_spread = c->ev_spread;
  a.n = c->n;
  a.nt = c->nt;
  a.maxneigh = c->maxneigh;
  a.nslots = c->nsm;
  a.tile_ctr = c->persist ? c->tile_ctr : nullptr;
  if (c->persist)
    MD_CUDA(cudaMemsetAsync(c->tile_ctr, 0, sizeof(int) * c->nsm, c->stream));
  const unsigned blocks = (unsigned)md_blocks(c->n * (int64_t)tpa);
  if (ev)
    MD_CUDA(cudaMemsetAsync(c->ev, 0, sizeof(double) * (size_t)c->nrep * MD_EV_STRIDE,
                            c->stream));
  const bool half = c->list_kind == MD_LIST_HALF;
  const bool compact = c->compact && c->precision == MD_PREC_FP64;
  if (md_pair_accumulates(c) && !prezeroed)  // sums by atomics start from zero
    MD_CUDA(cudaMemsetAsync(c->f, 0, sizeof(double) * 3 * c->n, c->stream));
  if (compact) {
    const bool fix = c->compact == 2;
    cudaError_t e =
        c->coul ? md_pair_q_coul_launch(a, fix, half, ev != 0, c->nt == 1, c->geo.cut_hi[0],
                                        c->cut_hi_dev, (unsigned)md_blocks(c->n), c->stream,
                                        c->carve)
                : fix ? md_pair_q_fix_launch(a, half, ev != 0, c->nt == 1, c->geo.cut_hi[0],
                                             c->cut_hi_dev, (unsigned)md_blocks(c->n),
                                             c->stream, c->carve, c->qu)
                      : md_pair_q_launch(a, half, ev != 0, c->nt == 1, c->geo.cut_hi[0],
                                         c->cut_hi_dev, (unsigned)md_blocks(c->n), c->stream,
                                         c->carve);
    c->launches++;
    MD_CUDA(e);
    if (fix && !defer_fold) MD_TRY(md_launch_fix_finalize(c));
    if (ev) MD_TRY(md_launch_virial_atoms(c));
    if (ev) MD_TRY(md_launch_ev_fold(c));
    return MD_OK;
  }
  if (c->coul && c->precision == MD_PREC_FP64) return MD_EINVAL;  // FP64 Coulomb: k_pair_q
  cudaError_t e =
      (c->precision == MD_PREC_FP64)
          ? md_pair_launch_fp64(a, half, ev != 0, c->nt == 1, tpa, blocks, c->stream, c->carve)
      : c->coul
          ? md_pair_launch_mixed_coul(a, half, ev != 0, c->nt == 1, tpa, blocks, c->stream,
                                      c->carve)
          : md_pair_launch_mixed(a, half, ev != 0, c->nt == 1, tpa, blocks, c->stream, c->carve);
  c->launches++;
  MD_CUDA(e);
  if (md_pair_fixed(c) && !defer_fold) MD_TRY(md_launch_fix_finalize(c));
  if (ev) MD_TRY(md_launch_virial_atoms(c));
  if (ev) MD_TRY(md_launch_ev_fold(c));
  return MD_OK;
}

}  // namespace

// Forces of the current positions into f (sums zeroed first, fixed-point
// sums folded): the form every caller outside the step segments uses.
int md_launch_pair(md_ctx* c, int ev, int tpa) { return launch_pair_impl(c, ev, tpa, 0, 0); }

int md_launch_pair_step(md_ctx* c) { return launch_pair_impl(c, 0, c->tpa, 1, 1); }

// ---- C ABI ----------------------------------------------------------------------

extern "C" {

const char* md_strerror(int code) {
  switch (code) {
    case MD_OK: return "success";
    case MD_EINVAL: return "invalid argument";
    case MD_ENOMEM: return "out of memory";
    case MD_ENEIGH: return "neighbor list capacity could not be grown enough";
    case MD_ECUDA: return "CUDA runtime error";
    case MD_ENONFINITE: return "non-finite energy or virial";
    case MD_ETIMEOUT: return "bounded device wait expired";
    default: return "unknown error";
  }
}

int md_create(const md_params* p, const double* x, const double* v, const int32_t* type,
              void* stream, md_ctx** out) {
  if (!out) return MD_EINVAL;
  *out = nullptr;
  if (!p) return MD_EINVAL;
  const int64_t off[2] = {0, p->n_atoms};
  return create_impl(p, 1, off, p->box, x, v, type, stream, out);
}

int md_create_batch(const md_params* p, int32_t n_replicas, const int64_t* rep_offset,
                    const double* boxes, const double* x, const double* v, const int32_t* type,
                    void* stream, md_ctx** out) {
  return create_impl(p, n_replicas, rep_offset, boxes, x, v, type, stream, out);
}

void md_destroy(md_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

int md_set_state(md_ctx* c, const double* x, const double* v, int32_t mem) {
  if (!c || !x || !v || mem < 0 || mem > (MD_MEM_HOST | MD_MEM_KEEP_LIST)) return MD_EINVAL;
  const bool keep = (mem & MD_MEM_KEEP_LIST) != 0;
  mem &= MD_MEM_HOST;
  const int64_t n = c->n;
  if (mem == MD_MEM_HOST) {
    if (!c->stage) MD_TRY(dalloc(&c->stage, 6 * n));
    MD_CUDA(cudaMemcpyAsync(c->stage, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                            c->stream));
    MD_CUDA(cudaMemcpyAsync(c->stage + 3 * n, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                            c->stream));
    x = c->stage;
    v = c->stage + 3 * n;
  }
  if (keep) {
    // the list stays valid while no atom moved more than skin/2 since the
    // build (a pair can then have closed in by at most skin); the FP32
    // displacement is within 1e-6 relative of the exact one
    MD_CUDA(cudaMemsetAsync(c->dmax + 3, 0, 2 * sizeof(unsigned int), c->stream));
    MD_TRY(md_launch_load_keep(c, x, v));
    MD_CUDA(cudaMemcpyAsync(c->h_pinned + 12, c->dmax + 3, 2 * sizeof(unsigned int),
                            cudaMemcpyDeviceToHost, c->stream));
    MD_CUDA(cudaStreamSynchronize(c->stream));
    unsigned int words[2];
    memcpy(words, (const char*)(c->h_pinned + 12), sizeof(words));
    float d2;
    memcpy(&d2, &words[0], sizeof(d2));
    const double lim = 0.5 * c->skin * (1.0 - 1e-5);
    if ((double)d2 < lim * lim) {
      c->step = 0;
      // positions identical to the ones held (bit for bit): the forces in f
      // are already those of these positions
      if (words[1]) MD_TRY(md_launch_pair(c, 0, c->tpa));
      MD_CUDA(cudaStreamSynchronize(c->stream));
      return MD_OK;
    }
  }
  MD_TRY(md_launch_load_state(c, x, v));
  MD_CUDA(cudaMemsetAsync(c->dmax, 0, sizeof(unsigned int), c->stream));
  c->step = 0;
  c->builds = 0;
  c->dangerous = 0;
  return md_fresh_start(c);
}

int md_get_state(md_ctx* c, double* x, double* v, double* f, int32_t mem) {
  if (!c || (mem != MD_MEM_DEVICE && mem != MD_MEM_HOST)) return MD_EINVAL;
  if (!x && !v && !f) return MD_OK;
  const int64_t n = c->n;
  if (mem == MD_MEM_DEVICE) return md_launch_store_state(c, x, v, f);
  if (!c->stage) MD_TRY(dalloc(&c->stage, 6 * n));
  double* sx = x ? c->stage : nullptr;
  double* sv = v ? c->stage + 3 * n : nullptr;
  // the staging buffer holds 6n doubles: forces go through it in a second pass
  MD_TRY(md_launch_store_state(c, sx, sv, nullptr));
  if (x) MD_CUDA(cudaMemcpyAsync(x, sx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
  if (v) MD_CUDA(cudaMemcpyAsync(v, sv, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
  if (f) {
    MD_CUDA(cudaStreamSynchronize(c->stream));
    double* sf = c->stage;
    MD_TRY(md_launch_store_state(c, nullptr, nullptr, sf));
    MD_CUDA(cudaMemcpyAsync(f, sf, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
  }
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return MD_OK;
}

int md_build_neighbors(md_ctx* c) {
  if (!c) return MD_EINVAL;
  return md_rebuild(c);
}

int md_compute_forces(md_ctx* c, int32_t flags) {
  if (!c || (flags & ~(MD_ENERGY | MD_VIRIAL))) return MD_EINVAL;
  return md_launch_pair(c, flags != 0, c->tpa);
}

int md_step(md_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return MD_EINVAL;
  if (nsteps == 0) return MD_OK;
  const int64_t every = c->rebuild_every;
  // the first pair launch of the step adds into f: K1 leaves it at zero
  MD_TRY(md_launch_integrate(c, MD_K1, 0, md_pair_accumulates(c)));
  if (c->check_disp) {
    // one step per segment; after each drift the largest displacement since
    // the build decides whether the list is rebuilt before the next forces
    const double half = 0.5 * c->skin;
    for (int64_t k = 0; k < nsteps; k++) {
      const int64_t s = c->step + k;
      bool rebuild = (s + 1) % every == 0;
      if (!rebuild) {
        MD_CUDA(cudaMemcpyAsync(c->h_pinned + 13, c->dmax, sizeof(unsigned int),
                                cudaMemcpyDeviceToHost, c->stream));
        MD_CUDA(cudaStreamSynchronize(c->stream));
        unsigned int bits;
        memcpy(&bits, (const char*)(c->h_pinned + 13), sizeof(bits));
        float d2;
        memcpy(&d2, &bits, sizeof(d2));
        rebuild = (double)d2 > half * half * (1.0 - 1e-5);
      }
      if (rebuild) MD_TRY(md_rebuild(c));
      MD_TRY(run_segment(c, 1, k == nsteps - 1));
    }
    c->step += nsteps;
    return MD_OK;
  }
  int64_t k = 0;
  while (k < nsteps) {
    const int64_t s = c->step + k;
    const int64_t r = (s + 1) % every;
    if (r == 0) MD_TRY(md_rebuild(c));
    // steps until the next rebuild point (exclusive)
    const int64_t to_next = (r == 0) ? every : every - r;
    const int64_t m = to_next < nsteps - k ? to_next : nsteps - k;
    const int last = (k + m == nsteps);
    MD_TRY(run_segment(c, (int)m, last));
    k += m;
  }
  c->step += nsteps;
  return MD_OK;
}

int md_energy(md_ctx* c, double out[MD_THERMO_N]) {
  if (!c || !out) return MD_EINVAL;
  MD_TRY(thermo_per_replica(c));
  double tot[MD_EV_STRIDE] = {0};
  for (int r = 0; r < c->nrep; r++)
    for (int k = 0; k < MD_EV_STRIDE; k++) tot[k] += c->ev_host[r * MD_EV_STRIDE + k];
  // each replica conserves its own momentum: 3 N_r - 3 degrees of freedom
  fill_thermo(tot, 3.0 * (double)c->n - 3.0 * c->nrep, out, md_ev_trace_share(c));
  for (int k = 0; k < MD_THERMO_N; k++)
    if (!isfinite(out[k])) return MD_ENONFINITE;
  return MD_OK;
}

int md_energy_replicas(md_ctx* c, double* out) {
  if (!c || !out) return MD_EINVAL;
  MD_TRY(thermo_per_replica(c));
  int bad = 0;
  for (int r = 0; r < c->nrep; r++) {
    const double nr = (double)(c->rep_off_host[r + 1] - c->rep_off_host[r]);
    fill_thermo(c->ev_host + r * MD_EV_STRIDE, 3.0 * nr - 3.0, out + r * MD_THERMO_N,
                md_ev_trace_share(c));
    for (int k = 0; k < MD_THERMO_N; k++)
      if (!isfinite(out[r * MD_THERMO_N + k])) bad = 1;
  }
  return bad ? MD_ENONFINITE : MD_OK;
}

int md_neighbor_count(md_ctx* c, int64_t* total, int32_t* max_count) {
  if (!c) return MD_EINVAL;
  int64_t t = 0;
  MD_TRY(md_list_entries(c, &t));
  if (total) *total = t;
  if (max_count) *max_count = c->max_count;
  return MD_OK;
}

int md_get_neighbors(md_ctx* c, int64_t* offsets, int32_t* idx) {
  if (!c || !offsets || !idx) return MD_EINVAL;
  return md_list_to_csr(c, offsets, idx);
}

int md_autotune(md_ctx* c) {
  if (!c) return MD_EINVAL;
  // threads per atom (Sec. 4.1: parallelism over neighbors) and, in FP64,
  // the warp-compacted kernel with FP64 or fixed-point reductions, each with
  // one block per tile and then with persistent per-SM tile scheduling, and
  // for the fixed-point kernel (Eq. 1 alone) one or two list entries per
  // lane per round of its filter; driver-default carveout (a largest-L1 carveout was measured slower or
  // equal for every configuration on GB300 and stays available through
  // md_set_kernel, as does the one-launch-per-step schedule)
  static const int cand[] = {1, 2, 4, 8, 16, 32};
  cudaEvent_t e0, e1;
  MD_CUDA(cudaEventCreate(&e0));
  MD_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_tpa = 1, best_compact = (c->coul && c->precision == MD_PREC_FP64) ? 2 : 0;
  int best_persist = 0, best_qu = 1;
  int rc = MD_OK;
  c->carve = -1;
  const int ncompact = c->precision == MD_PREC_FP64 ? 3 : 1;
  // the Coulomb style exists as the compacted FP64 kernel and as the mixed
  // kernel at 1, 2 or 4 threads per atom
  const int cp0 = (c->coul && c->precision == MD_PREC_FP64) ? 1 : 0;
  const int ntpa = c->coul ? 3 : 6;
  for (int cp = cp0; cp < ncompact && rc == MD_OK; cp++) {
    c->compact = cp;
    for (int qi = 0; qi < (cp ? 1 : ntpa) && rc == MD_OK; qi++) {
      const int tpa = cand[qi];
      for (int v = 0; v < ((cp == 2 && !c->coul) ? 4 : 2) && rc == MD_OK; v++) {
        const int pe = v & 1;
        c->persist = pe;
        c->qu = 1 + (v >> 1);
        rc = md_launch_pair(c, 0, tpa);  // warm-up
        if (rc != MD_OK) break;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) {
          rc = MD_ECUDA;
          break;
        }
        for (int r = 0; r < 5 && rc == MD_OK; r++) rc = md_launch_pair(c, 0, tpa);
        if (rc != MD_OK) break;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
          rc = MD_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_tpa = tpa;
          best_compact = cp;
          best_persist = pe;
          best_qu = c->qu;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MD_TRY(rc);
  md_drop_graphs(c);
  c->tpa = best_tpa;
  c->compact = best_compact;
  c->persist = best_persist;
  c->qu = best_qu;
  return MD_OK;
}

int md_set_coulomb(md_ctx* c, const double* q, double rc_coul, double qqrd2e) {
  if (!c) return MD_EINVAL;
  if (q) {
    double rcmax = 0.0;
    for (int k = 0; k < c->nt * c->nt; k++) rcmax = fmax(rcmax, c->rc[k]);
    if (!(rc_coul > 0.0) || rc_coul > rcmax || !isfinite(qqrd2e)) return MD_EINVAL;
    for (int t = 0; t < c->nt; t++)
      if (!isfinite(q[t])) return MD_EINVAL;
    for (int t = 0; t < c->nt; t++) c->qtype[t] = q[t];
    c->rc_coul = rc_coul;
    c->qqrd2e = qqrd2e;
    c->coul = 1;
    if (c->precision == MD_PREC_FP64 && c->compact == 0) c->compact = 2;
    if (c->precision != MD_PREC_FP64 && c->tpa > 4) c->tpa = 2;
  } else {
    c->coul = 0;
  }
  md_drop_graphs(c);  // graphs hold the single-type coefficients and cutoff bound by value
  MD_TRY(md_upload_coef(c));
  return md_launch_pair(c, 0, c->tpa);
}

int md_set_kernel(md_ctx* c, int32_t threads_per_atom, int32_t carveout, int32_t compacted,
                  int32_t persistent) {
  if (!c) return MD_EINVAL;
  if (persistent < 0 || persistent > 2) return MD_EINVAL;
  if (persistent == 2 && (c->precision != MD_PREC_FP64 || compacted != 2 || c->coul))
    return MD_EINVAL;
  if (compacted == 3 && c->coul) return MD_EINVAL;  // two entries: Eq. 1 alone
  const int t = threads_per_atom;
  if (t != 1 && t != 2 && t != 4 && t != 8 && t != 16 && t != 32) return MD_EINVAL;
  if (carveout < -1 || carveout > 100 || compacted < 0 || compacted > 3) return MD_EINVAL;
  if (compacted && (c->precision != MD_PREC_FP64 || t != 1)) return MD_EINVAL;
  if (c->coul && c->precision == MD_PREC_FP64 && !compacted) return MD_EINVAL;
  if (c->coul && c->precision != MD_PREC_FP64 && t > 4) return MD_EINVAL;
  md_drop_graphs(c);
  c->tpa = t;
  c->carve = carveout;
  c->compact = compacted == 3 ? 2 : compacted;
  c->qu = compacted == 3 ? 2 : 1;
  c->persist = persistent;
  return MD_OK;
}

int md_time_pair_kernel(md_ctx* c, int32_t enable) {
  if (!c || (enable != 0 && enable != 1)) return MD_EINVAL;
  if (enable && !c->pair_ev) {
    cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[2 * MD_PAIR_TIMING_MAX]();
    if (!ev) return MD_ENOMEM;
    for (int k = 0; k < 2 * MD_PAIR_TIMING_MAX; k++) {
      if (cudaEventCreate(&ev[k]) != cudaSuccess) {
        cudaGetLastError();
        for (int q = 0; q < k; q++) cudaEventDestroy(ev[q]);
        delete[] ev;
        return MD_ENOMEM;
      }
    }
    c->pair_ev = ev;
  }
  if (enable) c->pair_ev_used = 0;
  c->time_pair = enable;
  return MD_OK;
}

int md_pair_kernel_time(md_ctx* c, double* total_ms, int64_t* launches) {
  if (!c || !total_ms || !launches) return MD_EINVAL;
  MD_CUDA(cudaStreamSynchronize(c->stream));
  double t = 0.0;
  for (int k = 0; k < c->pair_ev_used; k++) {
    float ms = 0.f;
    MD_CUDA(cudaEventElapsedTime(&ms, c->pair_ev[2 * k], c->pair_ev[2 * k + 1]));
    t += ms;
  }
  *total_ms = t;
  *launches = c->pair_ev_used;
  return MD_OK;
}

int md_get_stats(md_ctx* c, md_stats* out) {
  if (!c || !out) return MD_EINVAL;
  memset(out, 0, sizeof(*out));
  int64_t total = 0;
  MD_TRY(md_list_entries(c, &total));
  MD_CUDA(cudaMemcpyAsync(c->h_pinned + 11, c->dmax, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                          c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  unsigned int bits;
  memcpy(&bits, (const char*)(c->h_pinned + 11), sizeof(bits));
  float d2;
  memcpy(&d2, &bits, sizeof(d2));
  out->step = c->step;
  out->builds = c->builds;
  out->dangerous_builds = c->dangerous;
  out->kernel_launches = c->launches;
  out->list_entries = total;
  out->max_neigh = c->maxneigh;
  out->max_count = c->max_count;
  for (int a = 0; a < 3; a++) out->cells[a] = c->rep_host[0].nc[a];
  out->threads_per_atom = c->tpa;
  out->carveout = c->carve;
  out->compacted = c->compact;
  out->coulomb = c->coul;
  out->persistent = c->persist;
  // list entries a lane takes per round of the force-only pair kernel's
  // walk: the compacted fixed-point kernel's tuned depth, the mixed
  // kernel's fixed two, one otherwise
  out->phase1_entries = c->precision == MD_PREC_MIXED ? MD_PAIR_U : (c->compact == 2 ? c->qu : 1);
  out->max_disp = sqrt((double)d2);
  out->pairs_in_range = c->pairs_in_range;
  out->n_replicas = c->nrep;
  out->total_cells = c->ncell;
  return MD_OK;
}

int md_synchronize(md_ctx* c) {
  if (!c) return MD_EINVAL;
  MD_CUDA(cudaMemcpyAsync(c->h_pinned + 14, c->dmax + 5, sizeof(unsigned int),
                          cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  MD_CUDA(cudaGetLastError());
  return md_barrier_status(c);
}

}  // extern "C"
