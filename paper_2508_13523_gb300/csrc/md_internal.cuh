// md_internal.cuh -- context layout and kernel entry points shared by the
// translation units of libmd.so.  Device code only for sm_103a.
//
// A context holds R >= 1 independent periodic boxes ("replicas") whose atoms
// are concatenated; a single box is R = 1.  Every kernel runs once per step
// over all atoms of all replicas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <utility>

#include "../../include/md.h"

#define MD_BLOCK 128     // threads per block of every per-atom kernel
#define MD_EV_STRIDE 16  // doubles per replica in the energy accumulators

// ---- error plumbing ---------------------------------------------------------
#define MD_TRY(expr)                      \
  do {                                    \
    int md_rc_ = (expr);                  \
    if (md_rc_ != MD_OK) return md_rc_;   \
  } while (0)
#define MD_CUDA(expr)                                   \
  do {                                                  \
    cudaError_t md_e_ = (expr);                         \
    if (md_e_ != cudaSuccess) return md_cuda_fail(md_e_); \
  } while (0)
int md_cuda_fail(cudaError_t e);

// ---- per type-pair Eq. 1 coefficients -------------------------------------
// U(r) = r^-6 (lj3 r^-6 - lj4),  fpair = r^-2 r^-6 (lj1 r^-6 - lj2)
// with lj1 = 48 eps sigma^12, lj2 = 24 eps sigma^6, lj3 = 4 eps sigma^12,
// lj4 = 4 eps sigma^6 (Eq. 1 and its derivative, Sec. 4).
// Second pair style (lj/cut/coul/cut): a cut Coulomb term qq / r with
// qq = qqrd2e q_a q_b from per-type charges, for r < rc_coul.
struct PairCoef {
  double cutsq, lj1, lj2, lj3, lj4;
  double qq;                // Coulomb qqrd2e q_a q_b (0 without the term)
  float cutsqf, lj1f, lj2f, lj3f, lj4f;
  float qqf, cutsq_coulf;
  // FP32 r^2 at or below *_lof is inside the cutoff, at or above *_hif
  // outside it, whatever the FP32 rounding of r^2 (relative band 2^-18);
  // between them the FP64 r^2 decides (mixed precision; 0, 0: no such cutoff)
  float cut_lof, cut_hif, coul_lof, coul_hif;
  int64_t cutsq_bits;       // bit pattern of cutsq: r2 < cutsq as an integer compare
  int64_t cutsq_coul_bits;  // rc_coul^2 (0: no Coulomb term)
  int64_t cutmax_bits;      // the larger of the two: a pair has a force below it
};

struct RepGeo;

// Grid of the hi parts of split positions (md_split): step 2^k, with every
// |x| < 2^24 2^k.  rep: the per-replica boxes (device), whose xfix gives
// each replica's fixed-point scale (XFix).
struct XGrid {
  int k;
  const RepGeo* rep;
};

// ---- per-replica box and cell grid -------------------------------------------
struct RepGeo {
  double L[3];
  long long halfL_bits[3];  // |d| > L/2 as an integer compare on |d|'s bits
  double cinv[3];           // cells per unit length: nc / L
  float Lf[3], Llo[3], halfLf[3];  // L as a float pair (Lf + Llo)
  int nc[3];
  int nb[3];                // 4x4x4-cell bricks along each axis: ceil(nc / 4)
  int lo[3], hi[3];         // stencil offsets along each axis (-1..1 or 0..0)
  int cell_base;            // first global cell of this replica
  int xfix;                 // fixed-point scale F of its positions (XFix): 61 - E
                            // with 2^E >= 1.25 x the largest edge
};

// Linear cell index: cells are ordered brick by brick (4 x 4 x 4 cells,
// bricks in x-major order, cells x-major inside a brick), so that atoms that
// are close in the sorted order are close in space along all three axes
// (a column order keeps them close along one axis only).
__host__ __device__ inline int md_cell_index(const RepGeo& g, int cx, int cy, int cz) {
  const int b = ((cx >> 2) * g.nb[1] + (cy >> 2)) * g.nb[2] + (cz >> 2);
  return g.cell_base + (b << 6) + (((cx & 3) << 4) | ((cy & 3) << 2) | (cz & 3));
}
__host__ __device__ inline void md_cell_coords(const RepGeo& g, int c, int& cx, int& cy,
                                               int& cz) {
  c -= g.cell_base;
  const int in = c & 63, b = c >> 6;
  const int bz = b % g.nb[2], by = (b / g.nb[2]) % g.nb[1], bx = b / (g.nb[2] * g.nb[1]);
  cx = (bx << 2) | (in >> 4);
  cy = (by << 2) | ((in >> 2) & 3);
  cz = (bz << 2) | (in & 3);
}

// ---- quantities shared by all replicas -----------------------------------------
struct Geo {
  double rlist2;             // (max rc + skin)^2, FP64, the exact test
  long long rlist2_bits;
  float lo2f, hi2f;          // certified FP32 bounds around rlist2 (build filter)
  int nt;                    // atom types
  float cutsqf[MD_MAX_TYPES * MD_MAX_TYPES];  // rc^2 per type pair (row order only)
  // certified FP32 upper bounds of rc^2 per type pair: an FP32 distance of
  // the hi parts above it means r >= rc exactly (compacted pair kernel)
  float cut_hi[MD_MAX_TYPES * MD_MAX_TYPES];
};

// Per-atom position record used by the mixed-precision gathers and the build
// filter: a double-float split of the FP64 position (md_split: hi on the
// context's power-of-two grid, |x - hi - lo| <= 2^-25 grid step) with the
// packed type/replica tag in hi.w's bits.
struct __align__(32) XSplit {
  float4 hi;
  float4 lo;
};

// The tag packed into the fourth word of x4 (as int64 bits) and of xs.hi
// (as int32 bits): type in the low 8 bits, replica index above.
#define MD_TAG(type, rep) ((int)(type) | ((int)(rep) << 8))
#define MD_TAG_TYPE(tag) ((tag) & 0x7f)
#define MD_TAG_REP(tag) ((tag) >> 8)
// Set in the tag of xs (XSplit hi.w) only: some coordinate of the atom is
// not a multiple of 2^-F of its box (or too large), so its pairs take the
// FP64 separation path of the compacted kernel (XFix).
#define MD_TAG_OFFGRID 0x80

// Positions as fixed-point integers X = x 2^F with F = RepGeo::xfix of the
// atom's box (F = 61 - E, 2^E >= 1.25 x the box's largest edge: 53 for a
// 168-wide box).  X is exact for every double with 2^(52 - F) <= |x| < 2^E
// (all of them are multiples of 2^-F: from 0.5 up in a 168-wide box), and
// for smaller x whose low significand bits happen to be zero; any other
// atom is flagged (MD_TAG_OFFGRID).  The difference X_j - X_i is then the
// exact separation x_j - x_i (which the FP64 subtraction also yields
// exactly here), below 2^60 in magnitude for pairs closer than half the
// box: the compacted FP64 kernel forms separations, r^2 and force
// contributions from it with integer instructions.
struct __align__(32) XFix {
  long long x, y, z;
  long long w;  // the atom's tag (as md_tag_of(x4)) | F << 32
};

// ---- context -----------------------------------------------------------------
struct GraphKey {
  int m;        // force/integrate pairs in the segment
  int last_k2;  // segment ends with the final half kick
  bool operator<(const GraphKey& o) const {
    return m != o.m ? m < o.m : last_k2 < o.last_k2;
  }
};

struct md_ctx {
  // parameters
  int64_t n;
  int nt;
  int list_kind, precision, rebuild_every, tpa;
  int check_disp;  // also rebuild when some atom moved more than skin/2 (checked per step)
  int carve;    // preferred shared-memory carveout (%) of the pair kernel; -1 default
  int compact;  // FP64: 0 = per-atom loop (md_pair.cuh), 1 = warp-compacted kernel
                // (md_pair_q.cuh) with FP64 reductions, 2 = warp-compacted with
                // fixed-point reductions
  int time_pair;           // md_time_pair_kernel: segments without graphs, events
                           // around every pair launch
  cudaEvent_t* pair_ev;    // 2 * MD_PAIR_TIMING_MAX events (start, stop), or NULL
  int pair_ev_used;        // event pairs recorded since the last enable
  int qu;       // list entries per phase-1 round of the force-only compacted
                // fixed-point kernel (1 or 2; md_autotune picks it)
  int persist;  // 1 = persistent per-SM tile scheduling of the pair kernel;
                // 2 = the same, and one cooperative launch per step (kick,
                // drift and forces; md_step_fused.cu)
  int nsm;      // streaming multiprocessors of the device
  int* tile_ctr;  // per-SM tile counters of the persistent pair kernel
  double skin, dt, rlist;
  double eps[MD_MAX_TYPES * MD_MAX_TYPES], sigma[MD_MAX_TYPES * MD_MAX_TYPES];
  double rc[MD_MAX_TYPES * MD_MAX_TYPES], mass[MD_MAX_TYPES];
  double filt_e;                // FP32 filter error bound on |d| (host, from the boxes)
  XGrid xgrid;                  // grid of the hi parts of the position splits
  int coul;                     // lj/cut/coul/cut: the Coulomb term is on
  double qtype[MD_MAX_TYPES];   // per-type charges
  double qqrd2e, rc_coul;
  double dtf[MD_MAX_TYPES];  // 0.5 dt / m per type
  PairCoef coef1;            // coefficients when nt == 1
  Geo geo;
  int nrep;                  // replicas
  RepGeo* rep;               // device, nrep
  RepGeo* rep_host;          // host copy
  int64_t* rep_off_host;     // host, nrep + 1 atom offsets
  int64_t ncell;
  cudaStream_t stream;
  int own_stream;  // the context created the stream (caller passed NULL)

  // atom state in cell-sorted order (fixed pointers: graphs capture them);
  // sorting never moves an atom out of its replica's range
  double4_32a* x4;  // x, y, z, tag bits in w
  double* v;        // SoA: vx[n], vy[n], vz[n]
  double* f;        // SoA: fx[n], fy[n], fz[n]
  unsigned long long* fix;  // SoA 3n fixed-point force accumulators (FP64 compact == 2,
                            // and every mixed form); zero between pair launches
  int32_t* id;      // caller index of each sorted atom
  XSplit* xs;       // double-float split of x4 (build filter, mixed gathers)
  XSplit* xb;       // split of the positions at the last build (displacement)
  XFix* xq;         // FP64 contexts: fixed-point positions (valid where xs's tag has no
                    // MD_TAG_OFFGRID); NULL for mixed precision
  int32_t* cell;    // global cell index of each sorted atom
  int32_t* tag0;    // tags in the caller's order
  PairCoef* coef;   // nt*nt coefficients (device)
  float* cut_hi_dev;  // Geo::cut_hi on the device
  void* vcoef;      // nt*nt adjoint coefficients (device, VjpCoef)

  // rebuild scratch
  double4_32a* x4_alt;
  double* v_alt;
  double* f_alt;
  int32_t* id_alt;
  int32_t *cnt, *start, *rank, *perm, *cell_alt;
  int64_t* scan_tmp;  // tile sums of the scans
  int64_t scan_tmp_n;

  // neighbor list: tiles of 32 atoms, column-major inside a tile:
  // entry k of atom i at nbr[(i/32)*maxneigh*32 + k*32 + i%32].  A row holds
  // the pairs inside rc at build time ("inner") at k = 0 .. nin-1 and the
  // skin pairs at k = maxneigh-1 down to maxneigh-nsk.
  int32_t* numneigh;  // nin[n] then nsk[n]
  int32_t* nbr;
  int32_t maxneigh;
  int64_t nbr_alloc;  // int32 entries allocated

  // reductions: per replica MD_EV_STRIDE doubles:
  // [0] E_pot, [1..6] W, [7] pairs within rc, [8] E_kin
  double* ev;          // device, nrep * MD_EV_STRIDE
  double* ev_host;     // pinned, nrep * MD_EV_STRIDE
  double* evs;         // device, nrep * ev_spread rows of MD_EV_STRIDE: the kernels'
                       // atomics land here, spread over rows, and k_ev_fold adds
                       // them into ev (leaving them zero)
  int ev_spread;       // rows per replica: 128 / nrep, at least 1
  unsigned int* dmax;  // [0] max displacement^2 bits, [1] max count,
                       // [2] max stencil candidates of an atom (last build),
                       // [3] displacement^2 of a state loaded with the list kept,
                       // [4] that state changed some position (0/1),
                       // [5] a fused step's grid barrier timed out (0/1),
                       // [6], [7] that barrier's arrivals and generation
  double* h_pinned;    // small pinned host mirror (16 doubles)
  int64_t* i64_tmp;    // device int64 scratch (counts)

  // host staging for MD_MEM_HOST
  double* stage;  // device, 6n doubles

  // adjoint buffers (allocated on first use)
  double4_32a* adj_c;    // cotangent of the forces, sorted order
  double* adj_xbar;      // SoA 3n, sorted order
  double* adj_vbar;      // SoA 3n, sorted order
  double* adj_carry;     // caller order: xbar, vbar, cotangent (9n)
  double4_32a* seg_x;    // positions of one checkpoint segment, sorted
  int64_t seg_cap;       // positions seg_x holds
  double* gbar;          // 2 nt^2 parameter derivatives
  unsigned long long* fmax_bits;  // steepest descent: max |F| as bits

  // graphs
  std::map<GraphKey, std::pair<cudaGraphExec_t, int>>* graphs;

  // counters
  int64_t step, builds, dangerous, launches;
  int32_t max_count;
  int64_t pairs_in_range;  // at the last md_energy
};

// ---- entry points of the translation units ---------------------------------
// md_neigh.cu
int md_rebuild(md_ctx* c);  // wrap, sort, build (+grow)
int md_scan_i32(md_ctx* c, const int32_t* in, int32_t* out, int64_t n);
int md_scan_i64(md_ctx* c, const int32_t* in, int64_t* out, int64_t n);
int md_list_entries(md_ctx* c, int64_t* total);
int md_list_to_csr(md_ctx* c, int64_t* offsets, int32_t* idx);
void md_drop_graphs(md_ctx* c);

// md_capi.cu
int md_launch_pair(md_ctx* c, int ev, int tpa);
// step-segment form: f (and the fixed-point sums) are already zero, and the
// next integrator launch folds the fixed-point sums
int md_launch_pair_step(md_ctx* c);
int md_pair_accumulates(const md_ctx* c);  // the pair launch adds into f (needs f = 0)
int md_pair_fixed(const md_ctx* c);        // the pair launch leaves sums in fix
int md_launch_fix_finalize(md_ctx* c);  // md_integrate.cu
int md_fresh_start(md_ctx* c);
int md_step_fused_ok(const md_ctx* c);
// MD_ETIMEOUT if a fused step's grid barrier gave up (h_pinned[14] holds the
// device word, copied before the caller's synchronization)
static inline int md_barrier_status(const md_ctx* c) {
  unsigned int w;
  __builtin_memcpy(&w, (const char*)(c->h_pinned + 14), sizeof(w));
  return w ? MD_ETIMEOUT : MD_OK;
}
// qq, rc_coul: the Coulomb term (rc_coul <= 0: none)
void md_set_coef(PairCoef& pc, double eps, double sigma, double rc, double qq = 0.0,
                 double rc_coul = 0.0);
int md_upload_coef(md_ctx* c);  // coefficients, FP32 filter bounds, single-type copy

// md_integrate.cu
enum { MD_K1 = 0, MD_K21 = 1, MD_K2 = 2 };
// fold: add the fixed-point sums into f first (and zero them); zero: K1/K21
// leave f = 0 for a pair launch that accumulates
int md_launch_integrate(md_ctx* c, int mode, int fold = 0, int zero = 0);
int md_launch_kinetic(md_ctx* c);
int md_launch_virial_atoms(md_ctx* c);  // sum_a (x_a - c) (x) F_a into evs words 1..6
int md_launch_ev_fold(md_ctx* c);       // ev += the sums of the evs rows; evs = 0
int md_launch_load_state(md_ctx* c, const double* x, const double* v);
int md_launch_store_state(md_ctx* c, double* x, double* v, double* f);
// caller order into the current sorted order, list kept; max displacement
// since the last build into dmax[0] and dmax[3]
int md_launch_load_keep(md_ctx* c, const double* x, const double* v);

static inline int64_t md_blocks(int64_t work, int block = MD_BLOCK) {
  return (work + block - 1) / block;
}
