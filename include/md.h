/*
 * md.h -- C ABI of libmd.so, the GB300 (sm_103a) Lennard-Jones lj/cut
 * short-range step: binned neighbor-list build with skin, pair
 * force/energy/virial kernel, fused velocity-Verlet NVE update.
 *
 * The physics is Eq. 1 of arXiv 2508.13523 (Sec. 4),
 *   E = sum_{i<k, r_ik < rc} 4 eps [ (sigma/r_ik)^12 - (sigma/r_ik)^6 ],
 * with forces the pairwise derivative of E (Sec. 4) summed over a neighbor
 * list built at rc + skin and rebuilt periodically (Sec. 4), either as a
 * half list with Newton's third law resolved by atomics or as a full list
 * with every pair computed twice (Sec. 4.1).  Units are reduced LJ units,
 * k_B = 1.  The box is orthorhombic and periodic with origin 0.
 *
 * Conventions for every entry point
 *  - Return value: MD_OK (0) or a negative MD_E* code; md_strerror() names
 *    it.  No entry point aborts, throws or traps on the device.
 *  - Pointers marked "device" must be device memory of the current CUDA
 *    device; "host" pointers are ordinary (preferably pinned) host memory.
 *    Per-atom arrays are in the caller's atom order, row-major:
 *    positions/velocities/forces are n_atoms x 3 doubles, types n_atoms
 *    int32 in [0, n_types).
 *  - The context owns every buffer it allocates; caller buffers are only
 *    read or written during the call (asynchronously on the context's
 *    stream for device pointers: keep them alive until the stream reaches
 *    that point).  Internally atoms are kept sorted by cell; the caller's
 *    order is restored on every copy out.
 *  - All work is enqueued on the stream given to md_create.  Calls that
 *    return host-visible results or must size buffers synchronize it; each
 *    such call says so.
 *  - A context is not thread safe; use one host thread per context.
 */
#ifndef LJMD_MD_H
#define LJMD_MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define MD_OK 0
#define MD_EINVAL (-1)      /* invalid argument (sizes, box, parameters)       */
#define MD_ENOMEM (-2)      /* device or host allocation failed                */
#define MD_ENEIGH (-3)      /* neighbor capacity could not be grown enough     */
#define MD_ECUDA (-4)       /* a CUDA runtime call failed                      */
#define MD_ENONFINITE (-5)  /* non-finite energy or virial                     */
#define MD_ETIMEOUT (-6)    /* a bounded device-side wait expired              */

/* ---- enumerations -------------------------------------------------------- */
#define MD_LIST_FULL 0  /* every pair in both atoms' lists, no atomics (Sec. 4.1) */
#define MD_LIST_HALF 1  /* every pair once, f_j updated by atomics (Sec. 4.1)     */

#define MD_PREC_FP64 0   /* all pair arithmetic in FP64                          */
#define MD_PREC_MIXED 1  /* FP32 pair arithmetic; every FP32 force
                            contribution summed exactly as a 64-bit
                            fixed-point count of 2^-44 and folded into the
                            FP64 force once per atom (order-independent,
                            within contributions x 2^-44 of the exact sum);
                            energy and virial summed in FP64; FP64 positions,
                            velocities and integration; a pair within 2^-18
                            (relative) of a cutoff in FP32 r^2 is decided on
                            an FP64 r^2, so both precisions sum over the same
                            pairs                                              */

#define MD_ENERGY 1  /* md_compute_forces: also accumulate the potential energy */
#define MD_VIRIAL 2  /* md_compute_forces: also accumulate the virial tensor    */

#define MD_MEM_DEVICE 0  /* the pointers given are device memory */
#define MD_MEM_HOST 1    /* the pointers given are host memory   */
#define MD_MEM_KEEP_LIST 2 /* md_set_state: keep the list when it is still valid */

#define MD_MAX_TYPES 8
#define MD_THERMO_N 10

/* ---- parameters ---------------------------------------------------------- */
typedef struct md_params {
  int64_t n_atoms;          /* >= 1 and < 2^31                                 */
  int32_t n_types;          /* 1 .. MD_MAX_TYPES                               */
  int32_t list_kind;        /* MD_LIST_FULL or MD_LIST_HALF                    */
  double box[3];            /* edge lengths L_x, L_y, L_z > 0; periodic        */
  const double* eps;        /* host, n_types^2 row-major, symmetric, > 0      */
  const double* sigma;      /* host, n_types^2 row-major, symmetric, > 0      */
  const double* rc;         /* host, n_types^2 row-major, symmetric, > 0;
                               every rc < L/2 along every axis (single image) */
  const double* mass;       /* host, n_types, > 0                              */
  double skin;              /* >= 0; the list holds pairs with r < max(rc)+skin */
  double dt;                /* time step                                       */
  int32_t precision;        /* MD_PREC_FP64 or MD_PREC_MIXED                   */
  int32_t rebuild_every;    /* >= 1: rebuild the list after the drift of every
                               step s with (s+1) % rebuild_every == 0         */
  int32_t threads_per_atom; /* 1, 2, 4, 8, 16 or 32; 0 = pick by timing        */
  int32_t max_neigh;        /* initial list capacity per atom; 0 = estimate.
                               The capacity grows automatically.               */
  int32_t check_disp;       /* 0: rebuild only every rebuild_every steps (the
                               displacement check is reported, as "dangerous
                               builds"); 1: also rebuild before any step at
                               which some atom has moved more than skin/2
                               since the last build (checked after every
                               drift; one host synchronization per step)      */
} md_params;

typedef struct md_ctx md_ctx;

/* Counters and settings of a context (md_get_stats). */
typedef struct md_stats {
  int64_t step;             /* steps taken since md_create / md_set_state      */
  int64_t builds;           /* neighbor-list builds                            */
  int64_t dangerous_builds; /* builds at which some atom had moved more than
                               skin/2 since the previous build, so that the
                               old list may have missed pairs (always 0 with
                               check_disp)                                     */
  int64_t kernel_launches;  /* kernels launched by this context (graph nodes
                               counted per graph launch)                       */
  int64_t list_entries;     /* entries in the current list (sum of counts)     */
  int32_t max_neigh;        /* current capacity per atom                       */
  int32_t max_count;        /* largest per-atom count at the last build        */
  int32_t cells[3];         /* cell grid (1 along an axis too short for 3)     */
  int32_t threads_per_atom; /* in use                                          */
  int32_t carveout;         /* preferred shared-memory carveout of the pair
                               kernel in percent, -1 = driver default         */
  int32_t compacted;        /* FP64: 0 per-atom pair kernel, 1 warp-compacted
                               kernel with FP64 reductions, 2 warp-compacted
                               kernel with fixed-point reductions            */
  int32_t persistent;       /* 1 if the pair kernel schedules tiles per SM; 2 if,
                               besides, each step is one cooperative launch   */
  double max_disp;          /* largest displacement since the last build (FP64
                               contexts: an upper bound within 4 grid steps of
                               the split, ~6e-5 at L = 168; mixed: FP32)      */
  int64_t pairs_in_range;   /* pairs with r < rc at the last md_energy call    */
  int32_t n_replicas;       /* boxes in the context (1 for md_create)          */
  int64_t total_cells;      /* cells over all boxes                            */
  int32_t coulomb;          /* 1 if the lj/cut/coul/cut style is on (md_set_coulomb) */
  int32_t phase1_entries;   /* list entries each lane takes per round of the
                               force-only pair kernel's walk: 1 or 2 for the
                               FP64 compacted fixed-point kernel (picked by
                               md_autotune or md_set_kernel), 2 for the mixed
                               kernel, 1 for the others                       */
} md_stats;

/* ---- single box ---------------------------------------------------------- */

/* Create a context for one periodic box and load its initial state.
 *   x, v: device, n_atoms x 3 positions and velocities (copied);
 *   type: device, n_atoms int32 (copied);
 *   stream: cudaStream_t to enqueue all work on; NULL makes the context
 *           create (and later destroy) its own blocking stream.
 * Wraps the positions into the box, sorts atoms by cell, builds the list and
 * computes the forces.  Synchronizes the stream.  On failure *out is NULL.
 * Passages: the state the force step needs (positions, types, per-type
 * eps and sigma, cutoffs) is that of Eq. 1 (Sec. 4); the list built at
 * rc + skin is the periodically updated neighbor list of Sec. 4; the
 * context keeps one device-resident copy of every per-atom array, the GPU
 * side of the host/device data of Sec. 3.2, and copies to or from the
 * caller only when asked (md_set_state, md_get_state). */
int md_create(const md_params* params, const double* x, const double* v,
              const int32_t* type, void* stream, md_ctx** out);

/* ---- batched replicas ---------------------------------------------------- */

/* Create one context for n_replicas independent periodic boxes that share
 * the parameters (types, eps, sigma, rc, masses, skin, dt, list kind,
 * precision, cadence) but not their size: box r owns the caller's atoms
 * rep_offset[r] .. rep_offset[r+1]-1 and has edges boxes[3r..3r+2].  Every
 * kernel of a step then runs once over all atoms of all boxes, so uneven
 * boxes share one launch per kernel (and one CUDA graph per segment).
 *   params->n_atoms: total atoms, = rep_offset[n_replicas];
 *   params->box: ignored;
 *   n_replicas: 1 .. 2^23 - 1;
 *   rep_offset: host, n_replicas + 1 increasing int64, rep_offset[0] = 0;
 *   boxes: host, n_replicas x 3 edges, each > 2 max(rc);
 *   x, v, type, stream, out: as md_create (atoms in the caller's order).
 * A box shorter than 3 (max rc + skin) along an axis has one cell along it
 * and its atoms are all candidates along that axis.  All other entry points
 * accept a batch context; md_energy sums over boxes, md_energy_replicas
 * reports each.
 * Passages: each box is the system of Eq. 1 (Sec. 4); batching answers the
 * saturation the paper reports for one GPU (Sec. 5.1, LJ throughput vs
 * atom count: small systems do not fill a GPU, which Sec. 4.1 also
 * addresses with parallelism over neighbors). */
int md_create_batch(const md_params* params, int32_t n_replicas, const int64_t* rep_offset,
                    const double* boxes, const double* x, const double* v,
                    const int32_t* type, void* stream, md_ctx** out);

/* Free every resource of the context (NULL is accepted).  The paper's
 * counterpart is the end of a run; it defines no separate operation. */
void md_destroy(md_ctx* ctx);

/* Replace positions and velocities (types and parameters stay), then wrap,
 * sort, rebuild the list and recompute forces as md_create does; the step
 * counter restarts at 0.  mem: MD_MEM_DEVICE or MD_MEM_HOST for x and v,
 * optionally ORed with MD_MEM_KEEP_LIST: if no atom is farther than skin/2
 * from where it was at the last build (positions unwrapped since then, as
 * md_get_state returns them), the atom order and the neighbor list are kept
 * and only the forces are recomputed (the test is conservative: in FP64
 * contexts it uses an upper bound of each displacement, see max_disp; the
 * list then still holds every pair
 * within rc, as after a build) -- not even they when every position equals,
 * bit for bit, the one the context holds (a state read by md_get_state and
 * written back with new velocities only); otherwise the call starts afresh
 * as without the flag.  Host input is staged through a device buffer on the
 * stream.  Synchronizes.
 * Passages: host-to-device transfer of the per-atom state on demand, as the
 * data synchronization of Sec. 3.2; the list is kept only while it is still
 * the list of Sec. 4 (no pair can have moved in from beyond rc + skin). */
int md_set_state(md_ctx* ctx, const double* x, const double* v, int32_t mem);

/* Copy the current state out in the caller's atom order.  Any of x, v, f may
 * be NULL.  With MD_MEM_HOST the call synchronizes the stream.
 * Passages: device-to-host transfer on demand (Sec. 3.2); f is the force of
 * Eq. 1's derivative (Sec. 4) at the current positions. */
int md_get_state(md_ctx* ctx, double* x, double* v, double* f, int32_t mem);

/* Wrap positions, sort atoms by cell and rebuild the neighbor list now
 * (Sec. 4: the list is periodically updated).  Grows the capacity and
 * rebuilds if an atom has more neighbors than fit.  Synchronizes. */
int md_build_neighbors(md_ctx* ctx);

/* Compute forces on the current list (Eq. 1 derivative, Sec. 4; half or full
 * list, Sec. 4.1).  flags: MD_ENERGY | MD_VIRIAL also accumulate the
 * potential energy / virial for md_energy.  Asynchronous. */
int md_compute_forces(md_ctx* ctx, int32_t flags);

/* Advance nsteps of velocity Verlet (NVE), rebuilding the list on the
 * cadence of params.rebuild_every.  Steps between rebuilds run as one CUDA
 * graph launch; each rebuild synchronizes once to check list capacity. */
int md_step(md_ctx* ctx, int64_t nsteps);

/* Thermodynamic state at the current positions and velocities (summed over
 * all boxes of a batch; the temperature then counts 3 N_r - 3 degrees of
 * freedom per box):
 * out[0] potential energy (Eq. 1), out[1] kinetic energy, out[2] total,
 * out[3] temperature 2 KE / (3N - 3), out[4..9] virial W_xx, W_yy, W_zz,
 * W_xy, W_xz, W_yz with W_ab = sum over pairs of fpair d_a d_b (summed as
 * sum over atoms of x_a F_b, less the terms of the pairs taken through a
 * periodic image).  In FP64 contexts with one type and Eq. 1 alone the
 * potential energy is summed as trace(W) / 12 - (lj4 / 2) sum r^-6, equal
 * to Eq. 1's sum since lj1 = 12 lj3 and lj2 = 6 lj4.  Recomputes the forces with energy and virial.
 * Synchronizes.
 * Returns MD_ENONFINITE if any value is not finite. */
int md_energy(md_ctx* ctx, double out[MD_THERMO_N]);

/* The same ten quantities for every box of the context: out is host memory
 * of n_replicas x MD_THERMO_N doubles, box r at out[r * MD_THERMO_N].
 * Synchronizes.  MD_ENONFINITE if any value is not finite.  Passage: Eq. 1
 * per box (Sec. 4); the batch itself has no counterpart in the paper. */
int md_energy_replicas(md_ctx* ctx, double* out);

/* Number of entries of the current neighbor list, *total, and the largest
 * per-atom count, *max_count (either may be NULL).  Synchronizes.
 * Passage: the list of Sec. 4 in its half or full kind (Sec. 4.1); counts
 * are 64-bit because list offsets outgrow 32 bits at scale (App. B). */
int md_neighbor_count(md_ctx* ctx, int64_t* total, int32_t* max_count);

/* The current neighbor list in the caller's atom order and numbering, as
 * CSR: offsets (device, n_atoms + 1 int64) and idx (device, *total int32
 * from md_neighbor_count).  Full list: j appears in i's row iff the pair is
 * within max(rc) + skin at the last build.  Half list: each such pair
 * appears once, in the row of the atom that owns it.  Row order is
 * unspecified.  Asynchronous.  Passage: the half and full list semantics of
 * Sec. 4.1 (each pair once, or in both atoms' rows); 64-bit offsets as
 * App. B recommends. */
int md_get_neighbors(md_ctx* ctx, int64_t* offsets, int32_t* idx);

/* Time the pair kernel for every allowed threads-per-atom value (Sec. 4.1:
 * parallelism over neighbors) and, in FP64, for the warp-compacted kernel
 * (in-range pairs queued per warp so that all 32 lanes do FP64 work; Sec.
 * 4.1's divergence) with either force summation (see md_set_kernel) on the
 * current list, the fixed-point one with one or two list entries per lane
 * per filter round (compacted 2 and 3), each with one block per tile and
 * with persistent per-SM tile scheduling (md_set_kernel's persistent 0 and
 * 1); keep the fastest.
 * The carveout keeps the driver's default and steps stay separate launches
 * (persistent 2 is measured slower on GB300); md_set_kernel sets them.
 * Synchronizes. */
int md_autotune(md_ctx* ctx);

/* Second pair style, lj/cut/coul/cut: Eq. 1 plus a cut Coulomb term.  The
 * paper's pair styles share one two-body base with the same neighbor lists
 * and force accumulation (Sec. 4); this style reuses ours.  For a pair of
 * types (a, b) at distance r < rc_coul the pair energy gains
 * qqrd2e q_a q_b / r and the force on atom i gains
 * qqrd2e q_a q_b (x_i - x_j) / r^3 (minimum image).  Charges are per type:
 * q (host, n_types doubles, copied).  rc_coul must be > 0 and at most the
 * largest rc (the lists are built at max rc + skin).  q == NULL turns the
 * term off.  The FP64 form runs the warp-compacted kernel (compacted 1 or 2;
 * compacted 0 becomes 2), the mixed form threads_per_atom 1, 2 or 4 (a
 * larger value becomes 2).  Forces are recomputed.  The adjoint entry points
 * return MD_EINVAL while the term is on (their derivative is of Eq. 1 only).
 * MD_EINVAL for a bad argument.  Synchronizes. */
int md_set_coulomb(md_ctx* ctx, const double* q, double rc_coul, double qqrd2e);

/* Fix the pair kernel's configuration instead of the tuner's choice:
 * threads_per_atom in {1,2,4,8,16,32}; carveout -1 (driver default) or
 * 0..100 (% shared memory); compacted 1 selects the warp-compacted FP64
 * kernel (FP64 contexts, threads_per_atom 1) summing forces with FP64
 * atomics, compacted 2 the same kernel summing each force contribution,
 * rounded to a multiple of 2^-44, exactly in 64-bit integers (the result
 * does not depend on the order of the additions and lies within
 * contributions x 2^-45 of the exact FP64 sum; a contribution too large for
 * that range is added in FP64), compacted 3 the compacted 2 kernel whose
 * filter takes two list entries per lane per round, their loads in flight
 * together (Eq. 1 alone; md_get_stats then reports compacted 2 and
 * phase1_entries 2); persistent 1 launches one
 * resident grid whose blocks take tiles of cell-sorted atoms from the range
 * of the SM they run on (neighbor positions stay in that SM's L1), 0 one
 * block per tile; persistent 2 (FP64 contexts with compacted 2, Eq. 1
 * alone) makes md_step run each step between rebuilds as one cooperative
 * launch over all atoms of all boxes: the kick and drift of every atom, a
 * grid-wide barrier, then the forces with persistent tile scheduling (the
 * barrier's wait is bounded: if it ever gives up, the next rebuild or
 * md_synchronize returns MD_ETIMEOUT).  MD_EINVAL otherwise. */
int md_set_kernel(md_ctx* ctx, int32_t threads_per_atom, int32_t carveout, int32_t compacted,
                  int32_t persistent);

/* Counters and settings; synchronizes the stream.
 * Passages: the list statistics (entries, capacity, builds) describe the
 * neighbor list of Sec. 4 and its half/full kind (Sec. 4.1); the kernel
 * settings are the threads-per-atom choice of Sec. 4.1 and the L1/shared
 * memory carveout studied in Sec. 4.4. */
int md_get_stats(md_ctx* ctx, md_stats* out);

/* Pair-kernel timing inside md_step (measurement support; the paper has no
 * counterpart).  md_time_pair_kernel(ctx, 1) clears the record and, until
 * md_time_pair_kernel(ctx, 0), makes md_step launch each segment's kernels
 * directly instead of as a CUDA graph, with a CUDA event recorded on the
 * context's stream before and after every pair-kernel launch (the first
 * MD_PAIR_TIMING_MAX launches; in the one-launch-per-step schedule the
 * events bracket the combined step launches).  The kernels and their
 * results are the same as with the graphs.  md_pair_kernel_time
 * synchronizes the stream and returns in *total_ms the summed elapsed time
 * of the recorded launches and in *launches their number.  MD_EINVAL for a
 * null context or output or an enable other than 0 or 1; MD_ENOMEM if the
 * events cannot be created. */
#define MD_PAIR_TIMING_MAX 1024
int md_time_pair_kernel(md_ctx* ctx, int32_t enable);
int md_pair_kernel_time(md_ctx* ctx, double* total_ms, int64_t* launches);

/* Wait for all work of the context and report any asynchronous error.  The
 * paper has no counterpart (a runtime call). */
int md_synchronize(md_ctx* ctx);

/* Static description of a return code.  The paper has no counterpart. */
const char* md_strerror(int code);

/* ---- gradients and relaxation ---------------------------------------------- */

/* Replace the per-type-pair eps and sigma (host, n_types^2 row-major,
 * symmetric, > 0); the cutoffs rc keep their values from md_create.  Takes
 * effect from the next force evaluation.  Synchronizes.  Passage: eps and
 * sigma are the coefficients of Eq. 1 (Sec. 4), which may vary between
 * systems. */
int md_set_lj(md_ctx* ctx, const double* eps, const double* sigma);

/* Vector-Jacobian product of the forces at the current positions (the
 * adjoint of the pairwise derivative of Eq. 1, Sec. 4), over the current
 * list:
 *   cot:  device, n_atoms x 3, the cotangent dL/dF (caller order);
 *   xbar: device, n_atoms x 3, receives dL/dx = J_F(x)^T cot (overwritten);
 *   gbar: host, 2 n_types^2, receives dL/deps then dL/dsigma as symmetric
 *         tables: entries (a,b) and (b,a) both hold the derivative with
 *         respect to the one parameter of the unordered type pair {a,b}.
 * The cutoffs are constants.  FP64 or mixed precision as the context.
 * Synchronizes. */
int md_force_vjp(md_ctx* ctx, const double* cot, double* xbar, double* gbar);

/* Forward pass for reverse mode through nsteps velocity-Verlet steps:
 * restarts from (x0, v0) (device, caller order, as md_set_state) and stores
 * checkpoints at steps 0, every, 2 every, ..., and nsteps:
 *   ckpt_x, ckpt_v: device, (ceil(nsteps/every) + 1) x n_atoms x 3 each;
 *   f_final: device, n_atoms x 3, forces at the final positions.
 * every must equal params.rebuild_every (each segment then uses the one list
 * built at its checkpoint).  Leaves the context at step nsteps.  Passage:
 * the forces are Eq. 1's derivative (Sec. 4) on the periodically rebuilt
 * list (Sec. 4); the integrator and the checkpoints have no counterpart in
 * the paper. */
int md_traj_forward(md_ctx* ctx, int64_t nsteps, int32_t every, const double* x0,
                    const double* v0, double* ckpt_x, double* ckpt_v, double* f_final);

/* Reverse mode through the run stored by md_traj_forward, for a loss that
 * depends on the final forces only:
 *   cot_final: device, n_atoms x 3, dL/dF at the final positions;
 *   x0bar, v0bar: device, n_atoms x 3, receive dL/dx0 and dL/dv0;
 *   gbar: host, 2 n_types^2, receives dL/deps and dL/dsigma (as
 *         md_force_vjp).
 * Each segment is recomputed from its checkpoint and differentiated
 * backwards (velocity-Verlet adjoint, force VJP per evaluation).  Leaves the
 * context at the first checkpoint.  Synchronizes.  Passage: the adjoint of
 * Eq. 1's derivative (Sec. 4) per force evaluation; reverse mode itself has
 * no counterpart in the paper. */
int md_traj_vjp(md_ctx* ctx, int64_t nsteps, int32_t every, const double* ckpt_x,
                const double* ckpt_v, const double* cot_final, double* x0bar, double* v0bar,
                double* gbar);

/* Steepest descent: nsteps of x <- x + alpha F / max_i |F_i|, with the list
 * rebuilt on the context's cadence (choose alpha * rebuild_every < skin / 2),
 * then a fresh build and forces.  Velocities are untouched.  Passage: the
 * forces of Eq. 1 (Sec. 4); the relaxation prepares a workload and has no
 * counterpart in the paper. */
int md_minimize(md_ctx* ctx, int64_t nsteps, double alpha);

/* ---- diagnostics ------------------------------------------------------------ */

/* The device reciprocal and reciprocal square root that every pair kernel
 * applies to r^2 (Eq. 1 and its derivative need r^-2, r^-6 and, for the
 * Coulomb style, 1/r; Sec. 4), evaluated elementwise:
 *   a:     device, n doubles, each > 0 and normal (the kernels' domain is
 *          r^2 inside the cutoff);
 *   rcp:   device, n doubles, receives 1/a[i] (or NULL);
 *   rsqrt: device, n doubles, receives 1/sqrt(a[i]) (or NULL);
 *   stream: cudaStream_t to enqueue on (NULL = legacy).
 * Both start from the hardware's approximate seed and refine it with one
 * cubic series round (Markstein); the tests bound their error in ulps of the
 * correctly rounded values.  Asynchronous.  MD_EINVAL for n < 0 or a NULL
 * input with n > 0. */
int md_eval_recip(int64_t n, const double* a, double* rcp, double* rsqrt, void* stream);

/* The grid-wide barrier of the one-launch-per-step schedule (md_set_kernel
 * persistent 2), on its own: a cooperative launch of `blocks` blocks
 * (1 .. 1024) whose barrier waits for blocks + missing arrivals (missing 0
 * or 1), each block giving up after limit_ms (0 < limit_ms <= 10000).  With
 * missing = 1 no barrier can complete: every block's wait runs out, sets
 * the error word and returns, and the call reports it -- the failure path
 * of a fused step, exercised without a fault or a hang.  The paper has no
 * counterpart (its steps are separate kernels).
 *   word: device, 3 unsigned ints of scratch (zeroed by the call);
 *   stream: cudaStream_t to enqueue on (NULL = legacy).
 * Returns MD_OK if the barrier completed, MD_ETIMEOUT if it gave up,
 * MD_EINVAL for bad arguments.  Synchronizes the stream. */
int md_eval_barrier(int32_t blocks, int32_t missing, double limit_ms, unsigned int* word,
                    void* stream);

/* ---- allocation-free kinetic energy -------------------------------------- */

/* Largest n_atoms md_kinetic_noalloc accepts. */
#define MD_NOALLOC_MAX_ATOMS 4194304

/* Kinetic energy and temperature of velocities the caller holds, without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc when they need the number -- a
 * real-time loop that must not enter the allocator (which can synchronize
 * the device), or a framework whose allocator owns all device memory and
 * lends none to libraries.  Such callers cannot create an md_ctx, which
 * allocates its buffers.
 *   n_atoms: 1 .. MD_NOALLOC_MAX_ATOMS, else MD_EINVAL;
 *   v:       device, n_atoms x 3 velocities, row-major;
 *   type:    device, n_atoms int32 types, or NULL for all type 0; atoms
 *            whose type is outside [0, n_types) contribute nothing;
 *   n_types, mass: host, n_types (1 .. MD_MAX_TYPES) masses > 0;
 *   out:     device, 2 doubles: out[0] = sum 0.5 m v^2,
 *            out[1] = 2 out[0] / (3 n_atoms - 3) (0 for one atom);
 *   stream:  cudaStream_t the two kernels are enqueued on (NULL = legacy).
 * Asynchronous; calls no cudaMalloc, cudaFree or allocating library routine.
 * Scratch: per-block partial sums live in one fixed 32 KB array in device
 * memory (static storage of libmd.so, held by every GPU that loads the
 * library until the process exits).  Every call overwrites the slots it
 * reads before reading them, so nothing needs clearing between calls, but
 * all calls share that one array: calls whose kernels may overlap on the GPU
 * (different streams without ordering, or several host threads) race and
 * must be serialized by the caller.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current, and looks it up again when the device's CUDA context has been
 * replaced since (cudaDeviceReset); make that first call before starting
 * any stream capture. */
int md_kinetic_noalloc(int64_t n_atoms, const double* v, const int32_t* type,
                       int32_t n_types, const double* mass, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LJMD_MD_H */
