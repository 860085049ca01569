/*
 * ljmd_oracle.c -- plain, slow, FP64 CPU oracle for the Lennard-Jones
 * lj/cut short-range step (arXiv 2508.13523, Sec. 4 and Sec. 4.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this file
 * or the library built from it: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py do.  It shares no code, header,
 * table or constant with the CUDA library; the two agree only because both
 * follow the same written definitions below.
 *
 * What it computes
 *   Energy, Eq. 1:  E = sum over pairs i<k with r_ik < rc of
 *                   4 eps [ (sigma/r_ik)^12 - (sigma/r_ik)^6 ]
 *   Forces, Sec. 4: the pairwise sum of the derivative of E, i.e. for a pair
 *                   with d = x_i - x_k (minimum image),
 *                   F_i += fpair * d,  F_k -= fpair * d,
 *                   fpair = -(dU/dr)/r = 24 eps s6 (2 s6 - 1) / r^2,
 *                   s6 = (sigma^2/r^2)^3.
 *   Virial:         W_ab = sum over pairs of fpair * d_a * d_b.
 *   Neighbor list:  Sec. 4 (a list built and periodically updated) and
 *                   Sec. 4.1 (half lists: each pair once).  Here it is the set
 *                   of pairs i<k whose minimum-image distance is below
 *                   rlist = max(rc) + skin; built brute force and with a cell
 *                   list, which must agree exactly.
 *   Integrator:     velocity Verlet, NVE (not described in the paper).
 *   Second pair style (lj/cut/coul/cut; the paper's pair styles share one
 *   two-body base, Sec. 4): Eq. 1 plus a cut Coulomb term for a pair of
 *   types (a, b) at r < rc_coul, U = qq_ab / r, fpair = qq_ab / r^3, with
 *   qq_ab = qqrd2e q_a q_b from per-type charges.  A NULL qq table means
 *   plain Eq. 1.
 *
 * Readings fixed here (the paper is silent on them):
 *   - orthorhombic periodic box with origin 0; minimum image per component
 *     d -= L * rint(d / L) (round half to even);
 *   - squared distance r2 = fma(dz, dz, fma(dy, dy, dx*dx));
 *   - strict cutoffs: r2 < rc*rc, r2 < rlist*rlist;
 *   - wrap into the box only when the list is rebuilt:
 *     x -= L * floor(x / L), and a result equal to L becomes 0;
 *   - Verlet half kick v = fma(dtf, f, v) with dtf = 0.5*dt/m, drift
 *     x = fma(dt, v, x); the list is rebuilt (with a wrap) after the drift of
 *     every step s with (s+1) % rebuild_every == 0, counting steps from 0.
 *
 * Built with gcc -O2 -ffp-contract=off, single threaded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- geometry ---------------------------------------------------------- */

double orc_min_image(double d, double L) { return d - L * rint(d / L); }

/* Wrap every coordinate into [0, L). */
void orc_wrap(int64_t n, double *x, const double *box) {
  for (int64_t i = 0; i < n; i++)
    for (int a = 0; a < 3; a++) {
      double L = box[a];
      double w = x[3 * i + a] - L * floor(x[3 * i + a] / L);
      if (w == L) w = 0.0;
      x[3 * i + a] = w;
    }
}

/* Minimum-image separation d = x_k - x_i and its squared length. */
static double sep(const double *x, int64_t i, int64_t k, const double *box,
                  double d[3]) {
  for (int a = 0; a < 3; a++)
    d[a] = orc_min_image(x[3 * k + a] - x[3 * i + a], box[a]);
  return fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
}

/* ---- neighbor pairs ---------------------------------------------------- */

/* All pairs i<k with minimum-image r2 < rlist^2, in (i, k) lexicographic
 * order.  Writes at most cap pairs; returns the total count. */
int64_t orc_pairs_brute(int64_t n, const double *x, const double *box,
                        double rlist, int64_t cap, int32_t *pi, int32_t *pk) {
  double rl2 = rlist * rlist, d[3];
  int64_t m = 0;
  for (int64_t i = 0; i < n; i++)
    for (int64_t k = i + 1; k < n; k++)
      if (sep(x, i, k, box, d) < rl2) {
        if (m < cap) { pi[m] = (int32_t)i; pk[m] = (int32_t)k; }
        m++;
      }
  return m;
}

/* Cell count along one axis: the largest nc with cell edge >= rlist (with a
 * small guard so that rounding in the cell index cannot lose a pair). */
static int cells_along(double L, double rlist) {
  int nc = (int)floor(L / rlist);
  if (nc > 0 && L / nc - rlist < 1e-9 * L) nc--;
  return nc;
}

/* Same pair set as orc_pairs_brute, found with a linked-cell list: bins of
 * edge >= rlist, 27-cell stencil.  Falls back to brute force when any axis
 * has fewer than 3 cells (the stencil would visit a cell twice).  Pairs come
 * out as (min, max) in no particular order.  Returns the total count. */
int64_t orc_pairs_cells(int64_t n, const double *x, const double *box,
                        double rlist, int64_t cap, int32_t *pi, int32_t *pk) {
  int nc[3];
  for (int a = 0; a < 3; a++) nc[a] = cells_along(box[a], rlist);
  if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3)
    return orc_pairs_brute(n, x, box, rlist, cap, pi, pk);
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t *head = malloc(sizeof(int64_t) * ncell);
  int64_t *next = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int *cidx = malloc(sizeof(int) * 3 * (n > 0 ? n : 1));
  for (int64_t c = 0; c < ncell; c++) head[c] = -1;
  for (int64_t i = n - 1; i >= 0; i--) {
    int64_t lin = 0;
    for (int a = 0; a < 3; a++) {
      double L = box[a];
      double w = x[3 * i + a] - L * floor(x[3 * i + a] / L);
      int c = (int)floor(w / L * nc[a]);
      if (c < 0) c = 0;
      if (c >= nc[a]) c = nc[a] - 1;
      cidx[3 * i + a] = c;
      lin = lin * nc[a] + c;
    }
    next[i] = head[lin];
    head[lin] = i;
  }
  double rl2 = rlist * rlist, d[3];
  int64_t m = 0;
  for (int64_t i = 0; i < n; i++) {
    for (int ox = -1; ox <= 1; ox++)
      for (int oy = -1; oy <= 1; oy++)
        for (int oz = -1; oz <= 1; oz++) {
          int cx = (cidx[3 * i] + ox + nc[0]) % nc[0];
          int cy = (cidx[3 * i + 1] + oy + nc[1]) % nc[1];
          int cz = (cidx[3 * i + 2] + oz + nc[2]) % nc[2];
          int64_t lin = ((int64_t)cx * nc[1] + cy) * nc[2] + cz;
          for (int64_t k = head[lin]; k >= 0; k = next[k]) {
            if (k <= i) continue;
            if (sep(x, i, k, box, d) < rl2) {
              if (m < cap) { pi[m] = (int32_t)i; pk[m] = (int32_t)k; }
              m++;
            }
          }
        }
  }
  free(head); free(next); free(cidx);
  return m;
}

/* Full neighbor list of each sampled atom by a scan over all atoms:
 * out[s*cap_per + t] holds the t-th k (ascending) with r2 < rlist^2, k != i.
 * counts[s] receives the full count (entries beyond cap_per are dropped). */
void orc_neighbors_of(int64_t n, const double *x, const double *box,
                      double rlist, int64_t nsample, const int64_t *sample,
                      int64_t cap_per, int32_t *out, int64_t *counts) {
  double rl2 = rlist * rlist, d[3];
  for (int64_t s = 0; s < nsample; s++) {
    int64_t i = sample[s], m = 0;
    for (int64_t k = 0; k < n; k++) {
      if (k == i) continue;
      if (sep(x, i, k, box, d) < rl2) {
        if (m < cap_per) out[s * cap_per + m] = (int32_t)k;
        m++;
      }
    }
    counts[s] = m;
  }
}

/* ---- Eq. 1 and its derivative ------------------------------------------ */

/* Pair (i, k) of types (ti, tk) at squared distance r2 < rc^2: returns
 * fpair and stores the pair energy. */
static double lj_pair(double r2, double eps, double sigma, double *e) {
  double inv_r2 = 1.0 / r2;
  double s2 = sigma * sigma * inv_r2;
  double s6 = s2 * s2 * s2;
  *e = 4.0 * eps * (s6 * s6 - s6);
  return 24.0 * eps * s6 * (2.0 * s6 - 1.0) * inv_r2;
}

/* Cut Coulomb for a pair at squared distance r2 < rc_coul^2: returns
 * fpair = qq / r^3 and stores the pair energy qq / r. */
static double coul_pair(double r2, double qq, double *e) {
  double r = sqrt(r2);
  *e = qq / r;
  return qq / (r2 * r);
}

/* fpair and energy of the pair (either term may be out of range); returns 0
 * when neither term applies. */
static int pair_terms(double r2, int t, const double *eps, const double *sigma,
                      const double *rc, const double *qq, double rc_coul,
                      double *fpair, double *e) {
  int hit = 0;
  double fp = 0.0, en = 0.0, e1;
  if (r2 < rc[t] * rc[t]) {
    fp = lj_pair(r2, eps[t], sigma[t], &e1);
    en = e1;
    hit = 1;
  }
  if (qq && r2 < rc_coul * rc_coul) {
    fp += coul_pair(r2, qq[t], &e1);
    en += e1;
    hit = 1;
  }
  *fpair = fp;
  *e = en;
  return hit;
}

/* Forces, energy and virial from a pair list (each pair once).
 * eps, sigma, rc: ntypes x ntypes row-major; qq (may be NULL): ntypes x
 * ntypes qqrd2e q_a q_b with cutoff rc_coul.  f: n x 3 (overwritten).
 * ev (may be NULL): ev[0] = E, ev[1..6] = W_xx, W_yy, W_zz, W_xy, W_xz, W_yz. */
void orc_forces(int64_t n, const double *x, const int32_t *type,
                const double *box, int32_t ntypes, const double *eps,
                const double *sigma, const double *rc, const double *qq,
                double rc_coul, int64_t npairs, const int32_t *pi,
                const int32_t *pk, double *f, double *ev) {
  memset(f, 0, sizeof(double) * 3 * n);
  double E = 0, W[6] = {0, 0, 0, 0, 0, 0}, d[3];
  for (int64_t p = 0; p < npairs; p++) {
    int64_t i = pi[p], k = pk[p];
    double r2 = sep(x, i, k, box, d); /* d = x_k - x_i */
    int t = type[i] * ntypes + type[k];
    double e, fpair;
    if (!pair_terms(r2, t, eps, sigma, rc, qq, rc_coul, &fpair, &e)) continue;
    /* force on i along x_i - x_k = -d */
    for (int a = 0; a < 3; a++) {
      f[3 * i + a] -= fpair * d[a];
      f[3 * k + a] += fpair * d[a];
    }
    E += e;
    W[0] += fpair * d[0] * d[0];
    W[1] += fpair * d[1] * d[1];
    W[2] += fpair * d[2] * d[2];
    W[3] += fpair * d[0] * d[1];
    W[4] += fpair * d[0] * d[2];
    W[5] += fpair * d[1] * d[2];
  }
  if (ev) {
    ev[0] = E;
    for (int c = 0; c < 6; c++) ev[1 + c] = W[c];
  }
}

/* Force on each sampled atom by a scan over all atoms (no list). */
void orc_force_of(int64_t n, const double *x, const int32_t *type,
                  const double *box, int32_t ntypes, const double *eps,
                  const double *sigma, const double *rc, const double *qq,
                  double rc_coul, int64_t nsample, const int64_t *sample,
                  double *f_out) {
  double d[3];
  for (int64_t s = 0; s < nsample; s++) {
    int64_t i = sample[s];
    double fi[3] = {0, 0, 0};
    for (int64_t k = 0; k < n; k++) {
      if (k == i) continue;
      double r2 = sep(x, i, k, box, d);
      int t = type[i] * ntypes + type[k];
      double e, fpair;
      if (!pair_terms(r2, t, eps, sigma, rc, qq, rc_coul, &fpair, &e)) continue;
      for (int a = 0; a < 3; a++) fi[a] -= fpair * d[a];
    }
    for (int a = 0; a < 3; a++) f_out[3 * s + a] = fi[a];
  }
}

double orc_kinetic(int64_t n, const double *v, const int32_t *type,
                   const double *mass) {
  double ke = 0;
  for (int64_t i = 0; i < n; i++) {
    double m = mass[type[i]];
    ke += 0.5 * m * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                     v[3 * i + 2] * v[3 * i + 2]);
  }
  return ke;
}

/* ---- velocity Verlet ---------------------------------------------------- */

static double max_rc(int32_t ntypes, const double *rc) {
  double m = 0;
  for (int t = 0; t < ntypes * ntypes; t++) if (rc[t] > m) m = rc[t];
  return m;
}

typedef struct {
  int64_t cap, n;
  int32_t *pi, *pk;
} pairlist;

static int build(pairlist *pl, int64_t natoms, const double *x,
                 const double *box, double rlist) {
  for (;;) {
    pl->n = orc_pairs_cells(natoms, x, box, rlist, pl->cap, pl->pi, pl->pk);
    if (pl->n <= pl->cap) return 0;
    free(pl->pi); free(pl->pk);
    pl->cap = pl->n + pl->n / 4 + 16;
    pl->pi = malloc(sizeof(int32_t) * pl->cap);
    pl->pk = malloc(sizeof(int32_t) * pl->cap);
    if (!pl->pi || !pl->pk) return -1;
  }
}

/* Run nsteps of NVE velocity Verlet on (x, v, f), in place.
 *   init != 0: wrap x first (a fresh start);
 *   init == 0: do not wrap (a continuation from a state between rebuilds).
 *   Either way the list is built from x and f is recomputed at x on entry.
 *   step0:     global index of the first step (sets the rebuild cadence).
 * thermo (may be NULL): for every step s with (s+1) % thermo_every == 0, and
 * for the initial state, appends (step, E_pot, E_kin, W_xx, W_yy, W_zz,
 * W_xy, W_xz, W_yz) -- 9 doubles per record.  Returns the record count, or
 * -1 on allocation failure. */
int64_t orc_run(int64_t n, double *x, double *v, double *f,
                const int32_t *type, const double *box, int32_t ntypes,
                const double *eps, const double *sigma, const double *rc,
                const double *qq, double rc_coul, const double *mass,
                double skin, double dt, int64_t nsteps, int64_t step0,
                int32_t rebuild_every, int32_t init, int32_t thermo_every,
                double *thermo) {
  double rcm = max_rc(ntypes, rc);
  if (qq && rc_coul > rcm) rcm = rc_coul;
  double rlist = rcm + skin, ev[7];
  pairlist pl = {0, 0, NULL, NULL};
  double *dtf = malloc(sizeof(double) * ntypes);
  for (int t = 0; t < ntypes; t++) dtf[t] = 0.5 * dt / mass[t];
  if (init) orc_wrap(n, x, box);
  if (build(&pl, n, x, box, rlist)) return -1;
  orc_forces(n, x, type, box, ntypes, eps, sigma, rc, qq, rc_coul, pl.n, pl.pi, pl.pk, f,
             ev);
  int64_t rec = 0;
  if (thermo) {
    double *t = thermo + 9 * rec++;
    t[0] = (double)step0; t[1] = ev[0];
    t[2] = orc_kinetic(n, v, type, mass);
    for (int c = 0; c < 6; c++) t[3 + c] = ev[1 + c];
  }
  for (int64_t s = step0; s < step0 + nsteps; s++) {
    for (int64_t i = 0; i < n; i++)
      for (int a = 0; a < 3; a++) {
        v[3 * i + a] = fma(dtf[type[i]], f[3 * i + a], v[3 * i + a]);
        x[3 * i + a] = fma(dt, v[3 * i + a], x[3 * i + a]);
      }
    if ((s + 1) % rebuild_every == 0) {
      orc_wrap(n, x, box);
      if (build(&pl, n, x, box, rlist)) return -1;
    }
    orc_forces(n, x, type, box, ntypes, eps, sigma, rc, qq, rc_coul, pl.n, pl.pi,
               pl.pk, f, ev);
    for (int64_t i = 0; i < n; i++)
      for (int a = 0; a < 3; a++)
        v[3 * i + a] = fma(dtf[type[i]], f[3 * i + a], v[3 * i + a]);
    if (thermo && thermo_every > 0 && (s + 1) % thermo_every == 0) {
      double *t = thermo + 9 * rec++;
      t[0] = (double)(s + 1); t[1] = ev[0];
      t[2] = orc_kinetic(n, v, type, mass);
      for (int c = 0; c < 6; c++) t[3 + c] = ev[1 + c];
    }
  }
  free(pl.pi); free(pl.pk); free(dtf);
  return rec;
}

/* ---- adjoint: vector-Jacobian products of the forces ----------------------
 *
 * For a pair (i, k) inside rc with e = x_i - x_k (minimum image), q = |e|^2,
 * the force on i is t = g(q) e and the force on k is -t, where (Sec. 4,
 * derivative of Eq. 1)
 *   g(q)  = 24 eps (2 sigma^12 q^-7 - sigma^6 q^-4),
 *   g'(q) = 24 eps (-14 sigma^12 q^-8 + 4 sigma^6 q^-5).
 * Given the cotangent c = dL/dF (n x 3), the chain rule gives with
 * w = c_i - c_k:
 *   dL/dx_i += J w,  dL/dx_k -= J w,  J = g I + 2 g' e e^T,
 *   dL/deps_ab   += (e . w) g / eps,
 *   dL/dsigma_ab += (e . w) 24 eps (24 sigma^12 q^-7 - 6 sigma^6 q^-4) / sigma.
 * The cutoffs rc_ab are constants (no derivative through the cutoff).
 * gbar: 2 nt^2 doubles, dL/deps then dL/dsigma, each a symmetric nt x nt
 * table whose (a,b) and (b,a) entries both hold the derivative with respect
 * to the one parameter of the unordered type pair {a,b}. */
void orc_force_vjp(int64_t n, const double *x, const int32_t *type,
                   const double *box, int32_t ntypes, const double *eps,
                   const double *sigma, const double *rc, int64_t npairs,
                   const int32_t *pi, const int32_t *pk, const double *c,
                   double *xbar, double *gbar) {
  int nt2 = ntypes * ntypes;
  memset(xbar, 0, sizeof(double) * 3 * n);
  memset(gbar, 0, sizeof(double) * 2 * nt2);
  double d[3];
  for (int64_t p = 0; p < npairs; p++) {
    int64_t i = pi[p], k = pk[p];
    double q = sep(x, i, k, box, d); /* d = x_k - x_i */
    int ta = type[i], tb = type[k];
    int t = ta * ntypes + tb;
    if (!(q < rc[t] * rc[t])) continue;
    double ep = eps[t], sg = sigma[t];
    double s6 = pow(sg, 6), s12 = s6 * s6;
    double g = 24.0 * ep * (2.0 * s12 * pow(q, -7) - s6 * pow(q, -4));
    double gp = 24.0 * ep * (-14.0 * s12 * pow(q, -8) + 4.0 * s6 * pow(q, -5));
    double e[3] = {-d[0], -d[1], -d[2]};
    double w[3], ew = 0;
    for (int a = 0; a < 3; a++) {
      w[a] = c[3 * i + a] - c[3 * k + a];
      ew += e[a] * w[a];
    }
    for (int a = 0; a < 3; a++) {
      double jw = g * w[a] + 2.0 * gp * e[a] * ew;
      xbar[3 * i + a] += jw;
      xbar[3 * k + a] -= jw;
    }
    int lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
    gbar[lo * ntypes + hi] += ew * g / ep;
    gbar[nt2 + lo * ntypes + hi] +=
        ew * 24.0 * ep * (24.0 * s12 * pow(q, -7) - 6.0 * s6 * pow(q, -4)) / sg;
  }
  for (int a = 0; a < ntypes; a++)
    for (int b = a + 1; b < ntypes; b++) {
      gbar[b * ntypes + a] = gbar[a * ntypes + b];
      gbar[nt2 + b * ntypes + a] = gbar[nt2 + a * ntypes + b];
    }
}

/* Reverse mode through nsteps of the velocity-Verlet run of orc_run (init =
 * 1: x0 is wrapped first).  The loss depends on the forces at the final
 * positions only, through cF = dL/dF(x_K) (n x 3).  Writes dL/dx0, dL/dv0
 * (n x 3) and gbar (2 nt^2, as orc_force_vjp).  The forward run is repeated
 * here storing every position and pair list; each force evaluation is then
 * differentiated with the list it used.
 *
 * Chain rule for one step (h = dt/2, a = F/m):
 *   v' = v + h a(x),  x1 = x + dt v',  v1 = v' + h a(x1)
 * gives, going backwards, v'bar = v1bar, Fbar(x1) += (h/m) v1bar,
 * v'bar += dt x1bar, xbar = x1bar + [VJP of F(x1) goes into x1bar first],
 * vbar = v'bar, Fbar(x) += (h/m) v'bar.  Returns 0, or -1 on allocation
 * failure. */
int orc_traj_vjp(int64_t n, const double *x0, const double *v0,
                 const int32_t *type, const double *box, int32_t ntypes,
                 const double *eps, const double *sigma, const double *rc,
                 const double *mass, double skin, double dt, int64_t nsteps,
                 int32_t rebuild_every, const double *cF, double *x0bar,
                 double *v0bar, double *gbar) {
  double rlist = max_rc(ntypes, rc) + skin, ev[7];
  int nt2 = ntypes * ntypes;
  int64_t K = nsteps, n3 = 3 * n;
  double *xs = malloc(sizeof(double) * n3 * (K + 1));
  double *v = malloc(sizeof(double) * n3);
  double *f = malloc(sizeof(double) * n3);
  int64_t nlists = K / rebuild_every + 2;
  pairlist *pl = calloc(nlists, sizeof(pairlist));
  int64_t *list_of = malloc(sizeof(int64_t) * (K + 1));
  double *dtf = malloc(sizeof(double) * ntypes);
  double *xbar = malloc(sizeof(double) * n3), *vbar = malloc(sizeof(double) * n3);
  double *cc = malloc(sizeof(double) * n3), *jx = malloc(sizeof(double) * n3);
  double *gb = malloc(sizeof(double) * 2 * nt2);
  if (!xs || !v || !f || !pl || !list_of || !dtf || !xbar || !vbar || !cc || !jx || !gb)
    return -1;
  for (int t = 0; t < ntypes; t++) dtf[t] = 0.5 * dt / mass[t];
  /* forward, as orc_run */
  memcpy(xs, x0, sizeof(double) * n3);
  memcpy(v, v0, sizeof(double) * n3);
  orc_wrap(n, xs, box);
  int64_t L = 0;
  if (build(&pl[L], n, xs, box, rlist)) return -1;
  list_of[0] = L;
  orc_forces(n, xs, type, box, ntypes, eps, sigma, rc, NULL, 0.0, pl[L].n, pl[L].pi, pl[L].pk,
             f, ev);
  for (int64_t s = 0; s < K; s++) {
    double *xo = xs + n3 * s, *xn = xs + n3 * (s + 1);
    for (int64_t i = 0; i < n; i++)
      for (int a = 0; a < 3; a++) {
        v[3 * i + a] = fma(dtf[type[i]], f[3 * i + a], v[3 * i + a]);
        xn[3 * i + a] = fma(dt, v[3 * i + a], xo[3 * i + a]);
      }
    if ((s + 1) % rebuild_every == 0) {
      orc_wrap(n, xn, box);
      L++;
      if (build(&pl[L], n, xn, box, rlist)) return -1;
    }
    list_of[s + 1] = L;
    orc_forces(n, xn, type, box, ntypes, eps, sigma, rc, NULL, 0.0, pl[L].n, pl[L].pi,
               pl[L].pk, f, ev);
    for (int64_t i = 0; i < n; i++)
      for (int a = 0; a < 3; a++)
        v[3 * i + a] = fma(dtf[type[i]], f[3 * i + a], v[3 * i + a]);
  }
  /* backward over the force evaluations e = K .. 0 */
  memset(xbar, 0, sizeof(double) * n3);
  memset(vbar, 0, sizeof(double) * n3);
  memset(gbar, 0, sizeof(double) * 2 * nt2);
  for (int64_t e = K; e >= 0; e--) {
    /* cotangent of F(x_e): the loss at e = K, (h/m) vbar_e from the kick
       that ends step e-1 and (h/m) vbar' from the kick that starts step e;
       here vbar already holds the adjoint of v_e = v' of step e */
    for (int64_t i = 0; i < n; i++)
      for (int a = 0; a < 3; a++) {
        double hm = dtf[type[i]];
        double cv = 0.0;
        if (e == K) cv += cF[3 * i + a];
        if (e >= 1) cv += hm * vbar[3 * i + a];  /* end of step e-1 */
        if (e < K) cv += hm * vbar[3 * i + a];   /* start of step e */
        cc[3 * i + a] = cv;
      }
    pairlist *p = &pl[list_of[e]];
    orc_force_vjp(n, xs + n3 * e, type, box, ntypes, eps, sigma, rc, p->n, p->pi, p->pk,
                  cc, jx, gb);
    for (int64_t k = 0; k < n3; k++) xbar[k] += jx[k];
    for (int k = 0; k < 2 * nt2; k++) gbar[k] += gb[k];
    if (e == 0) break;
    /* undo the drift of step e-1: x_e = x_{e-1} + dt v'  ->  v'bar += dt xbar */
    for (int64_t k = 0; k < n3; k++) vbar[k] += dt * xbar[k];
    /* v' = v_{e-1} + h a_{e-1}: vbar_{e-1} = v'bar (kept in vbar); its
       (h/m) v'bar reaches F(x_{e-1}) in the next iteration, and v_{e-1} is
       itself the end of step e-2, which adds (h/m) vbar_{e-1} there too */
  }
  memcpy(x0bar, xbar, sizeof(double) * n3);
  memcpy(v0bar, vbar, sizeof(double) * n3);
  for (int64_t l = 0; l <= L; l++) { free(pl[l].pi); free(pl[l].pk); }
  free(pl); free(xs); free(v); free(f); free(list_of); free(dtf);
  free(xbar); free(vbar); free(cc); free(jx); free(gb);
  return 0;
}

/* Steepest descent: nsteps of x <- x + alpha F / max_i |F_i|, the pair list
 * rebuilt at every step.  Used to relax random starting positions. */
int orc_sd_relax(int64_t n, double *x, const int32_t *type, const double *box,
                 int32_t ntypes, const double *eps, const double *sigma,
                 const double *rc, int64_t nsteps, double alpha) {
  double *f = malloc(sizeof(double) * 3 * n);
  pairlist pl = {0, 0, NULL, NULL};
  if (!f) return -1;
  double rcut = max_rc(ntypes, rc);
  for (int64_t s = 0; s < nsteps; s++) {
    if (build(&pl, n, x, box, rcut)) return -1;
    orc_forces(n, x, type, box, ntypes, eps, sigma, rc, NULL, 0.0, pl.n, pl.pi, pl.pk, f,
               NULL);
    double fmax = 0.0;
    for (int64_t i = 0; i < n; i++) {
      double a = sqrt(f[3 * i] * f[3 * i] + f[3 * i + 1] * f[3 * i + 1] +
                      f[3 * i + 2] * f[3 * i + 2]);
      if (a > fmax) fmax = a;
    }
    if (!(fmax > 0.0)) break;
    double step = alpha / fmax;
    for (int64_t k = 0; k < 3 * n; k++) x[k] += step * f[k];
  }
  free(f); free(pl.pi); free(pl.pk);
  return 0;
}
