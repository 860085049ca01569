"""Spatial decomposition of one periodic box over ranks: slabs along x with
ghost atoms (arXiv 2508.13523, Sec. 3-5: LAMMPS distributes a box over MPI
ranks, each owning the atoms of its subdomain and holding copies -- ghost
atoms -- of the atoms of neighboring subdomains within the list cutoff; with
`newton on` the forces on ghosts are sent back to their owners, with `newton
off` every cross-boundary pair is computed on both sides; Sec. 4.1 and
Fig. 2b compare the two).

Host-side bookkeeping and point-to-point communication only.  Messages go
through torch.distributed send/recv between neighboring ranks (gloo for CPU
tensors, NCCL for device tensors); there is no collective on the data path.
The per-rank force computation is a caller-supplied engine, so the same
exchange drives any force kernel.

Protocol per neighbor-list period (as LAMMPS does at every reneighboring):
  exchange  -- atoms that left the slab move to the rank that now owns them
               (positions wrapped into the box first);
  borders   -- each rank sends every neighbor the atoms within rlist of that
               neighbor's slab, with the periodic image shift that places
               them next to it; these are the neighbor's ghosts until the
               next period;
and every step:
  forward   -- the ghosts' current positions (same atoms, same shifts);
  reverse   -- (newton on) the forces computed on ghosts, added into their
               owners' forces in a fixed order.
A slab must be at least rlist wide (ghosts come only from the two adjacent
slabs) and at most L - 2 rlist (no atom is a ghost of its own rank), so
2 <= P <= L / rlist.
"""
from __future__ import annotations

import numpy as np

TAG_COUNT, TAG_DATA = 11, 12


def _dist():
    import torch.distributed as dist
    return dist


class SlabDomain:
    """One rank's slab [lo, hi) along x of a periodic orthorhombic box.

    box: the box edges (3,); nranks: P; rank: this rank; rlist: the list
    cutoff (max rc + skin).  Positions are (n, 3) float64 arrays in the
    box's frame; ghost positions carry the image shift that puts them within
    rlist of this slab."""

    def __init__(self, box, nranks: int, rank: int, rlist: float):
        self.box = np.asarray(box, dtype=np.float64)
        self.P = int(nranks)
        self.rank = int(rank)
        self.rlist = float(rlist)
        L = self.box[0]
        self.width = L / self.P
        if not (self.rlist <= self.width <= L - 2.0 * self.rlist):
            raise ValueError("slab width must lie in [rlist, L - 2 rlist]")
        self.lo = self.rank * self.width
        self.hi = L if self.rank == self.P - 1 else (self.rank + 1) * self.width
        self.nbrs = sorted({(self.rank - 1) % self.P, (self.rank + 1) % self.P} - {self.rank})
        self._send_sel = {}    # neighbor -> (indices into owned atoms, image shifts)
        self.ghost_ids = np.zeros(0, np.int64)
        self._ghost_from = []  # (neighbor, count) in the order ghosts are stored

    # ---- geometry ----------------------------------------------------------------
    def owner_of(self, xw):
        """Owning rank of each wrapped position (x in [0, L))."""
        r = np.floor(xw[:, 0] / self.width).astype(np.int64)
        return np.clip(r, 0, self.P - 1)

    def _slab_of(self, q):
        L = self.box[0]
        lo = q * self.width
        return lo, (L if q == self.P - 1 else (q + 1) * self.width)

    def ghost_selection(self, x, q):
        """Indices i of this rank's atoms and shifts s in {-1, 0, 1} such that
        x_i + s L lies within rlist of rank q's slab (outside it)."""
        L = self.box[0]
        lo, hi = self._slab_of(q)
        idx, sh = [], []
        for s in (-1, 0, 1):
            xs = x[:, 0] + s * L
            m = ((xs >= lo - self.rlist) & (xs < lo)) | ((xs >= hi) & (xs < hi + self.rlist))
            i = np.nonzero(m)[0]
            idx.append(i)
            sh.append(np.full(len(i), s, np.int64))
        return np.concatenate(idx), np.concatenate(sh)

    # ---- messages ------------------------------------------------------------------
    def _swap(self, payload: dict, width: int, dtype):
        """Send payload[q] ((k, width) array) to every neighbor q and return
        what each neighbor sent here, {q: (k', width) array}."""
        import torch
        dist = _dist()
        out = {}
        reqs = []
        counts = {}
        for q in self.nbrs:
            n_out = torch.tensor([len(payload[q])], dtype=torch.int64)
            n_in = torch.zeros(1, dtype=torch.int64)
            reqs.append(dist.isend(n_out, q, tag=TAG_COUNT))
            reqs.append(dist.irecv(n_in, q, tag=TAG_COUNT))
            counts[q] = n_in
        for r in reqs:
            r.wait()
        reqs = []
        bufs = {}
        for q in self.nbrs:
            data = torch.from_numpy(np.ascontiguousarray(payload[q], dtype=dtype).reshape(-1))
            bufs[q] = torch.zeros(int(counts[q].item()) * width, dtype=data.dtype)
            reqs.append(dist.isend(data, q, tag=TAG_DATA))
            reqs.append(dist.irecv(bufs[q], q, tag=TAG_DATA))
        for r in reqs:
            r.wait()
        for q in self.nbrs:
            out[q] = bufs[q].numpy().reshape(-1, width)
        return out

    def exchange(self, ids, x, v):
        """Migration: wrapped positions x of the owned atoms decide their
        owner; atoms of other ranks (adjacent ones only) are sent there with
        their ids and velocities.  Returns the new (ids, x, v), ordered by
        global id."""
        dest = self.owner_of(x)
        far = (dest != self.rank) & ~np.isin(dest, self.nbrs)
        if far.any():
            raise RuntimeError("an atom moved past a neighboring slab in one period")
        keep = dest == self.rank
        rec = np.concatenate([ids[:, None].astype(np.float64), x, v], axis=1)
        payload = {q: rec[dest == q] for q in self.nbrs}
        got = self._swap(payload, 7, np.float64)
        all_rec = np.concatenate([rec[keep]] + [got[q] for q in self.nbrs], axis=0)
        all_rec = all_rec[np.argsort(all_rec[:, 0], kind="stable")]
        return all_rec[:, 0].astype(np.int64), all_rec[:, 1:4].copy(), all_rec[:, 4:7].copy()

    def borders(self, ids, x):
        """Choose, for every neighbor, the owned atoms it needs as ghosts and
        send it their ids and shifted positions; receive this rank's ghosts.
        Returns (ghost_ids, ghost_x)."""
        L = self.box[0]
        payload = {}
        for q in self.nbrs:
            i, s = self.ghost_selection(x, q)
            self._send_sel[q] = (i, s)
            xs = x[i].copy()
            xs[:, 0] += s * L
            payload[q] = np.concatenate([ids[i, None].astype(np.float64), xs], axis=1)
        got = self._swap(payload, 4, np.float64)
        self._ghost_from = [(q, len(got[q])) for q in self.nbrs]
        g = np.concatenate([got[q] for q in self.nbrs], axis=0) if self.nbrs else np.zeros((0, 4))
        self.ghost_ids = g[:, 0].astype(np.int64)
        return self.ghost_ids, g[:, 1:4].copy()

    def forward(self, x):
        """The ghosts' current positions (the atoms and shifts of the last
        borders call) from the owned positions x."""
        L = self.box[0]
        payload = {}
        for q in self.nbrs:
            i, s = self._send_sel[q]
            xs = x[i].copy()
            xs[:, 0] += s * L
            payload[q] = xs
        got = self._swap(payload, 3, np.float64)
        parts = [got[q] for q, _ in self._ghost_from]
        return np.concatenate(parts, axis=0) if parts else np.zeros((0, 3))

    def reverse(self, f_owned, f_ghost):
        """newton on: send the forces computed on ghosts back to their owners
        and add the ones received into f_owned (in neighbor order, then in
        the order the atoms were sent).  Returns the summed owned forces."""
        payload = {}
        k = 0
        for q, cnt in self._ghost_from:
            payload[q] = f_ghost[k:k + cnt]
            k += cnt
        got = self._swap(payload, 3, np.float64)
        f = f_owned.copy()
        for q in self.nbrs:
            i, _ = self._send_sel[q]
            np.add.at(f, i, got[q])
        return f


def run_slabs(dom: SlabDomain, ids, x, v, engine, *, nsteps: int, dt: float, mass: float,
              box, rebuild_every: int, newton: bool):
    """Velocity Verlet NVE on this rank's slab (the step order of the
    single-box path: kick, drift, rebuild every `rebuild_every` steps,
    forces, kick).  ids, x, v: this rank's atoms (x wrapped into the box).
    engine(x_owned, x_ghost, ids_owned, ids_ghost, newton) -> (f_owned,
    f_ghost) computes the forces of the pairs this rank is responsible for:
    every pair with an owned atom (newton off), or each cross pair on one
    rank only (newton on; f_ghost then goes back to the owners).  Returns
    the final (ids, x, v, f)."""
    box = np.asarray(box, dtype=np.float64)

    def wrap(p):
        w = p - box * np.floor(p / box)
        return np.where(w == box, 0.0, w)

    def forces(x_own, xg):
        f_own, f_g = engine(x_own, xg, ids, gids, newton)
        return dom.reverse(f_own, f_g) if newton else f_own

    dtf = 0.5 * dt / mass
    x = wrap(x)
    ids, x, v = dom.exchange(ids, x, v)
    gids, xg = dom.borders(ids, x)
    f = forces(x, xg)
    for s in range(nsteps):
        v = v + dtf * f
        x = x + dt * v
        if (s + 1) % rebuild_every == 0:
            x = wrap(x)
            ids, x, v = dom.exchange(ids, x, v)
            gids, xg = dom.borders(ids, x)
        else:
            xg = dom.forward(x)
        f = forces(x, xg)
        v = v + dtf * f
    return ids, x, v, f


class LJMDSlabEngine:
    """A run_slabs engine on the GPU library, newton off: one LJMD context
    per neighbor-list period over this rank's owned and ghost atoms, whose
    forces on owned atoms are the whole sums (every pair with an owned atom
    is in the context's list; ghost-ghost pairs are computed too and
    discarded with the ghosts' forces).  The local frame is the box widened
    to 4 L along x, positions shifted by +L, so that nothing wraps along x;
    y and z keep the box's periodicity.  Between reneighborings the ghost
    set is fixed and positions are loaded with md_set_state's
    MD_MEM_KEEP_LIST.  md: the package module; the other arguments are the
    context's (Eq. 1 parameters per type, one type here)."""

    def __init__(self, md, box, eps=1.0, sigma=1.0, rc=2.5, mass=1.0, skin=0.3,
                 list_kind=None, precision=None):
        self.md = md
        self.box = np.asarray(box, dtype=np.float64)
        self.local_box = np.array([4.0 * self.box[0], self.box[1], self.box[2]])
        self.shift = np.array([self.box[0], 0.0, 0.0])
        self.kw = dict(eps=eps, sigma=sigma, rc=rc, mass=mass, skin=skin,
                       list_kind=md.MD_LIST_FULL if list_kind is None else list_kind,
                       precision=md.MD_PREC_FP64 if precision is None else precision)
        self.ctx = None
        self.key = None

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None

    def __call__(self, x_own, xg, ids_own, ids_g, newton):
        if newton:
            raise ValueError("LJMDSlabEngine computes newton off (ghost-ghost pairs included)")
        xl = np.concatenate([x_own, xg]) + self.shift
        key = (len(ids_own), len(ids_g), ids_own.tobytes(), ids_g.tobytes())
        zeros = np.zeros_like(xl)
        if key != self.key:
            self.close()
            k = self.kw
            self.ctx = self.md.LJMD(xl, zeros, None, self.local_box, k["eps"], k["sigma"],
                                    k["rc"], k["mass"], skin=k["skin"],
                                    list_kind=k["list_kind"], precision=k["precision"],
                                    threads_per_atom=1)
            self.key = key
        else:
            self.ctx.set_state(xl, zeros, keep_list=True)
        f = self.ctx.get_state(host=True)[2]
        n = len(x_own)
        return f[:n], f[n:]

