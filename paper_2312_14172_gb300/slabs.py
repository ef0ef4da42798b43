"""z-slab sub-domains: one lattice on several handles.

The paper's parallel scheme (Secs. 4.2.2-4.2.4) splits the fluid domain
among processes and, for the particles, separates responsibility (the
process holding a particle's centre integrates it) from the neighbourhood
(the processes its surface reaches compute partial surface forces and send
them to the responsible one, which sums them and sends the result back).
Here the domain is cut into z slabs, one handle each (one GPU each, or
several on one GPU); every slab is a box of its planes plus one ghost plane
on each side that faces another slab (HLBM_WALL_Z | HLBM_CUT_Z; on a wall of
the lattice the box's own z wall is that wall), and the step of
include/hlbm.h's "Sub-domains" runs across them:

  halo     before an odd step the ghost planes take the five crossing slots
           of the neighbours' boundary planes; after it the owned boundary
           planes take back the slots the neighbours' cells wrote into their
           ghost copies (the in-place AA storage moves populations across a
           face only on odd steps);
  forces   each slab's partial momentum exchange over its owned cells; the
           partials of a particle come from the slabs its circumscribed
           sphere reaches (route.senders), go to its owner (route.owner) and
           the sum goes back to every slab that holds a copy;
  update   every copy integrates the same totals (the owner's state is not
           sent: the copies stay bit-identical, and six numbers per particle
           travel instead of the whole state).

The host logic (which slab owns, sends to and holds which particle) is in
plain functions so that it can run, and be tested, across processes with
torch.distributed (DistributedExchange); SlabLattice drives all slabs from
one process through the C-ABI.
"""
import numpy as np

from . import hlbm

PLUS_Z, MINUS_Z = 1, -1


# ------------------------------------------------------------ partition
def slab_ranges(nz, nslabs):
    """Owned global planes [z0, z1) of each slab: nz split as evenly as
    possible, lower slabs taking the remainder."""
    if not (1 <= nslabs <= nz):
        raise ValueError("need 1 <= slabs <= nz")
    base, rem = divmod(nz, nslabs)
    out, z = [], 0
    for s in range(nslabs):
        m = base + (1 if s < rem else 0)
        out.append((z, z + m))
        z += m
    return out


def owner(zc, ranges, nz, periodic=True):
    """The slab whose owned planes hold the centre: the plane of the cell
    nearest to zc (cell k spans [k - 1/2, k + 1/2))."""
    k = int(np.floor(zc + 0.5))
    if periodic:
        k %= nz
    else:
        k = min(max(k, 0), nz - 1)
    for s, (z0, z1) in enumerate(ranges):
        if z0 <= k < z1:
            return s
    raise ValueError("centre outside the lattice")


def _intersects(lo, hi, z0, z1, nz, periodic):
    """Does the closed interval [lo, hi] of plane coordinates meet planes
    [z0, z1) (any periodic image when periodic)?"""
    shifts = (-nz, 0, nz) if periodic else (0,)
    return any(lo + s <= z1 - 1 and hi + s >= z0 for s in shifts)


def senders(zc, rc, ranges, nz, periodic=True):
    """Slabs whose owned planes can hold interior cells of a particle with
    centre height zc and circumscribed radius rc (the cells inside lie within
    rc of the centre): the slabs that send partial surface forces."""
    lo, hi = zc - rc - 1.0, zc + rc + 1.0
    return [s for s, (z0, z1) in enumerate(ranges) if _intersects(lo, hi, z0, z1, nz, periodic)]


def holders(zc, reach, ranges, nz, periodic=True):
    """Slabs that need a copy of a particle whose influence (the radius
    beyond which B of Eq. B vanishes, plus the motion allowed for) reaches
    reach from its centre: those whose owned or ghost planes it meets."""
    lo, hi = zc - reach - 1.0, zc + reach + 1.0
    return [s for s, (z0, z1) in enumerate(ranges) if _intersects(lo, hi, z0 - 1, z1 + 1, nz, periodic)]


def local_z(zc, z0, z1, nz, periodic=True, lo=1):
    """Height of a centre in a slab's local frame (local plane lo = global
    plane z0; lo = 1 below a ghost plane, 0 on a wall): the periodic image
    nearest to the slab's middle."""
    zl = zc - z0 + lo
    if periodic:
        mid = lo + 0.5 * (z1 - z0 - 1)
        zl -= nz * np.round((zl - mid) / nz)
    return zl


def sum_partials(partials, route_senders, n):
    """Totals per particle: the sum of the partials of the slabs that send
    them, in slab order.  partials: {slab: (F [n, 3], T [n, 3])} over the
    global particle index (zero where a slab holds no copy)."""
    F, T = np.zeros((n, 3)), np.zeros((n, 3))
    for p in range(n):
        for s in route_senders[p]:
            F[p] += partials[s][0][p]
            T[p] += partials[s][1][p]
    return F, T


# ------------------------------------------------------ one process, C-ABI
class SlabLattice:
    """A workload (see the workloads module; z periodic or walled) on
    nslabs >= 2 z-slab handles driven from this process.  A slab has a ghost
    plane on each side that faces another slab; on a wall of the lattice its
    owned planes reach the wall (the box's own z wall is the lattice's).
    margin: how far (in cells) particles may move before the fixed sets of
    copies would no longer cover them (checked every step).  Contact
    (hlbm_set_contact) is not carried across slabs."""

    def __init__(self, w, nslabs, precision="fp32", mea_mode="kernel", margin=4.0, devices=None):
        n = w["n"]
        self.nz = n[2]
        self.periodic = not (w["bc"] & hlbm.HLBM_WALL_Z)
        if nslabs < 2:
            raise ValueError("a slab decomposition needs two slabs or more (one box is one handle)")
        self.ranges = slab_ranges(self.nz, nslabs)
        P = w["particles"]
        self.np = len(P["shape"])
        self.X0 = np.asarray(P["X"], float).copy()
        self.margin = margin
        bc = (w["bc"] & 3) | hlbm.HLBM_WALL_Z | hlbm.HLBM_CUT_Z
        grids = w.get("grids", ())
        rinf = _influence_radius(P, w["eps"], grids)
        self.rc = _circumscribed_radius(P, grids)
        reach = rinf + margin
        self.hold = [holders(self.X0[p, 2], reach[p], self.ranges, self.nz, self.periodic) for p in range(self.np)]
        self.slabs = []
        for s, (z0, z1) in enumerate(self.ranges):
            has_lo = self.periodic or s > 0
            has_up = self.periodic or s < nslabs - 1
            lo, m = (1 if has_lo else 0), z1 - z0
            ids = [p for p in range(self.np) if s in self.hold[p]]
            prm = hlbm.make_params(tau=w["tau"], eps=w["eps"], gravity=w["gravity"],
                                   fluid_force=w.get("fluid_force", (0, 0, 0)), precision=precision,
                                   max_particles=max(1, len(ids)),
                                   grid_floats=sum(int(np.asarray(v).size) for v, _ in grids))
            dev = None if devices is None else devices[s % len(devices)]
            lat = hlbm.Lattice([(n[0], n[1], m + has_lo + has_up, bc)], prm, device=dev)
            for values, h in grids:
                lat.add_grid(values, h)
            lat.set_owned_planes(lo, lo + m)
            lat.set_mea_mode(mea_mode)
            if ids:
                X = self.X0[ids].copy()
                X[:, 2] = [local_z(z, z0, z1, self.nz, self.periodic, lo) for z in X[:, 2]]
                sub = {k: np.asarray(v)[ids] for k, v in P.items()}
                sub["X"] = X
                lat.add_workload_particles(sub)
            self.slabs.append({"lat": lat, "ids": ids, "z0": z0, "z1": z1, "lo": lo, "m": m})
        self.steps = 0

    def close(self):
        for sl in self.slabs:
            sl["lat"].close()

    # --- halo of the in-place storage: ghost plane lo - 1, owned planes
    # lo .. lo + m - 1, ghost plane lo + m
    def _halo_before_odd(self):
        for s, sl in enumerate(self.slabs):
            L, U = self._neighbour(s, -1), self._neighbour(s, +1)
            if L is not None:
                nb = self.slabs[L]
                sl["lat"].set_plane_slots(sl["lo"] - 1, MINUS_Z,
                                          nb["lat"].plane_slots(nb["lo"] + nb["m"] - 1, MINUS_Z))
            if U is not None:
                nb = self.slabs[U]
                sl["lat"].set_plane_slots(sl["lo"] + sl["m"], PLUS_Z, nb["lat"].plane_slots(nb["lo"], PLUS_Z))

    def _halo_after_odd(self):
        # read every ghost first: the owned planes written below are the
        # ghosts' sources on the neighbours
        got = []
        for s, sl in enumerate(self.slabs):
            L, U = self._neighbour(s, -1), self._neighbour(s, +1)
            a = b = None
            if L is not None:
                nb = self.slabs[L]
                a = nb["lat"].plane_slots(nb["lo"] + nb["m"], PLUS_Z)
            if U is not None:
                nb = self.slabs[U]
                b = nb["lat"].plane_slots(nb["lo"] - 1, MINUS_Z)
            got.append((a, b))
        for sl, (a, b) in zip(self.slabs, got):
            if a is not None:
                sl["lat"].set_plane_slots(sl["lo"], PLUS_Z, a)
            if b is not None:
                sl["lat"].set_plane_slots(sl["lo"] + sl["m"] - 1, MINUS_Z, b)

    def _neighbour(self, s, side):
        S = len(self.slabs)
        t = s + side
        if 0 <= t < S:
            return t
        return t % S if self.periodic else None

    # --- one step of the whole lattice
    def step(self, nsteps=1):
        for _ in range(nsteps):
            odd = self.steps & 1
            if odd:
                self._halo_before_odd()
            partials = {}
            for s, sl in enumerate(self.slabs):
                F, T = sl["lat"].step_forces()
                Fg, Tg = np.zeros((self.np, 3)), np.zeros((self.np, 3))
                Fg[sl["ids"]], Tg[sl["ids"]] = F, T
                partials[s] = (Fg, Tg)
            Z = self.particle_heights()
            route = [senders(Z[p], self.rc[p], self.ranges, self.nz, self.periodic) for p in range(self.np)]
            for p in range(self.np):
                if not set(route[p]) <= set(self.hold[p]):
                    raise RuntimeError(f"particle {p} moved beyond the slabs holding its copies")
            Ft, Tt = sum_partials(partials, route, self.np)
            for sl in self.slabs:
                sl["lat"].step_with_forces(Ft[sl["ids"]], Tt[sl["ids"]])
            if odd:
                self._halo_after_odd()
            self.steps += 1

    def particle_heights(self):
        """Global centre heights, from each particle's owner copy (all
        copies are equal)."""
        st = self.particle_state()
        return st["X"][:, 2]

    def particle_state(self):
        """The global particle state (from the copy in the first slab that
        holds each particle, mapped back to global z)."""
        out = {k: np.zeros((self.np, 4 if k == "quat" else 3)) for k in ("X", "U", "omega", "quat", "F", "T")}
        done = np.zeros(self.np, bool)
        for sl in self.slabs:
            if not sl["ids"]:
                continue
            st = sl["lat"].particle_state()
            for j, p in enumerate(sl["ids"]):
                if done[p]:
                    continue
                for k in out:
                    out[k][p] = st[k][j]
                out["X"][p, 2] += sl["z0"] - sl["lo"]
                if self.periodic:
                    out["X"][p, 2] %= self.nz
                done[p] = True
        return out

    def populations(self):
        """The global post-streaming populations f[19, nz, ny, nx], assembled
        from the slabs' owned planes."""
        parts = []
        for sl in self.slabs:
            f = sl["lat"].populations()
            parts.append(f[:, sl["lo"]:sl["lo"] + sl["m"]])
        return np.concatenate(parts, axis=1)


def _circumscribed_radius(P, grids):
    a = np.asarray(P["a"], float)
    out = np.zeros(len(P["shape"]))
    for p, s in enumerate(P["shape"]):
        if s == 0:
            out[p] = a[p, 0]
        elif s == 1:
            out[p] = a[p].max()
        elif s == 2:
            out[p] = np.linalg.norm(a[p])
        elif s == 3:
            out[p] = a[p, 0] + a[p, 2]
        else:  # grid: the farthest sample point of its grid bounds it
            v, h = grids[int(a[p, 0])]
            out[p] = 0.5 * h * np.linalg.norm(np.array(np.shape(v)[::-1]) - 1)
    return out


def _influence_radius(P, eps, grids):
    a = np.asarray(P["a"], float)
    rc = _circumscribed_radius(P, grids)
    out = rc + 0.5 * eps
    for p, s in enumerate(P["shape"]):
        if s == 1:
            out[p] = a[p].max() * (1.0 + eps / (2.0 * a[p].min()))
        elif s == 4:
            out[p] = rc[p]  # the whole grid
    return out


# ------------------------------------------- several processes (one slab each)
class DistributedExchange:
    """The exchanges of a slab step between processes, one slab per rank,
    over torch.distributed point-to-point messages (gloo on CPU; NCCL with
    device tensors): halo planes between neighbouring ranks, partial forces
    from the sending slabs to each particle's owner, totals from the owner
    to every holder.  Only ranks that share a particle or a face exchange
    messages; there is no collective on the data path."""

    def __init__(self, dist, rank, world, ranges, nz, periodic=True):
        self.dist, self.rank, self.world = dist, rank, world
        self.ranges, self.nz, self.periodic = ranges, nz, periodic

    def neighbour(self, side):
        t = self.rank + side
        if 0 <= t < self.world:
            return t
        return t % self.world if self.periodic and self.world > 1 else None

    def swap_faces(self, send_lower, send_upper, shape, dtype):
        """Send one plane buffer to each neighbour and receive theirs:
        (from_lower, from_upper), None where there is no neighbour."""
        import torch
        # tags tell the two faces apart when one rank is both neighbours:
        # 1 travels upwards (a lower face's data), 2 downwards
        ops, recv = [], {}
        for side, buf in ((-1, send_lower), (+1, send_upper)):
            nb = self.neighbour(side)
            if nb is None or nb == self.rank:
                continue
            ops.append(self.dist.P2POp(self.dist.isend, torch.as_tensor(np.ascontiguousarray(buf)), nb,
                                       tag=2 if side < 0 else 1))
            r = torch.empty(shape, dtype=dtype)
            recv[side] = r
            ops.append(self.dist.P2POp(self.dist.irecv, r, nb, tag=1 if side < 0 else 2))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        return (recv[-1].numpy() if -1 in recv else None, recv[+1].numpy() if +1 in recv else None)

    def total_forces(self, partial, Z, rc, holding):
        """partial: {p: (F[3], T[3])} of the particles this rank sends for
        (its owned cells); Z, rc: heights and circumscribed radii of all
        particles; holding: {p: sorted list of ranks holding p}.  Returns
        {p: (F, T)} totals for every particle this rank holds."""
        import torch
        n = len(Z)
        route = [senders(Z[p], rc[p], self.ranges, self.nz, self.periodic) for p in range(n)]
        owners = [owner(Z[p], self.ranges, self.nz, self.periodic) for p in range(n)]
        ops, inbox = [], {}
        # partial forces: every sender that is not the owner sends to it
        for p in range(n):
            o = owners[p]
            if self.rank in route[p] and self.rank != o:
                v = np.concatenate(partial.get(p, (np.zeros(3), np.zeros(3))))
                ops.append(self.dist.P2POp(self.dist.isend, torch.as_tensor(v), o, tag=p))
            if self.rank == o:
                for s in route[p]:
                    if s != o:
                        r = torch.empty(6, dtype=torch.float64)
                        inbox[(p, s)] = r
                        ops.append(self.dist.P2POp(self.dist.irecv, r, s, tag=p))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        totals = {}
        for p in range(n):
            if self.rank != owners[p]:
                continue
            acc = np.zeros(6)
            for s in route[p]:  # slab order: every run adds in the same order
                acc += (np.concatenate(partial.get(p, (np.zeros(3), np.zeros(3)))) if s == self.rank
                        else inbox[(p, s)].numpy())
            totals[p] = acc
        # totals: the owner sends to every other holder
        ops, got = [], {}
        for p in range(n):
            o = owners[p]
            for r in holding[p]:
                if r == o:
                    continue
                if self.rank == o:
                    ops.append(self.dist.P2POp(self.dist.isend, torch.as_tensor(totals[p]), r, tag=p))
                elif self.rank == r:
                    t = torch.empty(6, dtype=torch.float64)
                    got[p] = t
                    ops.append(self.dist.P2POp(self.dist.irecv, t, o, tag=p))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        out = {}
        for p in range(n):
            if self.rank not in holding[p]:
                continue
            v = totals[p] if self.rank == owners[p] else got[p].numpy()
            out[p] = (v[:3].copy(), v[3:].copy())
        return out
