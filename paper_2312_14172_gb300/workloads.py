"""Seeded synthetic inputs: lattices and particle sets of the HLBM workloads.

This module only draws inputs.  It holds none of the method's arithmetic (no
indicator, collision, force or integrator, and none of the distance
functions the method evaluates), so that the CUDA path and the FP64 oracle
can both be fed from it without sharing code.  The one piece of geometry
here samples the input shapes of the distance-grid workloads: a grid shape
is defined by its samples, which both sides then interpolate.

Random numbers come from numpy's PCG64 generator (``numpy.random.default_rng``)
seeded with 2312014172 + workload index.  Particles are placed by random
sequential insertion: a candidate centre is drawn uniformly and accepted when
its enclosing capsule (a sphere for spheres, a sphere-swept segment along the
long axis otherwise) keeps a gap of at least ``eps + 1`` lattice units to every
accepted particle (minimum image on periodic axes) and to every wall.

The workloads stand in for the hindered-settling study of the paper (Sec. 5.1:
random non-overlapping spheres in a periodic box, particles initially at rest,
fluid at rest) at the sizes of the five benchmark configurations:

  0  48^3 periodic, one sphere r = 6 at the centre, tau 0.8
  1  128^3, walls at z = 0 / z = 127, 200 spheres r ~ U(4, 8), tau 0.6
  2  256^3 periodic, 2000 ellipsoids and cuboids, aspect ratio ~ U(1, 4),
     equivalent radius 5, random orientation, eps 1.5, tau 0.6
  3  512 x 512 x 1024 periodic, 50 000 spheres, lognormal diameters
     (median 8, sigma 0.3, clipped to [4, 24]), tau 0.6
  4  64 periodic boxes of 64..96 cells per edge, 10..200 spheres of
     r ~ U(3, 7) each (capped at volume fraction 0.25), tau 0.6

Parameters the configurations leave open are fixed as: gravity 1e-5 along -z,
particle/fluid density ratio 2.5, eps 0.5 unless stated.
"""
import math

import numpy as np

SEED0 = 2312014172
SPHERE, ELLIPSOID, CUBOID, CAPSULE, GRID = 0, 1, 2, 3, 4
WALL_Z = 4


def _circ_radius(shape, a):
    if shape == SPHERE:
        return float(a[0])
    if shape == ELLIPSOID:
        return float(max(a))
    if shape == CAPSULE:
        return float(a[0] + a[2])
    return float(math.sqrt(a[0] ** 2 + a[1] ** 2 + a[2] ** 2))


def random_quaternions(rng, n):
    """Uniformly distributed unit quaternions (w, x, y, z), Shoemake's method."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    s1, s2 = np.sqrt(1.0 - u1), np.sqrt(u1)
    return np.stack([s2 * np.cos(2 * np.pi * u3), s1 * np.sin(2 * np.pi * u2),
                     s1 * np.cos(2 * np.pi * u2), s2 * np.sin(2 * np.pi * u3)], axis=1)


def _segment_distance(p, u, hp, q, v, hq):
    """Distance between the segments p +- hp u and q +- hq v (u, v unit)."""
    w0 = p - q
    b = float(u @ v)
    d = float(u @ w0)
    e = float(v @ w0)
    den = 1.0 - b * b
    if den > 1e-12:
        s = np.clip((b * e - d) / den, -hp, hp)
    else:
        s = 0.0
    t = np.clip(e + b * s, -hq, hq)
    s = np.clip(b * t - d, -hp, hp)
    return float(np.linalg.norm(w0 + s * u - t * v))


def sequential_insertion(rng, n_box, radii, bc, gap, max_tries=200000, axes=None, half_lengths=None):
    """Random sequential insertion of capsules (sphere-swept segments).

    Particle k occupies the points within radii[k] of the segment centre +-
    half_lengths[k] * axes[k] (a sphere when the half-length is 0).  A
    candidate centre is drawn uniformly and accepted when it keeps a gap to
    every accepted capsule (minimum image on periodic axes) and to the walls.
    Returns centres (k, 3) for the first k particles that could be placed.
    Uses a uniform bucket grid so that large counts stay fast.
    """
    n_box = np.asarray(n_box, float)
    radii = np.asarray(radii, float)
    count = len(radii)
    hl = np.zeros(count) if half_lengths is None else np.asarray(half_lengths, float)
    ax = np.tile([0.0, 0.0, 1.0], (count, 1)) if axes is None else np.asarray(axes, float)
    reach = radii + hl  # circumscribed radius of each capsule
    rmax = float(np.max(reach)) if count else 1.0
    bucket = 2.0 * rmax + gap
    nb = np.maximum(1, np.floor(n_box / bucket).astype(int))
    bsize = n_box / nb
    buckets = {}
    centres = []
    wall = [(bc >> a) & 1 for a in range(3)]
    for k in range(count):
        r = reach[k]
        placed = False
        lo = np.array([r + gap + 0.5 if wall[a] else 0.0 for a in range(3)])
        hi = np.array([n_box[a] - 1.0 - r - gap + 0.5 if wall[a] else n_box[a] for a in range(3)])
        if np.any(hi <= lo):
            break
        for _ in range(max_tries):
            c = lo + rng.random(3) * (hi - lo)
            b = np.floor(c / bsize).astype(int) % nb
            ok = True
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        key = tuple(((b + np.array([dx, dy, dz])) % nb).tolist())
                        for j in buckets.get(key, ()):
                            d = c - centres[j]
                            for a in range(3):
                                if not wall[a]:
                                    d[a] -= n_box[a] * np.round(d[a] / n_box[a])
                            dd = float(np.dot(d, d))
                            lim = reach[k] + reach[j] + gap
                            if dd >= lim * lim:
                                continue
                            if hl[k] == 0.0 and hl[j] == 0.0:
                                ok = False
                            else:
                                q = c - d  # image of particle j next to the candidate
                                ok = _segment_distance(c, ax[k], hl[k], q, ax[j], hl[j]) >= \
                                    radii[k] + radii[j] + gap
                            if not ok:
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                buckets.setdefault(tuple(b.tolist()), []).append(len(centres))
                centres.append(c)
                placed = True
                break
        if not placed:
            break
    return np.array(centres).reshape(-1, 3)


def sequential_insertion_spheres(rng, n_box, radii, bc, gap, batch=64, max_batches=400):
    """Random sequential insertion of spheres for boxes of up to a few thousand
    spheres: each round draws `batch` candidate centres uniformly and tests
    them against every accepted sphere at once (minimum image on periodic
    axes, the gap kept to walls); the first candidate that keeps the gap to
    all is accepted.  Returns centres (k, 3) of the first k spheres that could
    be placed within `max_batches` rounds each."""
    n_box = np.asarray(n_box, float)
    radii = np.asarray(radii, float)
    count = len(radii)
    wall = np.array([(bc >> a) & 1 for a in range(3)], bool)
    centres = np.zeros((count, 3))
    k = 0
    for j in range(count):
        r = radii[j]
        lo = np.where(wall, r + gap + 0.5, 0.0)
        hi = np.where(wall, n_box - 1.0 - r - gap + 0.5, n_box)
        if np.any(hi <= lo):
            break
        placed = False
        for _ in range(max_batches):
            c = lo + rng.random((batch, 3)) * (hi - lo)
            if k == 0:
                ok = np.ones(batch, bool)
            else:
                d = c[:, None, :] - centres[None, :k, :]
                per = ~wall
                d[:, :, per] -= n_box[per] * np.round(d[:, :, per] / n_box[per])
                lim = r + radii[:k] + gap
                ok = np.all(np.einsum("bka,bka->bk", d, d) >= lim[None, :] ** 2, axis=1)
            if ok.any():
                centres[k] = c[int(np.argmax(ok))]
                k += 1
                placed = True
                break
        if not placed:
            break
    return centres[:k].copy()


def sequential_insertion_grid(rng, n_box, radii, bc, gap, batch=64, max_batches=4000, axes=None,
                              half_lengths=None):
    """Random sequential insertion of capsules (as sequential_insertion:
    particle k occupies the points within radii[k] of the segment centre +-
    half_lengths[k] * axes[k]) for tens of thousands of particles: each
    round draws `batch` candidate centres for the next particle and tests
    them all at once against the accepted capsules of the 27 surrounding
    buckets of a uniform grid; the first candidate that keeps the gap to all
    of them (minimum image on periodic axes) and to the walls is accepted.
    Returns centres (k, 3) of the first k particles placed within
    `max_batches` rounds each."""
    n_box = np.asarray(n_box, float)
    radii = np.asarray(radii, float)
    count = len(radii)
    hl = np.zeros(count) if half_lengths is None else np.asarray(half_lengths, float)
    ax = np.tile([0.0, 0.0, 1.0], (count, 1)) if axes is None else np.asarray(axes, float)
    reach = radii + hl
    wall = np.array([(bc >> a) & 1 for a in range(3)], bool)
    per = ~wall
    bucket = 2.0 * (float(reach.max()) if count else 1.0) + gap
    nb = np.maximum(1, np.floor(n_box / bucket).astype(int))
    bsize = n_box / nb
    cap = 8
    grid = -np.ones((nb[0], nb[1], nb[2], cap), np.int64)
    fill = np.zeros((nb[0], nb[1], nb[2]), np.int64)
    offs = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    centres = np.zeros((count, 3))
    k = 0
    for j in range(count):
        r = reach[j]
        lo = np.where(wall, r + gap + 0.5, 0.0)
        hi = np.where(wall, n_box - 1.0 - r - gap + 0.5, n_box)
        if np.any(hi <= lo):
            break
        placed = False
        for _ in range(max_batches):
            c = lo + rng.random((batch, 3)) * (hi - lo)
            b = np.minimum(np.floor(c / bsize).astype(int), nb - 1)
            nbk = b[:, None, :] + offs[None, :, :]
            inb = np.ones(nbk.shape[:2], bool)  # buckets beyond a wall hold nothing
            for a in range(3):
                if per[a]:
                    nbk[:, :, a] %= nb[a]
                else:
                    inb &= (nbk[:, :, a] >= 0) & (nbk[:, :, a] < nb[a])
            nbk = np.clip(nbk, 0, nb - 1)
            idx = grid[nbk[:, :, 0], nbk[:, :, 1], nbk[:, :, 2]]  # (batch, 27, cap)
            idx = np.where(inb[:, :, None], idx, -1).reshape(batch, -1)
            valid = idx >= 0
            safe = np.where(valid, idx, 0)
            d = c[:, None, :] - centres[safe]
            d[:, :, per] -= n_box[per] * np.round(d[:, :, per] / n_box[per])
            dd = np.einsum("bka,bka->bk", d, d)
            lim = r + reach[safe] + gap
            near = valid & (dd < lim * lim)
            bi_, ki_ = np.nonzero(near)
            if len(bi_) and (hl[j] > 0.0 or np.any(hl[safe[bi_, ki_]] > 0.0)):
                # capsule distance for the pairs whose enclosing spheres meet:
                # segments c +- hl_j u and (c - d) +- hl_i v
                u, hp = ax[j], hl[j]
                other = safe[bi_, ki_]
                v, hq = ax[other], hl[other]
                dp = d[bi_, ki_]
                bb = v @ u
                dw = dp @ u
                ew = np.einsum("pa,pa->p", dp, v)
                den = 1.0 - bb * bb
                sp = np.where(den > 1e-12, np.clip((bb * ew - dw) / np.where(den > 1e-12, den, 1.0), -hp, hp), 0.0)
                tq = np.clip(ew + bb * sp, -hq, hq)
                sp = np.clip(bb * tq - dw, -hp, hp)
                seg = dp + sp[:, None] * u[None, :] - tq[:, None] * v
                segd = np.sqrt(np.einsum("pa,pa->p", seg, seg))
                near[bi_, ki_] = segd < radii[j] + radii[other] + gap
            ok = ~np.any(near, axis=1)
            if ok.any():
                i = int(np.argmax(ok))
                centres[k] = c[i]
                bi = tuple(b[i])
                if fill[bi] == grid.shape[3]:
                    grid = np.concatenate([grid, -np.ones(grid.shape[:3] + (grid.shape[3],), np.int64)], axis=3)
                grid[bi + (fill[bi],)] = k
                fill[bi] += 1
                k += 1
                placed = True
                break
        if not placed:
            break
    return centres[:k].copy()


def body_axis_z(quat):
    """World direction of the body z-axis of unit quaternions (w, x, y, z)."""
    w, x, y, z = quat[:, 0], quat[:, 1], quat[:, 2], quat[:, 3]
    return np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], axis=1)


def _particles(shape, a, X, rho_p, quat=None):
    n = len(shape)
    if quat is None:
        quat = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    return {
        "shape": np.asarray(shape, np.int32),
        "a": np.asarray(a, float).reshape(n, 3),
        "X": np.asarray(X, float).reshape(n, 3),
        "U": np.zeros((n, 3)),
        "omega": np.zeros((n, 3)),
        "quat": np.asarray(quat, float).reshape(n, 4),
        "rho_p": np.full(n, float(rho_p)),
    }


def rounded_box_grid(b, rr, h=0.5, eps=1.5, margin=1.0):
    """FP32 samples (values[z, y, x]) of the signed distance of a box of
    half-extents b with edges rounded by radius rr (the box of half-extents
    b - rr grown by rr), on a grid of spacing h centred at the origin that
    reaches eps/2 + margin beyond the shape (the input of a distance-grid
    particle)."""
    b = np.asarray(b, float)
    ext = b + 0.5 * eps + margin
    n = [2 * int(math.ceil(e / h)) + 1 for e in ext]
    ax = [(np.arange(k) - 0.5 * (k - 1)) * h for k in n]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    q = np.stack([np.abs(X), np.abs(Y), np.abs(Z)]) - (b - rr)[:, None, None, None]
    outside = np.sqrt((np.maximum(q, 0.0) ** 2).sum(0))
    inside = np.minimum(q.max(0), 0.0)
    return (outside + inside - rr).astype(np.float32), float(h)


def superellipsoid_grid(a, power=4.0, h=0.5, eps=1.5, margin=1.0):
    """FP32 samples of a signed field whose zero set is the superellipsoid
    |x/a0|^p + |y/a1|^p + |z/a2|^p = 1 (scaled so that it reads as a distance
    along the shortest semi-axis), on a grid as in rounded_box_grid."""
    a = np.asarray(a, float)
    ext = a + 0.5 * eps + margin
    n = [2 * int(math.ceil(e / h)) + 1 for e in ext]
    ax = [(np.arange(k) - 0.5 * (k - 1)) * h for k in n]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    F = (np.abs(X / a[0]) ** power + np.abs(Y / a[1]) ** power + np.abs(Z / a[2]) ** power) ** (1.0 / power)
    return ((F - 1.0) * a.min()).astype(np.float32), float(h)


def grid_shapes(n=(256, 256, 256), count=2000, r_eq=5.0, ar_values=(1.0, 2.0, 3.0, 4.0), rounding=1.0,
                tau=0.6, rho_ratio=2.5, eps=1.5, steps=500, seed_index=6, precision="fp32", name="grid_shapes"):
    """The non-spherical box with distance-grid particles: rounded boxes
    (b, b, AR b) of the volume of a sphere of radius r_eq, one grid per
    aspect ratio in ar_values, particle k using grid k mod len(ar_values),
    uniform random orientations, random sequential insertion of enclosing
    capsules (radius sqrt(2) b along the long axis)."""
    rng = np.random.default_rng(SEED0 + seed_index)
    vol = 4.0 / 3.0 * math.pi * r_eq ** 3
    grids, dims = [], []
    for ar in ar_values:
        # volume of the rounded box (b, b, AR b), solved for b by bisection
        def volume(b):
            c = np.array([b, b, ar * b]) - rounding
            return (8 * c.prod() + 8 * rounding * (c[0] * c[1] + c[1] * c[2] + c[0] * c[2])
                    + 2 * math.pi * rounding ** 2 * c.sum() + 4.0 / 3.0 * math.pi * rounding ** 3)
        lo, hi = rounding, 20.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if volume(mid) < vol else (lo, mid)
        b = 0.5 * (lo + hi)
        dims.append(np.array([b, b, ar * b]))
        grids.append(rounded_box_grid(dims[-1], rounding, eps=eps))
    kinds = [k % len(ar_values) for k in range(count)]
    quat = random_quaternions(rng, count)
    cap_r = np.array([math.sqrt(2.0) * dims[k][0] for k in kinds])
    cap_h = np.array([dims[k][2] for k in kinds])
    X = sequential_insertion(rng, n, cap_r, 0, eps + 1.0, axes=body_axis_z(quat), half_lengths=cap_h)
    m = len(X)
    P = _particles([GRID] * m, [[kinds[k], 0.0, 0.0] for k in range(m)], X, rho_ratio, quat[:m])
    w = _workload(f"{name}_{n[0]}x{n[1]}x{n[2]}_{m}", n, 0, tau, eps, P, steps, precision)
    w["grids"] = grids
    return w


def _workload(name, n, bc, tau, eps, particles, steps, precision, gravity=1e-5):
    return {"name": name, "n": tuple(int(v) for v in n), "bc": int(bc), "tau": float(tau),
            "eps": float(eps), "gravity": (0.0, 0.0, -float(gravity)), "fluid_force": (0.0, 0.0, 0.0),
            "particles": particles, "steps": int(steps), "precision": precision}


def single_sphere(n=48, radius=6.0, tau=0.8, rho_ratio=2.5, steps=200, centre=None):
    """Workload 0: one sphere in a periodic cube, fluid at rest."""
    c = np.full(3, (n - 1) / 2.0) if centre is None else np.asarray(centre, float)
    P = _particles([SPHERE], [[radius] * 3], [c], rho_ratio)
    return _workload(f"single_sphere_{n}^3", (n, n, n), 0, tau, 0.5, P, steps, "fp32")


def hindered_settling(n=(128, 128, 128), count=200, r_range=(4.0, 8.0), tau=0.6, rho_ratio=2.5,
                      eps=0.5, steps=1000, seed_index=1, walls=True):
    """Workload 1: spheres between two walls (z), periodic in x and y."""
    rng = np.random.default_rng(SEED0 + seed_index)
    radii = rng.uniform(r_range[0], r_range[1], count)
    bc = WALL_Z if walls else 0
    X = sequential_insertion(rng, n, radii, bc, eps + 1.0)
    k = len(X)
    P = _particles([SPHERE] * k, np.repeat(radii[:k, None], 3, axis=1), X, rho_ratio)
    return _workload(f"hindered_settling_{n[0]}x{n[1]}x{n[2]}_{k}", n, bc, tau, eps, P, steps, "fp32")


def nonspherical(n=(256, 256, 256), count=2000, r_eq=5.0, ar_range=(1.0, 4.0), tau=0.6,
                 rho_ratio=2.5, eps=1.5, steps=500, seed_index=2, precision="fp32", gap=None, grid=False,
                 name="nonspherical", kinds=(ELLIPSOID, CUBOID)):
    """Workload 2: prolate ellipsoids and elongated cuboids (kinds cycles
    through the shapes by index; capsules may join them) of equal volume
    4/3 pi r_eq^3, aspect ratio AR ~ U(1, 4) (longest extent over the
    width), uniform random orientation, periodic box.  gap: clearance
    between the enclosing capsules (default eps + 1); grid: the vectorised
    insertion."""
    rng = np.random.default_rng(SEED0 + seed_index)
    ar = rng.uniform(ar_range[0], ar_range[1], count)
    shapes, axes = [], []
    vol = 4.0 / 3.0 * math.pi * r_eq ** 3
    for k in range(count):
        kind = kinds[k % len(kinds)]
        if kind == ELLIPSOID:
            a = (r_eq ** 3 / ar[k]) ** (1.0 / 3.0)          # a^3 AR = r_eq^3
            axes.append([a, a, ar[k] * a])
        elif kind == CUBOID:
            h = (vol / (8.0 * ar[k])) ** (1.0 / 3.0)        # 8 h^3 AR = volume
            axes.append([h, h, ar[k] * h])
        elif kind == CAPSULE:
            # pi r^3 (2 (AR - 1) + 4/3) = volume, segment half-length (AR - 1) r
            r = (vol / (math.pi * (2.0 * (ar[k] - 1.0) + 4.0 / 3.0))) ** (1.0 / 3.0)
            axes.append([r, r, max((ar[k] - 1.0) * r, 1e-6)])
        else:
            raise ValueError(f"unknown shape {kind}")
        shapes.append(kind)
    quat = random_quaternions(rng, count)
    # enclosing capsules along the body z-axis (the long axis): an ellipsoid
    # (a, a, c) lies within radius a of the segment +-(c - a); a cuboid
    # (h, h, H) within radius sqrt(2) h of the segment +-H; a capsule is one
    cap_r = np.array([a[0] if s in (ELLIPSOID, CAPSULE) else math.sqrt(2.0) * a[0] for s, a in zip(shapes, axes)])
    cap_h = np.array([a[2] - a[0] if s == ELLIPSOID else a[2] for s, a in zip(shapes, axes)])
    g = eps + 1.0 if gap is None else gap
    insert = sequential_insertion_grid if grid else sequential_insertion
    X = insert(rng, n, cap_r, 0, g, axes=body_axis_z(quat), half_lengths=cap_h)
    k = len(X)
    quat = quat[:k]
    P = _particles(shapes[:k], axes[:k], X, rho_ratio, quat)
    return _workload(f"{name}_{n[0]}x{n[1]}x{n[2]}_{k}", n, 0, tau, eps, P, steps, precision)


def dense_batch(n=(512, 512, 1024), count=50000, median_d=8.0, sigma=0.3, tau=0.6, rho_ratio=2.5,
                eps=0.5, steps=200, seed_index=3, precision="fp16", gap=None, grid=False, name="dense_batch"):
    """Workload 3: many spheres with lognormal diameters in a large periodic
    box.  gap: clearance between spheres (default eps + 1); grid: the
    vectorised insertion."""
    rng = np.random.default_rng(SEED0 + seed_index)
    d = np.clip(median_d * np.exp(sigma * rng.standard_normal(count)), 4.0, 24.0)
    radii = d / 2.0
    g = eps + 1.0 if gap is None else gap
    X = (sequential_insertion_grid if grid else sequential_insertion)(rng, n, radii, 0, g)
    k = len(X)
    P = _particles([SPHERE] * k, np.repeat(radii[:k, None], 3, axis=1), X, rho_ratio)
    return _workload(f"{name}_{n[0]}x{n[1]}x{n[2]}_{k}", n, 0, tau, eps, P, steps, precision)


# The stated counts and size laws of workloads 2 and 3 give solid fractions
# of 0.062 and 0.075, not the 0.15 and 0.2 the configurations name.  These
# variants reach the named fractions: 4806 non-spherical particles, and
# sphere diameters of median 11.1.  Random sequential insertion with the
# usual gap of eps + 1 jams below them, so the clearance is half a cell.
def nonspherical_phi_matched(**kw):
    return nonspherical(count=4806, gap=0.5, grid=True, name="nonspherical_phi", **kw)


def dense_batch_phi_matched(**kw):
    return dense_batch(median_d=11.1, gap=0.5, grid=True, name="dense_batch_phi", **kw)


def ensemble(nboxes=64, edge=(64, 96), count=(10, 200), r_range=(3.0, 7.0), phi_max=0.25, tau=0.6,
             rho_ratio=2.5, eps=0.5, steps=500, seed_index=4):
    """Workload 4: independent periodic boxes, each with its own sphere set."""
    rng = np.random.default_rng(SEED0 + seed_index)
    boxes = []
    for b in range(nboxes):
        n = tuple(int(v) for v in rng.integers(edge[0], edge[1] + 1, 3))
        want = int(rng.integers(count[0], count[1] + 1))
        radii = rng.uniform(r_range[0], r_range[1], want)
        vol = n[0] * n[1] * n[2]
        frac = np.cumsum(4.0 / 3.0 * math.pi * radii ** 3) / vol
        keep = int(np.searchsorted(frac, phi_max, side="right"))
        radii = radii[:max(1, keep)]
        X = sequential_insertion_spheres(rng, n, radii, 0, eps + 1.0)
        k = len(X)
        P = _particles([SPHERE] * k, np.repeat(radii[:k, None], 3, axis=1), X, rho_ratio)
        boxes.append(_workload(f"box{b}", n, 0, tau, eps, P, steps, "fp32"))
    return boxes


def particle_volumes(P):
    """Volumes of the particles of a workload: 4/3 pi abc (spheres and
    ellipsoids), 8 abc (cuboids), 2 pi r^2 h + 4/3 pi r^3 (capsules)."""
    a = np.asarray(P["a"], float)
    shp = np.asarray(P["shape"])
    v = np.where(shp == CUBOID, 8.0, 4.0 / 3.0 * math.pi) * a[:, 0] * a[:, 1] * a[:, 2]
    cap = 2.0 * math.pi * a[:, 0] ** 2 * a[:, 2] + 4.0 / 3.0 * math.pi * a[:, 0] ** 3
    return np.where(shp == CAPSULE, cap, v)


def zero_net_flow(w):
    """The workload with a uniform body-force density on the fluid that
    balances the particles' weight minus buoyancy, F_f = -sum_p (rho_p - 1)
    V_p g / N_cells: the total momentum of fluid and particles then stays
    zero in a periodic box.  It stands in for the counter pressure gradient
    of the hindered-settling runs (Sec. 5.1), whose equation the paper does
    not print."""
    P = w["particles"]
    n = w["n"]
    weight = ((np.asarray(P["rho_p"], float) - 1.0) * particle_volumes(P)).sum()
    g = np.asarray(w["gravity"], float)
    out = dict(w)
    out["fluid_force"] = tuple(float(v) for v in -weight * g / (n[0] * n[1] * n[2]))
    out["name"] = w["name"] + "_zero_net_flow"
    return out


def hindered_settling_periodic(phi, d=8, box_d=8, tau=0.6, rho_ratio=2.5, eps=0.5, g=1e-5, seed_index=5):
    """Hindered settling as in the paper's runs (Sec. 5.1): monodisperse
    spheres of diameter d cells at solid fraction phi, at random without
    overlap (half a cell of clearance), in a periodic cube of box_d
    diameters, with the counter force of zero_net_flow."""
    n = int(round(box_d * d))
    r = 0.5 * d
    count = int(round(phi * n ** 3 / (4.0 / 3.0 * math.pi * r ** 3)))
    rng = np.random.default_rng(SEED0 + seed_index)
    X = sequential_insertion_grid(rng, (n, n, n), np.full(count, r), 0, 0.5)
    k = len(X)
    P = _particles([SPHERE] * k, np.full((k, 3), r), X, rho_ratio)
    w = _workload(f"hindered_periodic_{n}^3_phi{phi:g}_{k}", (n, n, n), 0, tau, eps, P, 0, "fp32", gravity=g)
    return zero_net_flow(w)


def by_index(i, **kw):
    return [single_sphere, hindered_settling, nonspherical, dense_batch, ensemble][i](**kw)
