"""Host logic of the z-slab decomposition (paper Secs. 4.2.2-4.2.4) on the
CPU: the partition, the particle routing sets (owner, partial-force senders,
copy holders) against brute force, and the point-to-point exchanges between
processes on gloo with two and three ranks -- each particle's partial
forces reach its owner from exactly the slabs its circumscribed sphere
reaches, every holder receives the same total, and halo planes go to the
neighbouring ranks only."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2312_14172_gb300 import slabs  # noqa: E402


def test_slab_ranges_cover_the_lattice():
    for nz in (7, 48, 100):
        for s in range(1, min(nz, 9) + 1):
            r = slabs.slab_ranges(nz, s)
            assert r[0][0] == 0 and r[-1][1] == nz and len(r) == s
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slabs.slab_ranges(4, 5)


def _planes_within(zc, rad, nz, periodic):
    """Planes k whose cells (height k) lie within rad of zc, by brute force
    over periodic images."""
    out = set()
    for k in range(nz):
        for s in ((-nz, 0, nz) if periodic else (0,)):
            if abs(k + s - zc) <= rad:
                out.add(k)
    return out


@pytest.mark.parametrize("periodic", [True, False])
def test_routing_sets_against_brute_force(periodic):
    """owner: the slab of the centre's cell; senders: every slab with a
    plane within r_c + 1 of the centre (where interior cells can be), and
    no other; holders: the senders and every slab whose ghost planes the
    influence reaches."""
    nz = 40
    ranges = slabs.slab_ranges(nz, 5)
    rng = np.random.default_rng(4)
    for _ in range(300):
        zc = rng.uniform(0, nz - 1) if not periodic else rng.uniform(-0.5, nz - 0.5)
        rc = rng.uniform(0.5, 9.0)
        o = slabs.owner(zc, ranges, nz, periodic)
        k = int(np.floor(zc + 0.5)) % nz
        assert ranges[o][0] <= k < ranges[o][1]
        planes = _planes_within(zc, rc + 1.0, nz, periodic)
        want = sorted({s for s, (z0, z1) in enumerate(ranges) if planes & set(range(z0, z1))})
        got = slabs.senders(zc, rc, ranges, nz, periodic)
        assert got == want, (zc, rc, got, want)
        assert o in got
        h = slabs.holders(zc, rc + 0.25, ranges, nz, periodic)
        assert set(got) <= set(h)
        for s in h:
            z0, z1 = ranges[s]
            ext = _planes_within(zc, rc + 0.25 + 1.0, nz, periodic)
            near = {(z0 - 1) % nz if periodic else z0 - 1, z1 % nz if periodic else z1} | set(range(z0, z1))
            assert ext & near


def test_local_frame_takes_the_nearest_image():
    nz = 60
    for (z0, z1) in slabs.slab_ranges(nz, 4):
        for zc in np.linspace(-0.4, nz - 0.6, 37):
            zl = slabs.local_z(zc, z0, z1, nz, True)
            assert abs((zl + z0 - 1 - zc) / nz - round((zl + z0 - 1 - zc) / nz)) < 1e-12
            assert abs(zl - 0.5 * (z1 - z0 + 1)) <= nz / 2 + 1e-9


def test_sum_partials_adds_the_senders_only():
    n = 4
    partials = {s: (np.full((n, 3), 10.0 ** s), np.full((n, 3), -(10.0 ** s))) for s in range(3)}
    F, T = slabs.sum_partials(partials, [[0], [0, 1], [1, 2], [0, 1, 2]], n)
    assert np.all(F[:, 0] == [1, 11, 110, 111]) and np.all(T[:, 2] == [-1, -11, -110, -111])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2312_14172_gb300 import slabs as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nz = 48
    ranges = S.slab_ranges(nz, world)
    ex = S.DistributedExchange(dist, rank, world, ranges, nz, periodic=True)
    # faces: each rank sends its rank-tagged planes, receives its neighbours'
    lo = np.full((5, 3, 4), 100.0 * rank + 1.0, np.float32)
    up = np.full((5, 3, 4), 100.0 * rank + 2.0, np.float32)
    from_lo, from_up = ex.swap_faces(lo, up, (5, 3, 4), torch.float32)
    # particles: heights, radii, holders; partial forces of the ranks that send
    rng = np.random.default_rng(5)
    n = 12
    Z = rng.uniform(0, nz, n)
    rc = rng.uniform(1.0, 8.0, n)
    holding = [S.holders(Z[p], rc[p] + 0.5, ranges, nz) for p in range(n)]
    route = [S.senders(Z[p], rc[p], ranges, nz) for p in range(n)]
    partial = {p: (np.array([p, rank, 1.0]) * (1 + rank), np.array([-p, 2.0 * rank, 3.0]))
               for p in range(n) if rank in route[p]}
    totals = ex.total_forces(partial, Z, rc, holding)
    out.put((rank, from_lo, from_up, {p: (totals[p][0].tolist(), totals[p][1].tolist()) for p in totals},
             [list(h) for h in holding], route))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_point_to_point_exchanges_on_gloo(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, from_lo, from_up, totals, holding, route) in res.items():
        lower, upper = (rank - 1) % world, (rank + 1) % world
        # from the lower neighbour its upper face, from the upper its lower face
        assert np.all(from_lo == 100.0 * lower + 2.0) and np.all(from_up == 100.0 * upper + 1.0)
        for p, hs in enumerate(holding):
            assert (p in totals) == (rank in hs)
            if p not in totals:
                continue
            F = sum(np.array([p, s, 1.0]) * (1 + s) for s in route[p])
            T = sum(np.array([-p, 2.0 * s, 3.0]) for s in route[p])
            assert np.allclose(totals[p][0], F, rtol=0, atol=0) and np.allclose(totals[p][1], T, rtol=0, atol=0)
