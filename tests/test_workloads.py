"""The seeded input generators (no method arithmetic): random sequential
insertion keeps the stated clearance between particles and to walls, and
the workloads have the stated sizes."""
import math

import numpy as np
import pytest

from paper_2312_14172_gb300 import workloads as W


def _segment_distance(p, u, hp, q, v, hq, n=401):
    # brute force: closest points sampled along both segments
    s = np.linspace(-hp, hp, n)[:, None, None] * u + p
    t = np.linspace(-hq, hq, n)[None, :, None] * v + q
    return float(np.sqrt(((s - t) ** 2).sum(-1)).min())


@pytest.mark.parametrize("bc", [0, 4, 7])
def test_grid_insertion_keeps_the_gap_between_spheres(bc):
    rng = np.random.default_rng(7)
    n = np.array([64, 48, 40])
    r = rng.uniform(2.0, 5.0, 150)
    gap = 1.5
    X = W.sequential_insertion_grid(rng, n, r, bc, gap)
    k = len(X)
    assert k > 40
    wall = np.array([(bc >> a) & 1 for a in range(3)], bool)
    d = X[:, None, :] - X[None, :, :]
    d[:, :, ~wall] -= n[~wall] * np.round(d[:, :, ~wall] / n[~wall])
    D = np.sqrt((d ** 2).sum(-1)) - (r[:k, None] + r[None, :k])
    np.fill_diagonal(D, np.inf)
    assert D.min() >= gap
    for a in np.nonzero(wall)[0]:
        assert np.all(X[:, a] - r[:k] >= gap + 0.5 - 1e-12)
        assert np.all(n[a] - 1.0 - X[:, a] - r[:k] >= gap - 0.5 - 1e-12)


def test_grid_insertion_keeps_the_gap_between_capsules():
    rng = np.random.default_rng(3)
    n = np.array([48, 48, 48])
    cnt = 40
    r = rng.uniform(1.5, 2.5, cnt)
    h = rng.uniform(0.0, 6.0, cnt)
    ax = W.body_axis_z(W.random_quaternions(rng, cnt))
    gap = 0.5
    X = W.sequential_insertion_grid(rng, n, r, 0, gap, axes=ax, half_lengths=h)
    k = len(X)
    assert k == cnt
    for i in range(k):
        for j in range(i):
            d = X[i] - X[j]
            d -= n * np.round(d / n)
            if np.linalg.norm(d) > r[i] + r[j] + h[i] + h[j] + gap:
                continue
            assert _segment_distance(X[i], ax[i], h[i], X[i] - d, ax[j], h[j]) >= r[i] + r[j] + gap - 0.05


def test_phi_matched_variants_reach_the_named_fractions_on_a_small_box():
    # the same laws on a box 1/64 of the volume: the fraction is what scales
    w = W.dense_batch_phi_matched(n=(128, 128, 256), count=50000 // 32)
    P = w["particles"]
    phi = (4.0 / 3.0 * math.pi * P["a"][:, 0] ** 3).sum() / (128 * 128 * 256)
    assert 0.17 < phi < 0.23


def test_nonspherical_with_capsules_keeps_the_volume_and_the_gap():
    """Capsules in workload 2 have the equal volume 4/3 pi r_eq^3 and aspect
    ratio (h + r) / r in the drawn range, and keep the clearance to the
    ellipsoids' and cuboids' enclosing capsules."""
    w = W.nonspherical(n=(48, 48, 48), count=24, steps=1, kinds=(W.CAPSULE, W.ELLIPSOID, W.CUBOID))
    P = w["particles"]
    shp, a = P["shape"], P["a"]
    cap = shp == W.CAPSULE
    assert cap.sum() >= 4
    V = W.particle_volumes(P)
    assert np.allclose(V, 4.0 / 3.0 * math.pi * 5.0 ** 3, rtol=1e-12)
    ar = (a[cap, 2] + a[cap, 0]) / a[cap, 0]
    assert np.all((ar >= 1.0) & (ar <= 4.0))
    assert np.all(a[cap, 1] == a[cap, 0])
    # brute-force clearance between the enclosing capsules
    r = np.where(shp == W.CUBOID, math.sqrt(2.0) * a[:, 0], a[:, 0])
    h = np.where(shp == W.ELLIPSOID, a[:, 2] - a[:, 0], a[:, 2])
    ax = W.body_axis_z(P["quat"])
    n = np.array(w["n"])
    X = P["X"]
    for i in range(len(X)):
        for j in range(i):
            d = X[i] - X[j]
            d -= n * np.round(d / n)
            if np.linalg.norm(d) > r[i] + r[j] + h[i] + h[j] + w["eps"] + 1.0:
                continue
            assert _segment_distance(X[i], ax[i], h[i], X[i] - d, ax[j], h[j]) >= r[i] + r[j] + w["eps"] + 1.0 - 0.05


def test_workloads_are_seeded_and_in_the_box():
    """The same call draws the same inputs (a fixed seed per workload), and
    every centre lies in its box with its clearance to the walls."""
    for make in (lambda: W.hindered_settling(n=(64, 48, 40), count=30, steps=1),
                 lambda: W.nonspherical(n=(48, 48, 48), count=12, steps=1,
                                        kinds=(W.CAPSULE, W.ELLIPSOID, W.CUBOID))):
        a, b = make(), make()
        for k in ("shape", "a", "X", "quat", "rho_p"):
            assert np.array_equal(a["particles"][k], b["particles"][k]), k
        n = np.array(a["n"], float)
        X = a["particles"]["X"]
        for ax in range(3):
            if (a["bc"] >> ax) & 1:  # walls: centres strictly inside the fluid cells
                assert np.all(X[:, ax] > -0.5) and np.all(X[:, ax] < n[ax] - 0.5)
            else:                    # periodic: one image in [0, n)
                assert np.all(X[:, ax] >= 0.0) and np.all(X[:, ax] < n[ax])
        if a["bc"] & 4:
            r = a["particles"]["a"][:, 0]
            assert np.all(X[:, 2] - r >= a["eps"] + 1.0 - 0.5 - 1e-12)
            assert np.all(n[2] - 1.0 - X[:, 2] - r >= a["eps"] + 1.0 - 0.5 - 1e-12)
