"""Pins of the oracle's lattice Boltzmann part against the paper and the
mathematics (Sec. 3.1 of arXiv:2312.14172): velocity set, weights, equilibrium
moments, conservation, streaming, viscosity, Poiseuille flow."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q19_sec3_1.txt")


def _golden_classes():
    rows = {}
    cs2 = None
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "cs2":
            cs2 = float(Fraction(line[1]))
        else:
            rows[int(line[2])] = (int(line[1]), float(Fraction(line[3])))
    return rows, cs2


def test_velocity_set_matches_sec_3_1(O):
    c, w, opp = O.velocity_set()
    rows, cs2 = _golden_classes()
    # the set itself: rest, the 6 axis vectors, the 12 face diagonals
    want = {(0, 0, 0)}
    for a in range(3):
        for s in (1, -1):
            v = [0, 0, 0]
            v[a] = s
            want.add(tuple(v))
    for a in range(3):
        for b in range(a + 1, 3):
            for s in (1, -1):
                for t in (1, -1):
                    v = [0, 0, 0]
                    v[a], v[b] = s, t
                    want.add(tuple(v))
    assert set(map(tuple, c.tolist())) == want and len(c) == 19
    assert tuple(c[0]) == (0, 0, 0)
    assert all(np.sum(np.abs(c[1:7]), axis=1) == 1)
    assert all(np.sum(np.abs(c[7:]), axis=1) == 2)
    n2 = np.sum(c * c, axis=1)
    for k, (count, wk) in rows.items():
        assert np.sum(n2 == k) == count
        assert np.allclose(w[n2 == k], wk, rtol=0, atol=1e-17)
    assert np.all(c[opp] == -c)
    # Gauss-Hermite moment conditions of the weights
    assert abs(w.sum() - 1.0) < 1e-15
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, cs2 * np.eye(3), atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-16)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0)


@pytest.mark.parametrize("rho,u", [(1.0, (0, 0, 0)), (1.03, (0.02, -0.01, 0.005)),
                                   (0.97, (-0.05, 0.04, 0.03))])
def test_equilibrium_moments(O, rho, u):
    """Eq. maxbolt on D3Q19: zeroth, first and second moments are rho, rho u and
    rho c_s^2 I + rho u u exactly."""
    c, w, _ = O.velocity_set()
    u = np.array(u, float)
    feq = O.equilibrium(rho, u)
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
    P = np.einsum("ia,ib,i->ab", c, c, feq)
    assert np.allclose(P, rho / 3.0 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
    if not np.any(u):
        assert np.allclose(feq, rho * w, atol=1e-17)


def _random_state(O, n, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    c, w, _ = O.velocity_set()
    f = w[:, None, None, None] * (1.0 + amp * rng.standard_normal((19, n[2], n[1], n[0])))
    return f


@pytest.mark.parametrize("bc", [0, 4, 7])
def test_mass_conserved_exactly(O, bc):
    """Collision (BGK and the EDM source have zero mass) and streaming (a
    permutation, bounce-back included) conserve total mass to rounding."""
    n = (13, 12, 14)
    o = O.Oracle(n, 0.7, 0.5, bc, (0, 0, -1e-4), (1e-5, -2e-5, 3e-6))
    o.add_particles([0], [[2.0] * 3], [[4.2, 3.1, 5.3]], U=[[1e-3, -2e-3, 5e-4]],
                    omega=[[1e-3, 2e-3, -1e-3]], rho_p=[2.0])
    f0 = _random_state(O, n, 1)
    o.set_populations(f0)
    m0 = f0.sum()
    o.step(12)
    assert abs(o.populations().sum() - m0) < 1e-12 * m0


def test_momentum_conserved_without_particles(O):
    n = (8, 6, 10)
    o = O.Oracle(n, 0.9, 0.5, 0)
    c, w, _ = O.velocity_set()
    f0 = _random_state(O, n, 2)
    o.set_populations(f0)
    p0 = np.einsum("ia,izyx->a", c, f0)
    o.step(15)
    p1 = np.einsum("ia,izyx->a", c, o.populations())
    assert np.allclose(p1, p0, rtol=0, atol=1e-13)


def test_uniform_equilibrium_is_fixed_point(O):
    n = (5, 6, 7)
    o = O.Oracle(n, 0.8, 0.5, 0)
    feq = O.equilibrium(1.02, [0.03, -0.02, 0.01])
    f0 = np.broadcast_to(feq[:, None, None, None], (19, n[2], n[1], n[0])).copy()
    o.set_populations(f0)
    o.step(10)
    assert np.allclose(o.populations(), f0, rtol=0, atol=1e-15)


def test_body_force_momentum_gain_is_exact(O):
    """Eq. kupershtokh: sum_i S_i = 0 and sum_i c_i S_i = rho Delta u, so a
    uniform force density F_f (Delta u = F_f / rho) adds exactly F_f per cell
    and step to the momentum of a periodic box."""
    n = (6, 5, 4)
    F = np.array([1e-5, -3e-6, 2e-6])
    o = O.Oracle(n, 0.75, 0.5, 0, (0, 0, 0), F)
    c, w, _ = O.velocity_set()
    f0 = _random_state(O, n, 3)
    o.set_populations(f0)
    p0 = np.einsum("ia,izyx->a", c, f0)
    o.step(7)
    p1 = np.einsum("ia,izyx->a", c, o.populations())
    ncell = n[0] * n[1] * n[2]
    assert np.allclose(p1 - p0, 7 * ncell * F, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("bc", [0, 1, 6])
def test_streaming_is_the_shift_of_eq_stream(O, bc):
    """Eq. stream checked against numpy.roll; bounce-back on wall axes."""
    n = (5, 4, 6)
    o = O.Oracle(n, 0.8, 0.5, bc)
    c, w, opp = O.velocity_set()
    rng = np.random.default_rng(4)
    post = rng.random((19, n[2], n[1], n[0]))
    o.stream_only(post)
    f = o.populations()
    for i in range(19):
        want = np.roll(post[i], shift=(c[i][2], c[i][1], c[i][0]), axis=(0, 1, 2))
        # populations that crossed a wall come back by bounce-back instead
        for a, ax in ((0, 2), (1, 1), (2, 0)):
            if bc >> a & 1 and c[i][a] != 0:
                sl = [slice(None)] * 3
                sl[ax] = 0 if c[i][a] > 0 else n[a] - 1
                want[tuple(sl)] = np.nan
        bad = np.isnan(want)
        assert np.array_equal(f[i][~bad], want[~bad])
        assert np.array_equal(f[i][bad], post[opp[i]][bad])


@pytest.mark.slow
def test_shear_wave_decays_with_eq_relaxation_viscosity(O):
    """Eq. relaxation: nu = (tau - 1/2) / 3.  A shear wave u_x = A sin(k z)
    decays as exp(-nu k^2 t) (Navier-Stokes, Sec. 2.1).  The rate is read
    between two times after the start-up transient; the lattice's own
    dispersion is O(k^2) ~ 2 % of nu at k = 2 pi / 48, so 1 % is allowed
    after the k^2 term is kept small (L = 48)."""
    L = 48
    n = (1, 1, L)
    c, w, _ = O.velocity_set()
    z = np.arange(L)
    k = 2 * np.pi / L
    A = 1e-4
    for tau in (0.6, 1.1):
        o = O.Oracle(n, tau, 0.5, 0)
        f0 = np.zeros((19, L, 1, 1))
        for zz in z:
            f0[:, zz, 0, 0] = O.equilibrium(1.0, [A * np.sin(k * zz), 0, 0])
        o.set_populations(f0)
        amps = []
        for T in (100, 500):
            o.step(T - o.steps_done)
            ux = np.einsum("i,izyx->zyx", c[:, 0].astype(float), o.populations())[:, 0, 0]
            amps.append(2.0 / L * np.sum(ux * np.sin(k * z)))
        nu_meas = -np.log(amps[1] / amps[0]) / (k * k * 400)
        nu = (tau - 0.5) / 3.0
        assert abs(nu_meas / nu - 1.0) < 1e-2


def _poiseuille_error(O, tau, H=12, steps=None):
    nu = (tau - 0.5) / 3.0
    g = 1e-6
    o = O.Oracle((1, 1, H), tau, 0.5, 4, (0, 0, 0), (g, 0, 0))
    steps = steps or int(12 * H * H / nu)
    o.step(steps)
    c, w, _ = O.velocity_set()
    f = o.populations()
    rho = f.sum(axis=0)[:, 0, 0]
    jx = np.einsum("i,izyx->zyx", c[:, 0].astype(float), f)[:, 0, 0]
    ux = (jx + g / 2.0) / rho  # EDM macroscopic velocity u + Delta u / 2
    z = np.arange(H)
    exact = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    return np.max(np.abs(ux - exact)) / np.max(exact)


@pytest.mark.slow
def test_poiseuille_profile(O):
    """Body-force driven channel between half-way bounce-back walls at z = -1/2
    and z = H - 1/2: the steady Navier-Stokes solution is the parabola
    u(z) = g / (2 nu) (z + 1/2) (H - 1/2 - z).  For BGK with bounce-back the
    numerical wall sits exactly half-way when (tau - 1/2)^2 = 3/16, and is off
    by O((tau - 1/2)^2 - 3/16) / H^2 otherwise."""
    tau_exact = 0.5 + math.sqrt(3.0 / 16.0)
    assert _poiseuille_error(O, tau_exact) < 1e-9
    assert _poiseuille_error(O, 0.8) < 1e-2
    # and the error grows away from the exact relaxation time
    assert _poiseuille_error(O, 1.5) > 10 * _poiseuille_error(O, tau_exact)


def test_openmp_build_gives_identical_results():
    """The oracle built with -fopenmp (used only to time it on every host
    core) computes every cell and particle with the same operations as the
    plain build: populations and particle states agree bit for bit."""
    from oracle import oracle as O
    from paper_2312_14172_gb300 import workloads as W
    w = W.hindered_settling(n=(40, 36, 32), count=6, r_range=(3.0, 5.0), steps=3)
    res = []
    for omp in (False, True):
        o = O.from_workload(w, omp=omp)
        o.step(3)
        res.append((o.populations(), o.particle_state()))
        o.close()
    assert np.array_equal(res[0][0], res[1][0])
    for k in res[0][1]:
        assert np.array_equal(res[0][1][k], res[1][1][k]), k
    assert O.threads(False) == 1 and O.threads(True) >= 1
