"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (FP32 storage of f - w, FP32 arithmetic, FP64 particle sums and
motion):
  populations       |f_gpu - f_ref| <= 1e-5 |f_ref| element by element
  particle motion   |dX_gpu - dX_ref| <= 1e-5 |dX_ref| + 1e-6 (dX = X - X0),
                    the same rule for U and omega against their own scale
FP16 storage: errors against FP64 are bounded loosely here; the stated
per-quantity figures against FP32 are the benchmark's (its fp16 and
batched_fp16 entries).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL_F = 1e-5


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2312_14172_gb300 import build, hlbm
    build.build()
    hlbm.load()
    return hlbm


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def _pops_close(fg, fo, rtol=RTOL_F):
    err = np.abs(fg - fo) / np.abs(fo)
    assert np.all(np.isfinite(fg))
    assert err.max() <= rtol, f"max relative population error {err.max():.3e}"
    return err.max()


FLOORS = {"X": 1e-6, "U": 1e-9, "omega": 1e-9}


def _motion_close(sg, so, X0, U0, W0, rtol=1e-5):
    """|d_gpu - d_ref| <= rtol * max|d_ref| + floor, d = value - initial value."""
    for key, ref0 in (("X", X0), ("U", U0), ("omega", W0)):
        dg = sg[key] - ref0
        do = so[key] - ref0
        err = np.abs(dg - do)
        scale = np.abs(do).max()
        assert err.max() <= rtol * scale + FLOORS[key], \
            f"{key}: max err {err.max():.3e}, scale {scale:.3e}"


def _random_pops(O, n, seed, amp=1e-3):
    c, w, _ = O.velocity_set()
    rng = np.random.default_rng(seed)
    return w[:, None, None, None] * (1.0 + amp * rng.standard_normal((19, n[2], n[1], n[0])))


def _pair(H, O, n, bc, tau=0.7, eps=0.5, g=(0, 0, 0), ff=(0, 0, 0), precision="fp32", maxp=1, **kw):
    lat = H.Lattice([tuple(n) + (bc,)], H.make_params(tau=tau, eps=eps, gravity=g, fluid_force=ff,
                                                      precision=precision, max_particles=maxp, **kw))
    orc = O.Oracle(n, tau, eps, bc, g, ff)
    return lat, orc


# ------------------------------------------------------------ no particles
@pytest.mark.parametrize("cells_x", [1, 2])
@pytest.mark.parametrize("nx", [45, 46])
@pytest.mark.parametrize("bc", [0, 4, 7, 3])
def test_fluid_only_random_state(H, O, bc, nx, cells_x):
    """Collision + streaming, ragged sizes spanning several tiles, every
    parity, both kernels; with an odd nx the two-cell kernel's last pair of
    a row holds one cell."""
    n = (nx, 19, 21)
    lat, orc = _pair(H, O, n, bc, tau=0.66, ff=(2e-6, -1e-6, 3e-6))
    lat.set_launch(4, 2, cells_x)
    f0 = _random_pops(O, n, 10 + bc)
    lat.set_populations(f0)
    orc.set_populations(f0)
    for steps in (1, 1, 3, 8):
        lat.step(steps)
        orc.step(steps)
        _pops_close(lat.populations(), orc.populations())
    lat.sync()
    lat.close()


@pytest.mark.parametrize("cells_x", [1, 2])
@pytest.mark.parametrize("bc", [0, 5])
def test_fluid_only_fp16_both_kernels(H, O, bc, cells_x):
    """FP16 storage of f - w (times 2^14) through both kernels, ragged odd
    nx, every parity: within the storage error of the oracle."""
    n = (45, 19, 21)
    lat, orc = _pair(H, O, n, bc, tau=0.66, ff=(2e-6, -1e-6, 3e-6), precision="fp16")
    lat.set_launch(4, 2, cells_x)
    f0 = _random_pops(O, n, 20 + bc)
    lat.set_populations(f0)
    orc.set_populations(f0)
    for steps in (1, 1, 3):
        lat.step(steps)
        orc.step(steps)
        fg, fo = lat.populations(), orc.populations()
        assert np.max(np.abs(fg - fo) / fo) < 1e-4
    lat.sync()
    lat.close()


@pytest.mark.parametrize("cells_x", [1, 2])
def test_particles_fp16_both_kernels(H, O, cells_x):
    """Spheres between walls with FP16 storage through both kernels and the
    moments form of the momentum exchange: populations within the storage
    error, particle displacements within 2 % of the oracle's."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(46, 40, 36), count=5, r_range=(3.0, 5.0), steps=10)
    P = w["particles"]
    lat = H.from_workload(w, precision="fp16")
    lat.set_mea_mode("moments")
    lat.set_launch(4, 4, cells_x)
    orc = O.from_workload(w)
    lat.step(10)
    orc.step(10)
    fg, fo = lat.populations(), orc.populations()
    assert np.max(np.abs(fg - fo) / fo) < 1e-4
    sg, so = lat.particle_state(), orc.particle_state()
    dX = so["X"] - P["X"]
    assert np.max(np.abs((sg["X"] - P["X"]) - dX)) <= 2e-2 * np.abs(dX).max() + 1e-6
    lat.close()


@pytest.mark.parametrize("cells_x", [1, 2])
def test_degenerate_thin_boxes(H, O, cells_x):
    for n, bc in (((1, 1, 16), 4), ((1, 7, 5), 0), ((33, 1, 1), 0), ((2, 2, 2), 7), ((2, 1, 16), 4),
                  ((2, 7, 5), 0), ((34, 1, 1), 1), ((4, 3, 3), 7), ((3, 2, 2), 7), ((33, 1, 1), 1),
                  ((1, 3, 3), 1)):
        lat, orc = _pair(H, O, n, bc, tau=0.9, ff=(1e-5, 0, 0))
        lat.set_launch(2, 2, cells_x)
        f0 = _random_pops(O, n, 3)
        lat.set_populations(f0)
        orc.set_populations(f0)
        lat.step(7)
        orc.step(7)
        _pops_close(lat.populations(), orc.populations())
        lat.close()


def test_set_get_roundtrip_both_parities(H, O):
    n = (40, 9, 17)
    lat, _ = _pair(H, O, n, 4)
    f0 = _random_pops(O, n, 5)
    for k in range(2):
        lat.set_populations(f0)
        got = lat.populations()
        assert np.max(np.abs(got - f0) / f0) < 1e-6  # FP32 rounding of f - w
        lat.step(1)
    lat.close()


# ------------------------------------------------------------ with particles
def _run_pair(H, O, w, steps, chunks=(1,), precision="fp32", mode="kernel"):
    P = w["particles"]
    lat = H.from_workload(w, precision=precision)
    lat.set_mea_mode(mode)
    orc = O.from_workload(w)
    X0, U0, W0 = P["X"].copy(), P["U"].copy(), P["omega"].copy()
    done = 0
    for c in chunks:
        lat.step(c)
        orc.step(c)
        done += c
    rest = steps - done
    if rest > 0:
        lat.step(rest)
        orc.step(rest)
    sg = lat.particle_state()
    so = orc.particle_state()
    fg = lat.populations()
    fo = orc.populations()
    lat.close()
    return sg, so, fg, fo, (X0, U0, W0)


@pytest.mark.parametrize("mode", ["kernel", "moments"])
def test_single_sphere_settling_200_steps(H, O, mode):
    """The small benchmark configuration in full: 48^3 periodic, one sphere
    r = 6, tau 0.8, density ratio 2.5, g = 1e-5, 200 steps."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.single_sphere()
    sg, so, fg, fo, (X0, U0, W0) = _run_pair(H, O, w, 200, chunks=(1, 1, 5), mode=mode)
    _pops_close(fg, fo)
    _motion_close(sg, so, X0, U0, W0)
    assert np.allclose(sg["F"], so["F"], rtol=1e-4, atol=1e-9)
    assert sg["U"][0][2] < 0


def test_sphere_off_centre_rotating(H, O):
    """A sphere near a periodic corner, moving and spinning: images, torque."""
    n = (40, 36, 44)
    lat, orc = _pair(H, O, n, 0, tau=0.7, g=(2e-6, -3e-6, -1e-5), maxp=2)
    args = dict(shape=[0, 0], shape_params=[[5.5] * 3, [4.2] * 3],
                X=[[0.7, 35.2, 1.9], [20.3, 17.8, 22.6]], U=[[1e-3, -2e-3, 5e-4], [0, 0, -1e-3]],
                omega=[[2e-3, -1e-3, 3e-3], [0, 4e-3, 0]], quat=None, rho_p=[2.5, 1.5])
    lat.add_particles(**args)
    orc.add_particles(args["shape"], args["shape_params"], args["X"], args["U"], args["omega"],
                      None, args["rho_p"])
    X0 = np.array(args["X"]); U0 = np.array(args["U"]); W0 = np.array(args["omega"])
    lat.step(60)
    orc.step(60)
    sg, so = lat.particle_state(), orc.particle_state()
    _pops_close(lat.populations(), orc.populations())
    _motion_close(sg, so, X0, U0, W0)
    assert np.allclose(sg["T"], so["T"], rtol=1e-3, atol=1e-8)
    # the orientation of a spinning sphere (integrated in the world frame on
    # the GPU, in the body frame by the oracle)
    assert np.allclose(sg["quat"], so["quat"], atol=1e-9)
    assert not np.allclose(sg["quat"][:, 0], 1.0)
    lat.close()


@pytest.mark.parametrize("mode", ["kernel", "moments"])
def test_hindered_settling_subbox_walls(H, O, mode):
    """Spheres between walls (the hindered-settling configuration) on a box
    the oracle finishes quickly, ragged in x and y."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(70, 45, 48), count=14, steps=50)
    assert len(w["particles"]["shape"]) >= 8
    sg, so, fg, fo, (X0, U0, W0) = _run_pair(H, O, w, 50, chunks=(1,), mode=mode)
    _pops_close(fg, fo)
    _motion_close(sg, so, X0, U0, W0)


def test_nonspherical_subbox(H, O):
    """Ellipsoids and cuboids with random orientations, eps = 1.5."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.nonspherical(n=(64, 56, 60), count=16, steps=50)
    assert len(w["particles"]["shape"]) >= 10
    # give them some spin so that the rotation update is exercised
    rng = np.random.default_rng(1)
    w["particles"]["omega"] = rng.uniform(-3e-3, 3e-3, w["particles"]["omega"].shape)
    sg, so, fg, fo, (X0, U0, W0) = _run_pair(H, O, w, 50, chunks=(1,), mode="moments")
    _pops_close(fg, fo)
    _motion_close(sg, so, X0, U0, W0)
    assert np.allclose(sg["quat"], so["quat"], atol=1e-9)


@pytest.mark.parametrize("mode", ["kernel", "moments"])
def test_capsules_subbox(H, O, mode):
    """Capsules (sphere-swept segments) among ellipsoids and cuboids, with
    random orientations and spin, eps = 1.5."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.nonspherical(n=(62, 56, 60), count=18, steps=50,
                               kinds=(workloads.CAPSULE, workloads.ELLIPSOID, workloads.CUBOID))
    assert (w["particles"]["shape"] == workloads.CAPSULE).sum() >= 4
    rng = np.random.default_rng(5)
    w["particles"]["omega"] = rng.uniform(-3e-3, 3e-3, w["particles"]["omega"].shape)
    sg, so, fg, fo, (X0, U0, W0) = _run_pair(H, O, w, 50, chunks=(1,), mode=mode)
    _pops_close(fg, fo)
    _motion_close(sg, so, X0, U0, W0)
    assert np.allclose(sg["quat"], so["quat"], atol=1e-9)


@pytest.mark.parametrize("cells_x", [1, 2])
def test_particles_across_the_periodic_seams(H, O, cells_x):
    """Particles across the periodic x, y and z seams, in the box's partial
    last tile (nx = 100), capsules with axes along x, just off it and
    oblique, an ellipsoid and a cuboid at random orientations: the
    populations and the motion stay those of the oracle."""
    n = (100, 36, 40)
    lat, orc = _pair(H, O, n, 0, tau=0.7, eps=1.5, g=(0, 0, -1e-5), maxp=8)

    def about_y(phi):
        return [math.cos(phi / 2), 0.0, math.sin(phi / 2), 0.0]

    rng = np.random.default_rng(11)
    qr = rng.standard_normal((2, 4))
    qr /= np.linalg.norm(qr, axis=1, keepdims=True)
    shape = [0, 3, 1, 2, 3, 3, 0]
    params = [[5.0] * 3, [2.5, 2.5, 5.0], [7.0, 3.0, 3.0], [4.0, 2.5, 2.0], [2.0, 2.0, 6.0], [2.0, 2.0, 5.0],
              [3.0] * 3]
    X = [[0.4, 10.0, 10.0], [92.5, 26.0, 30.0], [31.6, 20.0, 22.0], [64.2, 12.0, 30.0], [50.0, 28.0, 8.0],
         [72.0, 4.0, 18.0], [80.0, 35.5, 0.2]]
    quat = [[1.0, 0, 0, 0], about_y(math.pi / 2), list(qr[0]), list(qr[1]), about_y(math.pi / 2 - 0.04),
            about_y(math.pi / 2 - 0.02), [1.0, 0, 0, 0]]
    U = rng.uniform(-5e-3, 5e-3, (7, 3))
    W = rng.uniform(-3e-3, 3e-3, (7, 3))
    rho = [2.0] * 7
    lat.add_particles(shape=shape, shape_params=params, X=X, U=U, omega=W, quat=quat, rho_p=rho)
    orc.add_particles(shape, params, X, U, W, quat, rho)
    lat.set_launch(4, 4, cells_x)
    lat.step(30)
    orc.step(30)
    _pops_close(lat.populations(), orc.populations())
    _motion_close(lat.particle_state(), orc.particle_state(), np.array(X), U, W)
    lat.close()


def _contact_workload():
    """Particles set in contact with each other and with the lower z wall:
    spheres, a capsule, an ellipsoid and a cuboid, pairs closing in."""
    from paper_2312_14172_gb300 import workloads
    rng = np.random.default_rng(17)
    shapes = [0, 0, 3, 1, 2, 0]
    a = [[4.0] * 3, [3.5] * 3, [2.0, 2.0, 3.0], [2.2, 2.5, 4.5], [1.8, 2.2, 3.4], [3.0] * 3]
    X = np.array([[14.0, 14.0, 10.0], [14.0 + 4.0 + 3.5 + 0.4, 14.3, 10.5],  # gap 0.4
                  [34.0, 20.0, 9.0], [34.5, 20.0, 19.0],    # capsule 0.5 below the ellipsoid's capsule
                  [12.0, 32.0, 0.0], [20.3, 32.0, 3.2]])   # cuboid and sphere near the wall
    quat = workloads.random_quaternions(rng, len(shapes))
    quat[[0, 1, 2, 3, 5]] = [1, 0, 0, 0]  # capsule and ellipsoid axes along z
    # the rotated cuboid's enclosing capsule (radius |(1.8, 2.2)|, segment
    # +-3.4 along its long axis e) 0.3 above the wall at z = -1/2
    q = quat[4]
    ez = 1 - 2 * (q[1] ** 2 + q[2] ** 2)  # z component of the body z axis
    X[4, 2] = 3.4 * abs(ez) + math.hypot(1.8, 2.2) - 0.5 + 0.3
    P = workloads._particles(shapes, a, X, 2.5, quat)
    P["U"][0] = [2e-4, 0, 0]
    P["U"][1] = [-2e-4, 0, 0]
    P["U"][3] = [0, 0, -2e-4]
    P["omega"][4] = [0, 2e-3, 0]
    w = workloads._workload("contact", (46, 44, 40), workloads.WALL_Z, 0.7, 0.5, P, 60, "fp32")
    return w


@pytest.mark.parametrize("mode", ["kernel", "moments"])
def test_contact_subbox(H, O, mode):
    """The contact extension (hlbm_set_contact; repulsion between enclosing
    capsules and with the walls) against the oracle's: pairs closing in,
    a sphere resting near the wall, rotated non-spheres, gravity, 60 steps."""
    w = _contact_workload()
    k, zeta = 2e-3, 1.0
    P = w["particles"]
    lat = H.from_workload(w)
    lat.set_mea_mode(mode)
    lat.set_contact(k, zeta)
    orc = O.from_workload(w)
    orc.set_contact(k, zeta)
    Fc0, _ = orc.contact_forces()
    assert np.count_nonzero(np.abs(Fc0).sum(1)) >= 4  # contacts engaged from the start
    for c in (1, 59):
        lat.step(c)
        orc.step(c)
    sg, so = lat.particle_state(), orc.particle_state()
    _pops_close(lat.populations(), orc.populations())
    _motion_close(sg, so, P["X"], P["U"], P["omega"])
    assert np.allclose(sg["quat"], so["quat"], atol=1e-9)
    # without contact the same run ends elsewhere
    lat2 = H.from_workload(w)
    lat2.set_mea_mode(mode)
    lat2.step(60)
    s2 = lat2.particle_state()
    lat2.close()
    lat.close()
    dX = so["X"] - P["X"]
    assert np.max(np.abs(s2["X"] - sg["X"])) > 0.05 * np.abs(dX).max()


def test_contact_arguments_and_snapshot(H):
    """hlbm_set_contact refuses a negative or non-finite stiffness and a
    range <= 0; the parameters travel with a snapshot (the restored run
    continues bit for bit)."""
    w = _contact_workload()
    lat = H.from_workload(w)
    for bad in ((-1.0, 1.0), (float("nan"), 1.0), (1e-3, 0.0), (1e-3, float("inf"))):
        with pytest.raises(H.HLBMError):
            lat.set_contact(*bad)
    lat.set_contact(2e-3, 1.0)
    lat.step(5)
    snap = lat.save()
    lat.step(7)
    ref = lat.particle_state()
    P = w["particles"]
    lat2 = H.Lattice([tuple(w["n"]) + (w["bc"],)],
                     H.make_params(tau=w["tau"], eps=w["eps"], gravity=w["gravity"], max_particles=len(P["shape"])))
    lat2.load_snapshot(snap)
    lat2.step(7)
    got = lat2.particle_state()
    for key in ("X", "U", "omega", "quat", "F", "T"):
        assert np.array_equal(got[key], ref[key]), key
    lat.close()
    lat2.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_fluid_momentum_is_the_sum_of_the_moments(H, O, precision):
    """hlbm_fluid_momentum: sum over the cells of rho - 1 and of the momentum
    sum_i c_i f_i (Sec. 3.1), on the GPU, against the same sums of the
    populations the handle returns, after even and odd step counts, with
    walls and particles."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(45, 38, 36), count=5, r_range=(3.0, 5.0), steps=10)
    lat = H.from_workload(w, precision=precision)
    lat.set_fluid_force((2e-6, -1e-6, 3e-6))
    c = np.array(bench_C19())
    for k in (3, 4):
        lat.step(k)
        f = lat.populations()
        m, j = lat.fluid_momentum()
        ref_m = (f.sum(0) - 1.0).sum()
        ref_j = np.einsum("ai,izyx->a", c, f)
        assert abs(m - ref_m) <= 1e-9, (m, ref_m)
        assert np.allclose(j, ref_j, rtol=1e-6, atol=1e-9), (j, ref_j)
        assert np.abs(ref_j).max() > 1e-4
    lat.close()


def bench_C19():
    return [[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
            [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
            [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]]


def _grid_workload():
    from paper_2312_14172_gb300 import workloads
    w = workloads.grid_shapes(n=(62, 56, 60), count=16, r_eq=4.0, steps=50)
    rng = np.random.default_rng(8)
    w["particles"]["omega"] = rng.uniform(-3e-3, 3e-3, w["particles"]["omega"].shape)
    w["particles"]["U"] = rng.uniform(-1e-3, 1e-3, w["particles"]["U"].shape)
    return w


@pytest.mark.parametrize("mode", ["kernel", "moments"])
def test_grid_shapes_subbox(H, O, mode):
    """Signed-distance grid particles (rounded boxes of four aspect ratios,
    random orientations, spin and drift, eps = 1.5) against the oracle's grid
    shapes: populations and motion after 50 steps."""
    w = _grid_workload()
    assert len(w["particles"]["shape"]) >= 12 and len(w["grids"]) == 4
    sg, so, fg, fo, (X0, U0, W0) = _run_pair(H, O, w, 50, chunks=(1,), mode=mode)
    _pops_close(fg, fo)
    _motion_close(sg, so, X0, U0, W0)
    assert np.allclose(sg["quat"], so["quat"], atol=1e-9)


def test_grid_registration_and_snapshot(H):
    """hlbm_add_grid refuses what the oracle refuses (faces below eps/2, no
    negative sample, off-centre body, too many samples), a grid particle must
    name a registered grid, and a snapshot carries the grids: the restored
    run continues bit for bit."""
    from paper_2312_14172_gb300 import workloads
    w = _grid_workload()
    lat = H.from_workload(w)
    v, h = w["grids"][0]
    bad = v.copy()
    bad[0, 3, 3] = 0.0
    for values in (bad, np.abs(v) + 1.0, np.roll(v, 3, axis=2)):
        with pytest.raises(H.HLBMError):
            lat.add_grid(values, h)
    with pytest.raises(H.HLBMError):  # no room left: grid_floats holds the workload's grids
        lat.add_grid(v, h)
    lat.step(3)
    snap = lat.save()
    lat.step(4)
    ref = lat.particle_state()
    fr = lat.populations()
    P = w["particles"]
    lat2 = H.Lattice([tuple(w["n"]) + (w["bc"],)],
                     H.make_params(tau=w["tau"], eps=w["eps"], gravity=w["gravity"], max_particles=len(P["shape"]),
                                   grid_floats=sum(g[0].size for g in w["grids"])))
    lat2.load_snapshot(snap)
    lat2.step(4)
    got = lat2.particle_state()
    for key in ("X", "U", "omega", "quat", "F", "T"):
        assert np.array_equal(got[key], ref[key]), key
    assert np.array_equal(lat2.populations(), fr)
    lat.close()
    lat2.close()
    lat3 = H.Lattice([(20, 20, 20, 0)], H.make_params(max_particles=1))
    with pytest.raises(H.HLBMError):
        lat3.add_particles([4], [[0, 0, 0]], [[10.0, 10.0, 10.0]], rho_p=[2.0])
    lat3.close()


def test_fp16_storage_error_is_small(H, O):
    from paper_2312_14172_gb300 import workloads
    w = workloads.single_sphere(n=40, radius=5.0, steps=100)
    sg, so, fg, fo, (X0, U0, W0) = _run_pair(H, O, w, 100, precision="fp16")
    assert np.max(np.abs(fg - fo) / fo) < 1e-4
    dX = so["X"] - X0
    assert np.max(np.abs((sg["X"] - X0) - dX)) <= 2e-2 * np.abs(dX).max() + 1e-6


def test_set_fluid_force_equals_the_force_given_at_creation(H, O):
    """hlbm_set_fluid_force before the first step gives the same run as the
    same force in the parameters (bit for bit), and a later change takes
    effect from the next step on (the oracle with the new force from the
    same state agrees); a non-finite force is refused."""
    n = (40, 18, 20)
    ff = (3e-6, -2e-6, 4e-6)
    f0 = _random_pops(O, n, 5)
    lat_a, orc = _pair(H, O, n, 4, tau=0.7, ff=ff)
    lat_b, _ = _pair(H, O, n, 4, tau=0.7)
    lat_b.set_fluid_force(ff)
    for lat in (lat_a, lat_b):
        lat.set_populations(f0)
        lat.step(3)
    fa, fb = lat_a.populations(), lat_b.populations()
    assert np.array_equal(fa, fb)
    # change the force after three steps: the oracle with the new force
    # continues from the same populations
    ff2 = (-1e-6, 5e-6, 0.0)
    lat_b.set_fluid_force(ff2)
    lat_b.step(2)
    orc2 = O.Oracle(n, 0.7, 0.5, 4, (0, 0, 0), ff2)
    orc2.set_populations(fb)
    # the oracle stores logical populations and can continue from any step
    orc2.step(2)
    _pops_close(lat_b.populations(), orc2.populations())
    with pytest.raises(H.HLBMError) as e:
        lat_b.set_fluid_force((0.0, float("nan"), 0.0))
    assert e.value.code == H.HLBM_ERR_ARG
    lat_a.close()
    lat_b.close()


# ------------------------------------------------------------ batch
@pytest.mark.parametrize("what", ["moved", "velocities"])
def test_set_particle_state_then_steps_match_the_oracle(H, O, what):
    """A state imposed between steps (hlbm_set_particle_state) on the GPU and
    on the oracle, from the same populations, gives the same run: moved and
    turned particles take the bounding-box momentum exchange on the new
    interior cells; new velocities alone keep the recorded moments."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.nonspherical(n=(62, 56, 60), count=12, steps=20,
                               kinds=(workloads.CAPSULE, workloads.ELLIPSOID, workloads.CUBOID))
    lat = H.from_workload(w)
    lat.set_mea_mode("moments")
    orc = O.from_workload(w)
    lat.step(4)
    s = lat.particle_state()
    rng = np.random.default_rng(9)
    n = np.array(w["n"], float)
    U = rng.uniform(-1e-3, 1e-3, s["U"].shape)
    Wv = rng.uniform(-2e-3, 2e-3, s["omega"].shape)
    if what == "moved":
        X = np.mod(s["X"] + rng.uniform(-0.4, 0.4, s["X"].shape), n)
        # turned by about 0.1 rad: the clearance of the workload (eps + 1
        # between enclosing capsules) keeps the particles apart
        q = s["quat"] + 0.05 * rng.standard_normal(s["quat"].shape)
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        lat.set_particle_state(X, U, Wv, q)
        orc.set_particle_state(X, U, Wv, q)
    else:
        X, q = s["X"], s["quat"]
        lat.set_particle_state(None, U, Wv, None)
        orc.set_particle_state(X, U, Wv, q)
    orc.set_populations(lat.populations())
    X0, U0, W0 = lat.particle_state()["X"], U, Wv
    lat.step(10)
    orc.step(10)
    sg, so = lat.particle_state(), orc.particle_state()
    _pops_close(lat.populations(), orc.populations())
    _motion_close(sg, so, X0, U0, W0)
    assert np.allclose(sg["quat"], so["quat"], atol=1e-9)
    lat.close()


def test_unchanged_state_round_trip_keeps_the_run_bit_for_bit(H, O):
    """Writing back the state just read (the end-to-end pattern) changes
    nothing: the next step keeps the momentum exchange from the recorded
    moments, and the run is the one without the round trip, bit for bit
    (the orientation is normalised again on upload, to the last bit)."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(70, 45, 48), count=14, steps=20)
    a, b = H.from_workload(w), H.from_workload(w)
    for lat in (a, b):
        lat.set_mea_mode("moments")
        lat.step(5)
    for _ in range(4):
        a.step(1)
        s = b.particle_state()
        b.set_particle_state(s["X"], s["U"], s["omega"], s["quat"])
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())
    sa, sb = a.particle_state(), b.particle_state()
    for k in ("X", "U", "omega", "F", "T"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.allclose(sa["quat"], sb["quat"], rtol=0, atol=1e-15)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_reruns_are_bit_identical(H, O, precision):
    """Two runs of the same inputs agree bit for bit: the collision has no
    order-dependent sums, the bounding-box momentum exchange adds its plane
    partials in plane order, and the moments-mode one adds fixed-point
    integers, so neither the order of the interior-cell list (filled by
    atomics) nor that of a tile's particle list (likewise) shows."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.nonspherical(n=(62, 56, 60), count=18, steps=12,
                               kinds=(workloads.CAPSULE, workloads.ELLIPSOID, workloads.CUBOID))
    runs = []
    for _ in range(2):
        lat = H.from_workload(w, precision=precision)
        lat.set_mea_mode("moments")
        lat.step(12)
        runs.append((lat.populations(), lat.particle_state()))
        lat.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    for k in ("X", "U", "omega", "quat", "F", "T"):
        assert np.array_equal(runs[0][1][k], runs[1][1][k]), k


def test_batch_of_boxes_matches_separate_oracles(H, O):
    from paper_2312_14172_gb300 import workloads
    boxes = workloads.ensemble(nboxes=3, edge=(24, 40), count=(2, 5), r_range=(2.5, 4.0))
    params = H.make_params(tau=boxes[0]["tau"], eps=0.5, gravity=boxes[0]["gravity"],
                           max_particles=sum(len(b["particles"]["shape"]) for b in boxes))
    lat = H.Lattice([tuple(b["n"]) + (b["bc"],) for b in boxes], params)
    for k, b in enumerate(boxes):
        lat.add_workload_particles(b["particles"], box_id=[k] * len(b["particles"]["shape"]))
    orcs = [O.from_workload(b) for b in boxes]
    lat.step(25)
    for o in orcs:
        o.step(25)
    sg = lat.particle_state()
    p0 = 0
    for k, (b, o) in enumerate(zip(boxes, orcs)):
        _pops_close(lat.populations(box=k), o.populations())
        m = len(b["particles"]["shape"])
        so = o.particle_state()
        sub = {key: v[p0:p0 + m] for key, v in sg.items()}
        _motion_close(sub, so, b["particles"]["X"], b["particles"]["U"], b["particles"]["omega"])
        p0 += m
    lat.close()


# ------------------------------------------------------------ errors
def test_errors_are_reported(H, O):
    n = (32, 16, 16)
    lat, _ = _pair(H, O, n, 0, maxp=3, bin_capacity=1)
    # two particles sharing a 32x8x8 tile overflow a capacity of one
    lat.add_particles([0, 0], [[2.0] * 3, [2.0] * 3], [[5, 5, 5], [20, 5, 5]], rho_p=[2, 2])
    lat.step(1)
    with pytest.raises(H.HLBMError) as e:
        lat.sync()
    assert e.value.code == H.HLBM_ERR_CAPACITY
    lat.sync()  # flags were cleared
    with pytest.raises(H.HLBMError) as e:
        lat.add_particles([0], [[2.0] * 3], [[10, 10, 10]], rho_p=[2])
    assert e.value.code == H.HLBM_ERR_STATE
    # the interior cells are counted by a collision in the moments mode only
    with pytest.raises(H.HLBMError) as e:
        lat.interior_cells()
    assert e.value.code == H.HLBM_ERR_STATE
    lat.set_mea_mode("moments")
    with pytest.raises(H.HLBMError) as e:
        lat.interior_cells()  # no step since the change of mode
    assert e.value.code == H.HLBM_ERR_STATE
    lat.close()
    # a NaN population makes the density non-finite
    lat, _ = _pair(H, O, n, 0)
    f = _random_pops(O, n, 1)
    f[3, 4, 5, 6] = np.nan
    lat.set_populations(f)
    lat.step(2)
    with pytest.raises(H.HLBMError) as e:
        lat.sync()
    assert e.value.code == H.HLBM_ERR_UNSTABLE
    lat.close()
    with pytest.raises(H.HLBMError):
        H.Lattice([(8, 8, 8, 0)], H.make_params(tau=0.4))


def test_launch_shapes_agree(H, O):
    """Every collision launch shape gives the same results up to FP32 rounding
    order: the same kernel in any brick shape up to the order in which the
    momentum-exchange sums are added, the one- and two-cell kernels also up to
    the order of their FP32 operations."""
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(64, 40, 40), count=8, steps=10)
    ref = None
    for ty, tz, cx in ((1, 1, 1), (2, 8, 1), (4, 2, 1), (8, 4, 1), (8, 8, 1), (2, 2, 2), (4, 8, 2),
                       (8, 1, 2), (1, 4, 2)):
        lat = H.from_workload(w)
        lat.set_launch(ty, tz, cx)
        assert lat.get_launch() == (ty, tz, cx)
        lat.step(6)
        f = lat.populations()
        s = lat.particle_state()
        lat.close()
        if ref is None:
            ref = (f, s)
        else:
            # the kernels differ in FP32 rounding order; the force is a sum
            # of differences of populations and carries their rounding
            tol_f = 1e-6 if cx == 1 else 1e-5
            assert np.max(np.abs(f - ref[0]) / ref[0]) < 1e-6
            assert np.allclose(s["X"], ref[1]["X"], rtol=0, atol=1e-9)
            assert np.max(np.abs(s["F"] - ref[1]["F"])) <= tol_f * np.abs(ref[1]["F"]).max()


def test_autotune_leaves_the_run_where_it_was(H):
    """hlbm_autotune times its candidates on a copy of the state: a run that
    tunes after 5 steps and then takes 5 more ends where a run that takes the
    chosen shape and mode without tuning ends (bit for bit); a second tuning
    of the same configuration takes the kept choice without timing."""
    import time
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(64, 40, 40), count=8, steps=10)
    a = H.from_workload(w)
    a.step(5)
    ty, tz, cx, ms = a.autotune(nsteps=2)
    assert a.steps_done == 5
    mode = a.get_mea_mode()
    a.step(5)
    b = H.from_workload(w)
    b.step(5)
    b.set_launch(ty, tz, cx)
    b.set_mea_mode(mode)
    b.step(5)
    sa, sb = a.particle_state(), b.particle_state()
    for key in ("X", "U", "omega", "quat", "F", "T"):
        assert np.array_equal(sa[key], sb[key]), key
    assert np.array_equal(a.populations(), b.populations())
    c = H.from_workload(w)
    t0 = time.perf_counter()
    again = c.autotune(nsteps=2)
    assert again == (ty, tz, cx, ms) and time.perf_counter() - t0 < 0.5
    assert c.get_launch() == (ty, tz, cx) and c.get_mea_mode() == mode
    for lat in (a, b, c):
        lat.close()


@pytest.mark.parametrize("kind", ["spheres_walls", "nonspherical"])
def test_moment_momentum_exchange_matches_kernel(H, O, kind):
    """The momentum exchange from the arrivals and the moments the previous
    collision recorded equals the bounding-box kernel's on the same state
    (which runs on the first step after any change of state)."""
    from paper_2312_14172_gb300 import workloads
    if kind == "spheres_walls":
        w = workloads.hindered_settling(n=(64, 40, 44), count=10, steps=10)
    else:
        w = workloads.nonspherical(n=(48, 48, 52), count=8, steps=10)
    rng = np.random.default_rng(2)
    w["particles"]["omega"] = rng.uniform(-4e-3, 4e-3, w["particles"]["omega"].shape)
    w["particles"]["U"] = rng.uniform(-2e-3, 2e-3, w["particles"]["U"].shape)
    lat = H.from_workload(w)
    lat.set_mea_mode("moments")
    lat.step(7)
    s = lat.particle_state()
    f = lat.populations()
    # a second lattice with the same state: its first step uses the kernel
    P = dict(w["particles"])
    P.update(X=s["X"], U=s["U"], omega=s["omega"], quat=s["quat"])
    w2 = dict(w)
    w2["particles"] = P
    lat2 = H.from_workload(w2)
    lat2.set_populations(f)
    lat.step(1)
    lat2.step(1)
    s1, s2 = lat.particle_state(), lat2.particle_state()
    scale = np.abs(s2["F"]).max()
    assert scale > 0
    assert np.max(np.abs(s1["F"] - s2["F"])) <= 1e-5 * scale
    tscale = np.abs(s2["T"]).max()
    assert np.max(np.abs(s1["T"] - s2["T"])) <= 1e-4 * tscale + 1e-9
    assert np.max(np.abs(lat.populations() - lat2.populations()) / f) < 1e-6
    lat.close()
    lat2.close()
