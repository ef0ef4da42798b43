"""The allocation-free momentum exchange, hlbm_mea_noalloc.

Callers that cannot allocate device memory -- a particle code living inside
another framework's memory pool, or one whose device memory is all handed to
it by its host application -- call hlbm_mea_noalloc on populations they own;
every intermediate of that call sits in one fixed device array inside the
library.  These tests check it three ways, each on two calls in a row (the
array keeps the previous call's contents):

  * against the FP64 oracle's momentum exchange (Eqs. hlbm:mea,
    hydrodynamicforce, hydrodynamictorque) on the same populations, for FP32
    and scaled FP16 storage and for both AA parities, with and without walls;
  * against the regular momentum-exchange kernel of a handle's first step;
  * on the checks of hlbm_add_particles: centres shifted by whole periods
    give the same result, invalid particles get NaN and leave the others
    untouched.

The file is collected last so that a run that stops at the first failure has
run every other test first; it passes alone in a fresh process too (its
first call sets the array up).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
# D3Q19 in the library's order (include/hlbm.h)
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
              [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
OPP = np.array([0] + [i + 1 if i % 2 else i - 1 for i in range(1, 19)])
NX, NY, NZ = 40, 36, 44
SCALE_LOG2 = 14


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


def _particles(seed):
    """Four shapes near the box faces: the sphere's and the cuboid's interior
    cells reach the planes z = 0 and z = nz - 1 (periodic images, or the
    links into a wall), the ellipsoid and the capsule cross the x and y
    faces."""
    rng = np.random.default_rng(seed)
    shape = np.array([0, 1, 2, 3], np.int32)
    params = np.array([[5.2, 5.2, 5.2], [3.0, 4.0, 7.5], [2.0, 3.5, 4.5], [3.3, 0.0, 4.0]])
    X = np.array([[10.3, 11.7, 4.7], [NX - 6.6, 20.1, 14.8], [22.4, 6.2, NZ - 3.8], [1.2, NY - 2.4, 20.5]])
    U = rng.uniform(-2e-3, 2e-3, (4, 3))
    omega = rng.uniform(-3e-3, 3e-3, (4, 3))
    quat = rng.standard_normal((4, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    return shape, params, X, U, omega, quat


def _deviations(precision, seed):
    """Random deviations f - w as the storage holds them (FP32, or FP16 times
    2^SCALE_LOG2), and the exact FP64 value each stored number stands for."""
    rng = np.random.default_rng(seed)
    dev = 1e-3 * rng.standard_normal((19, NZ, NY, NX)) * W[:, None, None, None]
    if precision == 0:
        stored = dev.astype(np.float32)
        return stored, stored.astype(np.float64)
    stored = (dev * 2.0 ** SCALE_LOG2).astype(np.float16)
    return stored, stored.astype(np.float64) * 2.0 ** -SCALE_LOG2


def _aa_layout(dev, parity, bc):
    """The AA storage of the logical deviations dev_i(x) (post-streaming):
    parity 0 keeps slot i of x; parity 1 puts f_i(x) in slot ibar of x - c_i,
    or in slot i of x when x - c_i lies beyond a wall (z walls when bc = 4)."""
    if parity == 0:
        return dev.copy()
    S = np.empty_like(dev)
    for i in range(19):
        j = OPP[i]
        # slot j of y holds f_i(y + c_i) when y + c_i is a fluid cell
        v = dev[i]
        for ax, c in zip((2, 1, 0), C[i]):
            if c:
                v = np.roll(v, -c, axis=ax)
        S[j] = v
    if bc & 4:
        for i in range(19):
            cz = C[i][2]
            if cz == 0:
                continue
            # y + c_i beyond the wall: slot ibar of y holds f_ibar(y) instead
            z = NZ - 1 if cz > 0 else 0
            S[OPP[i], z] = dev[OPP[i], z]
    return S


def _call(H, torch, f_d, bc, precision, parity, arr, n, F, T, scale_log2=SCALE_LOG2):
    return H.hlbm_mea_noalloc(f_d.data_ptr(), NX * NY * NZ, NX, NY, NZ, bc, precision,
                              scale_log2 if precision else 0, parity, n,
                              arr["shape"].data_ptr(), arr["params"].data_ptr(), arr["X"].data_ptr(),
                              arr["U"].data_ptr(), arr["omega"].data_ptr(), arr["quat"].data_ptr(),
                              F.data_ptr(), T.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _device(torch, **kw):
    cuda = torch.device("cuda")
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(cuda) for k, v in kw.items()}


def _run_twice(H, stored, bc, precision, parity, parts, check):
    """Two calls in a row, outputs poisoned before each; check(F, T, call)."""
    import torch
    shape, params, X, U, omega, quat = parts
    n = len(shape)
    f_d = torch.from_numpy(np.ascontiguousarray(stored.reshape(19, -1))).to("cuda")
    arr = _device(torch, shape=shape, params=params, X=X, U=U, omega=omega, quat=quat)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    T = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    for call in range(2):
        F.fill_(7.0 * (-1) ** call)
        T.fill_(7.0 * (-1) ** call)
        assert _call(H, torch, f_d, bc, precision, parity, arr, n, F, T) == H.HLBM_OK
        torch.cuda.synchronize()
        check(F.cpu().numpy(), T.cpu().numpy(), call)


@pytest.mark.parametrize("bc", [0, 4])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_the_oracle(H, O, precision, parity, bc):
    """Force and torque equal the FP64 oracle's momentum exchange on the same
    populations (the oracle holds the logical f_i(x) the storage stands for)."""
    parts = _particles(5 + bc + 2 * parity + 4 * precision)
    shape, params, X, U, omega, quat = parts
    stored, dev = _deviations(precision, 17 + parity + 3 * bc)
    o = O.Oracle((NX, NY, NZ), 0.7, 0.5, bc)
    o.add_particles(shape, params, X, U=U, omega=omega, quat=quat, rho_p=[2.0] * 4)
    # fluid at rest: only the links into a wall leave a force (1/3 per
    # wall-adjacent interior cell); it is kept apart so that the tolerance
    # follows the part the populations decide
    rest = [o.mea(p) for p in range(4)]
    o.set_populations(W[:, None, None, None] + dev)
    ref = [o.mea(p) for p in range(4)]
    o.close()
    Fr, Tr = np.array([r[0] for r in rest]), np.array([r[1] for r in rest])
    Fo, To = np.array([r[0] for r in ref]), np.array([r[1] for r in ref])
    assert min(r[2] for r in ref) > 50  # interior cells per particle
    assert (np.abs(Fr).max() > 1.0) == bool(bc)
    layout = _aa_layout(stored.astype(np.float64), parity, bc).astype(stored.dtype)
    tol_F = 2e-5 * np.abs(Fo - Fr).max() + 1e-7 * np.abs(Fr).max()
    tol_T = 2e-5 * np.abs(To - Tr).max() + 1e-7 * np.abs(Tr).max()

    def check(F, T, call):
        assert np.max(np.abs(F - Fo)) <= tol_F, (call, F, Fo)
        assert np.max(np.abs(T - To)) <= tol_T, (call, T, To)

    _run_twice(H, layout, bc, precision, parity, parts, check)


@pytest.mark.parametrize("bc", [0, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_the_momentum_exchange_kernel(H, precision, bc):
    """The same populations in a handle: its first step's momentum exchange
    (bounding-box kernel, parity 0) gives the same force and torque."""
    parts = _particles(7 + bc)
    shape, params, X, U, omega, quat = parts
    stored, dev = _deviations(precision, 7 + bc)
    lat = H.Lattice([(NX, NY, NZ, bc)], H.make_params(tau=0.7, max_particles=4, precision=precision,
                                                     fp16_scale_log2=SCALE_LOG2))
    lat.set_populations(W[:, None, None, None] + dev)
    lat.add_particles(shape, params, X, U, omega, quat, rho_p=[2.0] * 4)
    lat.step(1)
    ref = lat.particle_state()
    lat.close()

    def check(F, T, call):
        assert np.max(np.abs(F - ref["F"])) <= 1e-6 * np.abs(ref["F"]).max(), call
        assert np.max(np.abs(T - ref["T"])) <= 1e-6 * np.abs(ref["T"]).max() + 1e-12, call

    _run_twice(H, stored, bc, precision, 0, parts, check)


def test_noalloc_wraps_centres_and_flags_invalid_particles(H):
    """Centres shifted by whole periods on the periodic axes give bit for bit
    the same force and torque (the centre is taken modulo the box); particles
    hlbm_add_particles would refuse get NaN and leave the valid ones alone."""
    bc = 4  # periodic x, y; walls at z
    shape, params, X, U, omega, quat = _particles(31)
    X = np.round(X * 4) / 4  # dyadic centres: a shift by whole periods is exact
    stored, _ = _deviations(0, 31)
    base = {}

    def keep(F, T, call):
        base[call] = (F.copy(), T.copy())

    _run_twice(H, stored, bc, 0, 0, (shape, params, X, U, omega, quat), keep)
    assert np.all(np.isfinite(base[0][0])) and np.abs(base[0][0]).max() > 0
    shift = np.array([[3 * NX, -2 * NY, 0], [-NX, 5 * NY, 0], [-7 * NX, NY, 0], [NX, -NY, 0]], float)

    def same(F, T, call):
        assert np.array_equal(F, base[call][0]) and np.array_equal(T, base[call][1]), call

    _run_twice(H, stored, bc, 0, 0, (shape, params, X + shift, U, omega, quat), same)

    # invalid particles appended after the four valid ones
    bad_shape = np.array([0, 1, 2, 0, 0, 7, 4], np.int32)
    bad_params = np.array([[4.0, 4, 4], [3.0, -1.0, 2.0], [2.0, 2.0, 2.0], [4.0, 4, 4], [19.0, 19, 19],
                           [3.0, 3, 3], [0.0, 0, 0]])
    bad_X = np.array([[20.0, 18, 20], [20.0, 18, 20], [20.0, 18, 20], [20.0, 18, NZ - 0.25],
                      [20.0, 18, 22], [20.0, 18, 20], [20.0, 18, 20]])
    bad_q = np.tile([1.0, 0, 0, 0], (7, 1))
    bad_q[2] = 0.0  # zero quaternion
    bad_U = np.zeros((7, 3))
    bad_U[0, 1] = np.nan  # non-finite velocity
    # 1: negative size; 3: centre beyond the upper z wall (n - 1/2);
    # 4: 2 (r + 2) >= nx; 5: unknown shape; 6: a distance grid (grids
    # belong to a handle)
    n = 4 + len(bad_shape)
    allp = (np.concatenate([shape, bad_shape]), np.concatenate([params, bad_params]),
            np.concatenate([X, bad_X]), np.concatenate([U, bad_U]),
            np.concatenate([omega, np.zeros((7, 3))]), np.concatenate([quat, bad_q]))

    def flagged(F, T, call):
        assert F.shape == (n, 3)
        assert np.all(np.isnan(F[4:])) and np.all(np.isnan(T[4:])), call
        assert np.array_equal(F[:4], base[call][0]) and np.array_equal(T[:4], base[call][1]), call

    _run_twice(H, stored, bc, 0, 0, allp, flagged)


def test_noalloc_rejects_bad_arguments(H):
    rc = H.hlbm_mea_noalloc(1, 64, 4, 4, 4, 0, H.HLBM_FP32, 0, 0, H.HLBM_NOALLOC_MAX_PARTICLES + 1,
                            1, 1, 1, None, None, None, 1, 1, None)
    assert rc == H.HLBM_ERR_ARG  # more particles than the scratch array holds
    rc = H.hlbm_mea_noalloc(1, 10, 4, 4, 4, 0, H.HLBM_FP32, 0, 0, 1, 1, 1, 1, None, None, None, 1, 1, None)
    assert rc == H.HLBM_ERR_ARG  # plane shorter than the box
    rc = H.hlbm_mea_noalloc(1, 64, 4, 4, 4, 0, H.HLBM_FP32, 0, 2, 1, 1, 1, 1, None, None, None, 1, 1, None)
    assert rc == H.HLBM_ERR_ARG  # parity other than 0 or 1
    rc = H.hlbm_mea_noalloc(None, 64, 4, 4, 4, 0, H.HLBM_FP32, 0, 0, 1, 1, 1, 1, None, None, None, 1, 1,
                            None)
    assert rc == H.HLBM_ERR_ARG  # NULL populations
