"""The benchmark workloads at their full sizes, in the launch configuration
the benchmark picks for them (two cells per thread, momentum exchange from
recorded moments), against the FP64 oracle where it finishes in seconds and
against closed forms where it does not.

  hindered settling   128^3, walls at z, 200 spheres: three steps (both
                      parities, the bounding-box momentum exchange on the
                      first step and the moments form after it), every
                      population and every particle, and the number of
                      cells inside particles (exact)
  non-spherical       256^3, 2000 ellipsoids and cuboids: two steps, every
                      particle and every population, and the number of
                      cells inside particles (exact)
  dense batch         512 x 512 x 1024, 50 000 spheres, FP16 storage: the
                      first step from rest has a closed form for every
                      particle (the fluid at rest exerts no force, so
                      U_1 = (1 - 1/rho_p) g, X_1 = X_0 + U_1, omega_1 = 0);
                      two more steps stay finite and raise no error
  ensemble            64 boxes of 64..96^3 in one batch: two steps, four
                      boxes against their own oracles

Tolerances are those of the parity tests (populations 1e-5 relative,
particle displacement 1e-5 relative + 1e-6).
"""
import numpy as np
import pytest

from test_gpu_parity import _motion_close, _pops_close

pytestmark = pytest.mark.gpu


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


def _compare(lat, orc, w, steps):
    P = w["particles"]
    X0, U0, W0 = P["X"].copy(), P["U"].copy(), P["omega"].copy()
    for n in steps:
        lat.step(n)
        orc.step(n)
    sg, so = lat.particle_state(), orc.particle_state()
    _motion_close(sg, so, X0, U0, W0)
    scale = np.abs(so["F"]).max()
    assert np.max(np.abs(sg["F"] - so["F"])) <= 1e-4 * scale + 1e-9
    _pops_close(lat.populations(), orc.populations())


def _interior_cells(lat, orc, n):
    """The cells the next momentum exchange sums over: the collision's count
    equals the oracle's (the same FP32 inside decision at the same state;
    integers, so exactly)."""
    want = sum(orc.mea(p)[2] for p in range(n))
    assert want > 0 and lat.interior_cells() == want


def test_hindered_settling_full_size(H, O):
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling()
    assert tuple(w["n"]) == (128, 128, 128) and len(w["particles"]["shape"]) == 200
    lat = H.from_workload(w)
    lat.set_mea_mode("moments")
    lat.set_launch(4, 4, 2)
    orc = O.from_workload(w)
    _compare(lat, orc, w, (1, 2))
    _interior_cells(lat, orc, 200)
    lat.close()


def test_nonspherical_full_size(H, O):
    from paper_2312_14172_gb300 import workloads
    w = workloads.nonspherical()
    assert tuple(w["n"]) == (256, 256, 256) and len(w["particles"]["shape"]) == 2000
    lat = H.from_workload(w)
    lat.set_mea_mode("moments")
    lat.set_launch(4, 8, 2)
    orc = O.from_workload(w)
    _compare(lat, orc, w, (1, 1))
    _interior_cells(lat, orc, 2000)
    lat.close()


def test_dense_batch_full_size_first_step(H):
    from paper_2312_14172_gb300 import workloads
    w = workloads.dense_batch()
    assert tuple(w["n"]) == (512, 512, 1024) and len(w["particles"]["shape"]) == 50000
    P = w["particles"]
    lat = H.from_workload(w, precision="fp16")
    lat.set_mea_mode("moments")
    lat.set_launch(4, 8, 2)
    lat.step(1)
    s = lat.particle_state()
    g = np.asarray(w["gravity"], float)
    U1 = (1.0 - 1.0 / np.asarray(P["rho_p"], float))[:, None] * g[None, :]
    assert np.all(np.abs(s["F"]) == 0.0)
    assert np.max(np.abs(s["U"] - U1)) <= 1e-12 * np.abs(U1).max()
    L = np.asarray(w["n"], float)
    dX = s["X"] - P["X"]
    dX -= L * np.round(dX / L)  # periodic wrap of a centre next to a face
    assert np.max(np.abs(dX - U1)) <= 1e-9  # positions up to 1e3: FP64 rounding of X
    assert np.all(s["omega"] == 0.0)
    lat.step(2)
    s = lat.particle_state()
    for k in ("X", "U", "omega", "F", "T"):
        assert np.all(np.isfinite(s[k]))
    # the particles fall: the fluid cannot stop them within three steps
    assert np.all(s["U"][:, 2] < 0)
    lat.close()


def test_ensemble_full_size(H, O):
    from paper_2312_14172_gb300 import workloads
    boxes = workloads.ensemble()
    assert len(boxes) == 64
    params = H.make_params(tau=boxes[0]["tau"], eps=boxes[0]["eps"], gravity=boxes[0]["gravity"],
                           max_particles=sum(len(b["particles"]["shape"]) for b in boxes))
    lat = H.Lattice([tuple(b["n"]) + (b["bc"],) for b in boxes], params)
    for k, b in enumerate(boxes):
        lat.add_workload_particles(b["particles"], box_id=[k] * len(b["particles"]["shape"]))
    lat.set_mea_mode("moments")
    lat.step(2)
    sg = lat.particle_state()
    first = np.cumsum([0] + [len(b["particles"]["shape"]) for b in boxes])
    for k in (0, 17, 40, 63):
        b = boxes[k]
        o = O.from_workload(b)
        o.step(2)
        _pops_close(lat.populations(box=k), o.populations())
        sub = {key: v[first[k]:first[k + 1]] for key, v in sg.items()}
        P = b["particles"]
        _motion_close(sub, o.particle_state(), P["X"], P["U"], P["omega"])
    lat.close()
