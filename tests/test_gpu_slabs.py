"""The z-slab decomposition on one GPU: one lattice cut into two or three
slab handles (ghost planes, owned planes, HLBM_CUT_Z) advanced by the split
step, the halo exchange of the crossing slots and the routing of partial
surface forces to each particle's owner (paper Secs. 4.2.2-4.2.4), against
the FP64 oracle of the whole lattice and against one handle holding it
all.  Particles cross the slab faces, and the runs span both AA parities."""
import numpy as np
import pytest

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


def _workload(bc):
    """Spheres, an ellipsoid and a capsule across the slab faces of a
    44 x 40 x 48 box (periodic, or walls at z), moving along z."""
    from paper_2312_14172_gb300 import workloads
    shapes = [0, 0, 0, 1, 3, 0]
    a = [[5.0] * 3, [4.0] * 3, [3.5] * 3, [2.5, 3.0, 5.0], [2.5, 2.5, 3.0], [4.5] * 3]
    X = np.array([[12.0, 12.0, 15.6], [30.0, 14.0, 31.7], [20.0, 28.0, 2.0 if bc == 0 else 7.5],
                  [32.0, 30.0, 16.2], [10.0, 28.0, 32.4], [22.0, 20.0, 45.5 if bc == 0 else 40.0]])
    q = workloads.random_quaternions(np.random.default_rng(3), len(shapes))
    P = workloads._particles(shapes, a, X, 2.5, q)
    P["U"][:, 2] = [3e-3, -3e-3, -2e-3, 2e-3, -1e-3, 3e-3]
    P["omega"][3] = [1e-3, -2e-3, 3e-3]
    return workloads._workload("slabs", (44, 40, 48), bc, 0.7, 0.5, P, 40, "fp32")


@pytest.mark.parametrize("bc,nslabs,mode", [(0, 3, "kernel"), (0, 2, "moments"), (4, 3, "moments")])
def test_slabs_match_the_oracle_and_one_handle(H, O, bc, nslabs, mode):
    from paper_2312_14172_gb300 import slabs
    w = _workload(bc)
    P = w["particles"]
    sl = slabs.SlabLattice(w, nslabs, mea_mode=mode)
    one = H.from_workload(w)
    one.set_mea_mode(mode)
    orc = O.from_workload(w)
    X0, U0, W0 = P["X"].copy(), P["U"].copy(), P["omega"].copy()
    for k in (1, 1, 3, 15):
        sl.step(k)
        one.step(k)
        orc.step(k)
    fs, fo, f1 = sl.populations(), orc.populations(), one.populations()
    assert np.max(np.abs(fs - fo) / fo) <= 1e-5
    assert np.max(np.abs(fs - f1) / f1) <= 1e-6
    ss, so = sl.particle_state(), orc.particle_state()
    L = np.array(w["n"], float)
    for key, ref0 in (("X", X0), ("U", U0), ("omega", W0)):
        dg, do = ss[key] - ref0, so[key] - ref0
        if key == "X" and bc == 0:
            dg[:, 2] -= L[2] * np.round(dg[:, 2] / L[2])
            do[:, 2] -= L[2] * np.round(do[:, 2] / L[2])
        assert np.max(np.abs(dg - do)) <= 1e-5 * np.abs(do).max() + 1e-9, key
    assert np.allclose(ss["F"], so["F"], rtol=0, atol=1e-5 * np.abs(so["F"]).max())
    # particles did cross slab faces: some particle has copies in two slabs
    assert any(len(h) > 1 for h in sl.hold)
    sl.close()
    one.close()


def test_split_step_equals_the_step(H):
    """On one handle, hlbm_step_forces then hlbm_step_with_forces with the
    forces it returned gives the step bit for bit (both exchange modes), and
    the split step's rules hold."""
    w = _workload(0)
    for mode in ("kernel", "moments"):
        a, b = H.from_workload(w), H.from_workload(w)
        a.set_mea_mode(mode)
        b.set_mea_mode(mode)
        a.step(3)
        b.step(3)
        for _ in range(4):
            a.step(1)
            F, T = b.step_forces()
            with pytest.raises(H.HLBMError):
                b.step(1)  # a split step is open
            b.step_with_forces(F, T)
        sa, sb = a.particle_state(), b.particle_state()
        for key in ("X", "U", "omega", "quat", "F", "T"):
            assert np.array_equal(sa[key], sb[key]), (mode, key)
        assert np.array_equal(a.populations(), b.populations())
        with pytest.raises(H.HLBMError):
            b.step_with_forces(F, T)  # none open
        a.close()
        b.close()
