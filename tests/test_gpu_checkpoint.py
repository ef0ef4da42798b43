"""Snapshots (hlbm_checkpoint_bytes / hlbm_save / hlbm_load): a handle
restored from a snapshot holds the saved state bit for bit and continues the
run as the saving handle does; foreign, truncated or mismatched snapshots
are refused."""
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


W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _random_pops(n, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    return W[:, None, None, None] * (1.0 + amp * rng.standard_normal((19, n[2], n[1], n[0])))


def _subbox(H, precision, mode):
    from paper_2312_14172_gb300 import workloads
    w = workloads.hindered_settling(n=(70, 45, 48), count=14, steps=20)
    lat = H.from_workload(w, precision=precision)
    lat.set_mea_mode(mode)
    return w, lat


def test_fluid_only_snapshot_continues_bit_for_bit(H):
    n = (45, 20, 22)
    prm = dict(tau=0.7, fluid_force=(2e-6, -1e-6, 3e-6))
    a = H.Lattice([n + (4,)], H.make_params(**prm))
    a.set_populations(_random_pops(n, 3))
    a.step(3)
    snap = a.save()
    b = H.Lattice([n + (4,)], H.make_params(**prm))
    b.load_snapshot(snap)
    assert b.steps_done == 3
    assert np.array_equal(b.populations(), a.populations())
    a.step(4)
    b.step(4)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


@pytest.mark.parametrize("precision,mode", [("fp32", "moments"), ("fp32", "kernel"), ("fp16", "moments")])
def test_snapshot_with_particles_restores_and_continues(H, precision, mode):
    w, a = _subbox(H, precision, mode)
    a.step(7)  # odd count: the next step has the other parity
    snap = a.save()
    b = H.Lattice([w["n"] + (w["bc"],)], H.make_params(tau=w["tau"], eps=w["eps"], gravity=w["gravity"],
                                                       precision=precision,
                                                       max_particles=max(1, len(w["particles"]["shape"]))))
    b.load_snapshot(snap)
    # the restored state is the saved one, bit for bit
    assert b.steps_done == 7
    assert b.get_mea_mode() == mode
    assert np.array_equal(b.populations(), a.populations())
    sa, sb = a.particle_state(), b.particle_state()
    for k in ("X", "U", "omega", "quat", "F", "T"):
        assert np.array_equal(sa[k], sb[k]), k
    if mode == "moments":
        assert b.interior_cells() == a.interior_cells() > 0
    assert b.save() == snap
    # and the run continues exactly as the saving handle's does (the
    # momentum-exchange sums are integers, independent of the list's order)
    a.step(6)
    b.step(6)
    assert np.array_equal(a.populations(), b.populations())
    sa, sb = a.particle_state(), b.particle_state()
    for k in ("X", "U", "omega", "quat", "F", "T"):
        assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()


def test_snapshots_that_do_not_fit_are_refused(H):
    n = (40, 18, 20)
    a = H.Lattice([n + (0,)], H.make_params(tau=0.7, max_particles=2))
    a.add_particles([0], [[4.0] * 3], [[20.0, 9.0, 10.0]], rho_p=[2.0])
    a.step(2)
    snap = a.save()

    def fresh(**kw):
        dims = kw.pop("dims", n)
        bc = kw.pop("bc", 0)
        p = dict(tau=0.7, max_particles=2)
        p.update(kw)
        return H.Lattice([dims + (bc,)], H.make_params(**p))

    cases = [
        (dict(dims=(40, 18, 21)), snap),
        (dict(bc=4), snap),
        (dict(precision="fp16"), snap),
        (dict(tau=0.8), snap),
        (dict(max_particles=0), snap),
        ({}, snap[:len(snap) // 2]),
        ({}, b"XXXXXXXX" + snap[8:]),
        ({}, b""),
    ]
    for kw, data in cases:
        b = fresh(**kw)
        with pytest.raises(H.HLBMError) as e:
            b.load_snapshot(data)
        assert e.value.code == H.HLBM_ERR_ARG, (kw, len(data))
        b.close()
    # only into a new handle
    b = fresh()
    b.step(1)
    with pytest.raises(H.HLBMError) as e:
        b.load_snapshot(snap)
    assert e.value.code == H.HLBM_ERR_STATE
    b.close()
    # and the refused loads left a usable handle that accepts the snapshot
    b = fresh()
    with pytest.raises(H.HLBMError):
        b.load_snapshot(snap[:100])
    b.load_snapshot(snap)
    a.step(1)
    b.step(1)
    assert np.max(np.abs(a.populations() - b.populations()) / a.populations()) <= 1e-6
    a.close()
    b.close()
