"""The C-ABI library loads without a GPU and exports every function that
include/hlbm.h declares; argument validation that needs no GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2312_14172_gb300 import build, hlbm
    build.build()
    hlbm.load()
    return hlbm


def _declared():
    src = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hlbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("hlbm_init_lattice", "hlbm_add_particles", "hlbm_step", "hlbm_particle_state"):
        assert n in names


def test_library_exports_every_declared_symbol(H):
    import ctypes
    lib = ctypes.CDLL(H.LIB_PATH)
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(H.EXPORTS) == sorted(_declared())


def test_required_bytes_and_validation(H):
    p = H.make_params(max_particles=4)
    small = H.hlbm_required_bytes([(48, 48, 48, 0)], p)
    # 19 FP32 planes dominate
    assert 19 * 48 ** 3 * 4 <= small < 19 * 48 ** 3 * 4 + (64 << 20)
    p16 = H.make_params(max_particles=4, precision="fp16")
    assert H.hlbm_required_bytes([(48, 48, 48, 0)], p16) < small
    batch = H.hlbm_required_bytes([(48, 48, 48, 0), (33, 17, 9, 4)], p)
    assert batch > small
    for bad in (dict(tau=0.5), dict(tau=float("nan")), dict(eps=0.0), dict(precision=7),
                dict(fp16_scale_log2=17), dict(max_particles=-1), dict(bin_capacity=65)):
        kw = dict(max_particles=4)
        kw.update(bad)
        assert H.hlbm_required_bytes([(8, 8, 8, 0)], H.make_params(**kw)) == 0, bad
    assert H.hlbm_required_bytes([(0, 8, 8, 0)], p) == 0
    assert H.hlbm_required_bytes([(8, 8, 8, 9)], p) == 0


def test_init_without_gpu_fails_loudly(H):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        H.Lattice([(8, 8, 8, 0)], H.make_params())
