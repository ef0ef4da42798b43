"""Host-side helpers of the benchmark that need no GPU: the kernel-source
hash that ties a committed ncu traffic figure to the code it was taken on,
and the solid fraction of a workload."""
import math
import os
import shutil
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2312_14172_gb300 import workloads  # noqa: E402

SOURCES = ("lbm_pair_kernels.cu", "lbm_common.cuh", "hlbm_internal.cuh")


def _copy(tmp):
    d = os.path.join(tmp, "paper_2312_14172_gb300", "csrc")
    os.makedirs(d)
    for f in SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_2312_14172_gb300", "csrc", f), d)
    return d


def _hash_at(root, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", root)
    return bench.kernel_source_hash(2)


def test_source_hash_ignores_comments_and_sees_code(tmp_path, monkeypatch):
    d = _copy(str(tmp_path))
    h0 = _hash_at(str(tmp_path), monkeypatch)
    path = os.path.join(d, "lbm_common.cuh")
    src = open(path).read()
    # a changed or added comment, line or block, leaves the hash alone
    open(path, "w").write(src.replace("#pragma once", "// a new note\n#pragma once /* aside */", 1))
    assert _hash_at(str(tmp_path), monkeypatch) == h0
    # a changed constant does not
    assert "MAX_CAND = 64" in src
    open(path, "w").write(src.replace("MAX_CAND = 64", "MAX_CAND = 32", 1))
    assert _hash_at(str(tmp_path), monkeypatch) != h0


def test_solid_fraction_counts_every_shape():
    P = {"shape": np.array([workloads.SPHERE, workloads.ELLIPSOID, workloads.CUBOID, workloads.CAPSULE]),
         "a": np.array([[2.0, 2.0, 2.0], [1.0, 2.0, 3.0], [1.0, 2.0, 3.0], [1.5, 1.5, 4.0]])}
    V = (4 / 3 * math.pi * 8 + 4 / 3 * math.pi * 6 + 8 * 6
         + math.pi * 1.5 ** 2 * 8 + 4 / 3 * math.pi * 1.5 ** 3)
    assert abs(bench.solid_fraction(P, 1000) - V / 1000) < 1e-12


def test_state_errors_measures_each_quantity():
    """The per-quantity error table of the FP16/FP32-against-FP64 entries:
    a known perturbation of one quantity shows up in that quantity alone,
    with the stated normalisations."""
    rng = np.random.default_rng(3)
    n = (6, 5, 4)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = w[:, None, None, None] * (1 + 1e-2 * rng.standard_normal((19, 4, 5, 6)))
    st = {"X": np.array([[1.0, 2.0, 1.5], [5.5, 0.2, 2.0]]), "U": rng.standard_normal((2, 3)),
          "omega": rng.standard_normal((2, 3)), "F": rng.standard_normal((2, 3)),
          "T": rng.standard_normal((2, 3))}
    X0 = st["X"] - np.array([[0.5, 0.0, 0.0], [0.0, -0.25, 0.0]])
    ref = {"f": f, "state": st}
    same = bench.state_errors(ref, {"f": f.copy(), "state": {k: v.copy() for k, v in st.items()}}, n, 4, X0)
    assert all(v["max"] == 0 and v["l2"] == 0 for v in same.values())
    g = {k: v.copy() for k, v in st.items()}
    g["F"][1] += [0.0, 3e-3, 4e-3]  # |dF| = 5e-3 on one particle
    g["X"][0, 0] += 0.5 - 6.0        # displacement 0.5 -> 1.0, seen through the periodic wrap
    e = bench.state_errors(ref, {"f": f, "state": g}, n, 4, X0)
    assert abs(e["F"]["max"] - 5e-3 / np.linalg.norm(st["F"], axis=1).max()) < 1e-12
    assert abs(e["X"]["max"] - 0.5 / 0.5) < 1e-12
    assert e["rho"]["max"] == 0 and e["T"]["max"] == 0 and e["U"]["l2"] == 0
    # a uniform density change of 1e-6 relative
    e = bench.state_errors(ref, {"f": f * (1 + 1e-6), "state": st}, n, 4, X0)
    assert abs(e["rho"]["max"] - 1e-6) < 1e-12 and e["u"]["max"] < 1e-12
    # the output velocity with the forcing shift: B = 1 at one cell owned by particle 0
    B = np.zeros((4, 5, 6))
    pid = -np.ones((4, 5, 6), int)
    B[1, 2, 3], pid[1, 2, 3] = 1.0, 0
    g = {k: v.copy() for k, v in st.items()}
    g["U"][0] += [2e-3, 0, 0]
    e = bench.state_errors(ref, {"f": f, "state": g}, n, 4, X0, coupling=(B, pid))
    u = np.einsum("ai,izyx->azyx", bench.C19, f) / f.sum(0)
    r = np.array([3.0, 2.0, 1.0]) - st["X"][0]
    r[:2] -= np.array(n[:2]) * np.round(r[:2] / np.array(n[:2]))
    up = st["U"][0] + np.cross(st["omega"][0], r)
    us = u.copy()
    us[:, 1, 2, 3] = u[:, 1, 2, 3] + 0.5 * (up - u[:, 1, 2, 3])
    assert abs(e["u_out"]["max"] - 1e-3 / np.linalg.norm(us, axis=0).max()) < 1e-12


def test_settling_correlations_of_the_paper():
    """The three correlations of Sec. 5 as written there: all give 1 at
    phi = 0; Richardson-Zaki's index is 4.65 below Re = 0.2, 4.35 Re^-0.03
    up to 1, 4.45 Re^-0.1 up to 500 and 2.39 beyond; Garside-Al-Dibouni's
    tends to 5.1 for small Re and to 2.7 for large; Barnea-Mizrahi does not
    depend on Re."""
    c0 = bench.settling_correlations(0.0, 5.0)
    assert c0["richardson_zaki"] == 1.0 and c0["garside_al_dibouni"] == 1.0 and c0["barnea_mizrahi"] == 1.0
    assert bench.settling_correlations(0.1, 0.1)["n_rz"] == 4.65
    assert abs(bench.settling_correlations(0.1, 0.5)["n_rz"] - 4.35 * 0.5 ** -0.03) < 1e-15
    assert abs(bench.settling_correlations(0.1, 30.0)["n_rz"] - 4.45 * 30.0 ** -0.1) < 1e-15
    assert bench.settling_correlations(0.1, 600.0)["n_rz"] == 2.39
    assert abs(bench.settling_correlations(0.1, 1e-9)["n_gad"] - 5.1) < 1e-6
    assert abs(bench.settling_correlations(0.1, 1e9)["n_gad"] - 2.7) < 1e-6
    phi = 0.2
    bm = (1 - phi) / ((1 + phi ** (1 / 3)) * math.exp(5 * phi / (3 * (1 - phi))))
    for re in (0.1, 10.0, 100.0):
        c = bench.settling_correlations(phi, re)
        assert abs(c["barnea_mizrahi"] - bm) < 1e-15
        assert abs(c["richardson_zaki"] - (1 - phi) ** c["n_rz"]) < 1e-15


def test_clock_sampler_keeps_the_samples_inside_the_timed_window():
    """The clocks entry counts only samples taken inside the timed window
    (median SM clock, the reasons seen there)."""
    import threading
    import bench
    s = bench.ClockSampler(0)
    s.rows = [(1.0, 1900.0, 2070.0, []), (2.0, 2000.0, 2070.0, ["sw_power_cap"]), (3.0, 2070.0, 2070.0, []),
              (9.0, 500.0, 2070.0, ["hw_slowdown"])]
    s.thread = threading.Thread(target=lambda: None)
    s.thread.start()
    s.mark(1.5, 3.5, 0.0, 0.0)
    c = s.stop()
    assert c["samples"] == 2 and c["sm_mhz"] == 2035.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["in_window"] and c["source"] == "nvml"
