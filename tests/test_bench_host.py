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
