"""The bench's DRAM-traffic record is tied to the code it was captured on:
`bench.kernel_hash` ignores comments and blank space, changes with any code
change of the solver's sources, and does not depend on the device IC
factor's own translation unit (the solver kernels do not include it);
`bench.load_traffic` returns the figure only for a matching hash and
workload.  Runs on a copy of the sources in a temporary directory."""
import json
import os
import shutil
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    import bench

    src = os.path.join(ROOT, "paper_1312_1553_gb300", "csrc")
    dst = tmp_path / "paper_1312_1553_gb300" / "csrc"
    shutil.copytree(src, dst)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench, dst


def _edit(path, old, new):
    s = path.read_text()
    assert old in s
    path.write_text(s.replace(old, new, 1))


def test_hash_ignores_comments_and_follows_code(tree):
    bench, csrc = tree
    h0 = bench.kernel_hash()
    _edit(csrc / "nle_device.cuh", "namespace nle {", "namespace nle {\n// a new comment line\n\n")
    assert bench.kernel_hash() == h0
    _edit(csrc / "nle_device.cuh", "namespace nle {", "namespace nle {\nconstexpr int kProbe = 1;")
    assert bench.kernel_hash() != h0


def test_hash_does_not_follow_the_factor_kernel(tree):
    bench, csrc = tree
    h0 = bench.kernel_hash()
    _edit(csrc / "nle_ict.cu", "namespace nle {", "namespace nle {\nconstexpr int kProbe = 1;")
    assert bench.kernel_hash() == h0
    _edit(csrc / "nle_setup.cpp", "namespace nle {", "namespace nle {\nconstexpr int kProbe = 1;")
    assert bench.kernel_hash() != h0


def test_traffic_only_for_matching_hash_and_workload(tree):
    bench, _ = tree
    rec = {"k_newton": {"bytes_per_launch": 1.5e9, "kernel_hash": bench.kernel_hash(), "workload": "w"}}
    path = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    with open(path, "w") as fh:
        json.dump(rec, fh)
    assert bench.load_traffic("k_newton", "w") == 1.5e9
    assert bench.load_traffic("k_newton", "other") is None
    assert bench.load_traffic("k_dacg", "w") is None
    rec["k_newton"]["kernel_hash"] = "0" * 16
    with open(path, "w") as fh:
        json.dump(rec, fh)
    assert bench.load_traffic("k_newton", "w") is None

