"""Host logic of bench.py (no GPU): the digest of the library sources that
gates a profiled DRAM-traffic figure, the lookup of that figure in the
profile summaries, and the kernel that an autotune code launches."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

LINE = ('<!-- traffic kernel="k_xstage_apply<double, 4, 0, 0>" workload="ring-p4-nel128" '
        'bytes_per_launch=123 csrc_sha256=%s -->')


def _tree(tmp_path):
    d = tmp_path / "paper_1712_08565_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "a.cu").write_text("int x;")
    (d / "notes.txt").write_text("not a source")
    (tmp_path / "profiles").mkdir()
    return d


def test_digest_follows_the_sources(tmp_path, monkeypatch):
    d = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.csrc_digest()
    (d / "notes.txt").write_text("changed")
    assert bench.csrc_digest() == h
    (d / "a.cu").write_text("int y;")
    assert bench.csrc_digest() != h
    (d / "a.cu").write_text("int x;")
    assert bench.csrc_digest() == h
    (d / "b.cuh").write_text("")
    assert bench.csrc_digest() != h


def test_traffic_only_on_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    d = _tree(tmp_path)
    (d / "other.cu").write_text("int w;")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", {"k_xstage_apply": ["a.cu"]})
    k = "k_xstage_apply<double, 4, 0, 0>"
    (tmp_path / "profiles" / "x.md").write_text("summary\n" + LINE % bench.csrc_digest(k) + "\n")
    assert bench.profiled_traffic(k, "ring-p4-nel128") == 123
    assert bench.profiled_traffic("k_xstage_apply<double, 2, 0, 0>", "ring-p4-nel128") is None
    assert bench.profiled_traffic(k, "ring-p6-nel192") is None
    (d / "other.cu").write_text("int v;")  # a file the kernel is not built from
    assert bench.profiled_traffic(k, "ring-p4-nel128") == 123
    (d / "a.cu").write_text("int z;")  # one of its sources changed after the capture
    assert bench.profiled_traffic(k, "ring-p4-nel128") is None


@pytest.mark.parametrize("code,elem,p,name", [
    (104, "double", 4, "k_xstage_apply<double, 4, 0, 0>"),
    (1102, "double", 6, "k_xstage_apply<double, 2, 0, 1>"),
    (124, "double", 4, "k_xstage_apply<double, 4, 2, 0>"),
    (148, "float", 6, "k_xstage_tiled<float, 4, 0>"),
    (1158, "double", 3, "k_xstage_tiled<double, 8, 1>"),
    (468, "float", 6, "k_xstage_stencil<float, 6>"),
])
def test_kernel_of_an_autotune_code(code, elem, p, name):
    assert bench.xstage_kernel_name(code, elem, p) == name
