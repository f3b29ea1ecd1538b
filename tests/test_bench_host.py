"""Host logic of bench.py: the stored DRAM traffic is reported only for the
kernel source and apply variant it was captured on."""
import hashlib
import json

import bench


def _setup(tmp_path, variant):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cuh"
    src.write_text("// kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    entry = {"dram_bytes_per_launch": 123.0, "sources": ["kernel.cuh"], "sha256": sha, "variant": variant}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k@w": entry}))
    return src


def test_traffic_needs_matching_source_and_variant(tmp_path, monkeypatch):
    src = _setup(tmp_path, [32, 4, 4, 0, 0])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k@w", [32, 4, 4, 0, 0]) == 123.0
    assert bench.ncu_traffic("k@w") == 123.0  # no variant to compare (block tiles)
    assert bench.ncu_traffic("k@w", [16, 4, 4, 0, 0]) is None  # another variant's counters
    assert bench.ncu_traffic("missing@w", [32, 4, 4, 0, 0]) is None
    src.write_text("// kernel v2\n")  # the kernel changed since the capture
    assert bench.ncu_traffic("k@w", [32, 4, 4, 0, 0]) is None


def test_cheb_degree_list_parsing():
    class A:
        cheb_degrees = "2, 3"
    assert bench.cheb_degrees(A) == (2, 3)
    A.cheb_degrees = ""
    assert bench.cheb_degrees(A) == ()


def test_tuning_tables_pass_every_entry_through():
    """A tuned table (as heat_tuning_get returns it) is set again with all
    five entries; entries a table lacks are left to the library (None)."""
    calls = []

    class FakeLib:
        @staticmethod
        def heat_tuning_set(*args):
            calls.append(args)

    t = {"variant": [-1, 1, 0], "seg_nodes": [512, 720, 512], "pw_quads": [2, 4, 4], "open_w": [2, 2, 2],
         "loop": [0, 1, 0]}
    bench.set_table(FakeLib, t)
    assert calls[-1] == (t["variant"], t["seg_nodes"], t["pw_quads"], t["open_w"], t["loop"])
    bench.set_table(FakeLib, {"variant": [-1, 0, 0], "seg_nodes": [512] * 3})
    assert calls[-1] == ([-1, 0, 0], [512] * 3, None, None, None)
