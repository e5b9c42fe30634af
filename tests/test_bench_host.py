"""The benchmark's host side, without a device: every workload it names is
defined with the fields the timed loop and the reference arm read, and the
reference arm's oracle timing runs on a bounded sample of the small ones."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = ("qnn12", "hea6", "ladder20", "ladder20_ps", "grid7x7_amp", "grid7x7_amp_rg", "grid5x10_lightcone",
         "hea_sv20", "multi12", "hea6_tree")


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


@pytest.mark.parametrize("name", NAMES)
def test_workload_definitions(bench, name):
    wl = bench.workload(name)
    for key in ("spec", "params", "B", "grad", "desc"):
        assert key in wl, key
    assert wl["desc"].startswith(name.split("_")[0])
    assert wl["B"] >= 1 and wl["grad"] in ("none", "adjoint", "param_shift")
    if "multi" in wl:
        m = wl["multi"]
        assert len(m["specs"]) == len(m["params"]) and wl["B"] == sum(p.shape[0] for p in m["params"])
    if "tree" in wl:
        assert wl["tree"]["output"] in ("expval", "amplitude")


@pytest.mark.parametrize("name", ["qnn12", "hea6", "multi12"])
def test_reference_arm_oracle_sample(bench, name):
    """A bounded sample of oracle rows (value and shift-rule gradient) on the
    host: a row partly done when the budget runs out counts by the
    state-vector evaluations it finished."""
    rps, rows, el, cores = bench.oracle_rows_per_s(bench.workload(name), budget_s=0.5, max_rows=2)
    assert 0 < rows <= 2 + 1e-9 and rps > 0 and cores >= 1 and np.isfinite(rps)
    rps1, rows1, _, cores1 = bench.oracle_rows_per_s(bench.workload(name), budget_s=0.2, nthreads=1)
    assert rows1 > 0 and cores1 == 1


def test_recorded_traffic_is_gated_on_sources_and_launch(bench, tmp_path, monkeypatch):
    """A DRAM-traffic record counts only for the kernel, the source files and
    the launch configuration it was captured with."""
    import json
    from paper_2301_05451_gb300 import build
    files = ["include/tdq.h", "paper_2301_05451_gb300/csrc/engine.cuh"]
    launch = {"threads": 256, "fwd_reg_bits": 4, "rev_reg_bits": 4, "tile_qubits": 12}
    rec = {"kernel": "tdq_k1r_* (reverse tile passes)", "dram_bytes_per_launch": 123.0,
           "source_digest": build.files_digest(files), "source_files": files, "launch": launch}
    (tmp_path / "profiles").mkdir()
    path = tmp_path / "profiles" / "traffic.json"

    def write(r):
        path.write_text(json.dumps({"w": r}))

    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    write(rec)
    assert bench.recorded_traffic("w", "tdq_k1r", launch) == 123.0
    assert bench.recorded_traffic("w", "tdq_k2", launch) is None  # another kernel
    assert bench.recorded_traffic("other", "tdq_k1r", launch) is None  # no record
    assert bench.recorded_traffic("w", "tdq_k1r", dict(launch, threads=128)) is None  # another launch
    write(dict(rec, source_digest="0" * 64))
    assert bench.recorded_traffic("w", "tdq_k1r", launch) is None  # other sources
