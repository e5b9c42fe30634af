"""The stored expected values under tests/golden/ still belong to the inputs
the workload generators produce, and agree with the oracle on entries that
are cheap to recompute (CPU only)."""
import hashlib
import json
import os

import numpy as np

from paper_2301_05451_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_c3_ladder20_golden_matches_generator_and_oracle(orc):
    spec, params, _ = W.ladder20()
    gold = json.load(open(os.path.join(GOLDEN, "c3_ladder20.json")))
    digest = hashlib.sha256(np.ascontiguousarray(params, dtype=np.float32).tobytes()).hexdigest()
    assert gold["params_sha256"] == digest
    assert len(gold["values"]) == 64 and sorted(gold["grads"]) == ["0", "63"]
    assert all(len(g) == spec.n_params == 240 for g in gold["grads"].values())
    # two values by the state vector
    rows = [0, 63]
    v = orc.expvals(spec, W.resolve_angles(spec, params[rows]))[:, 0]
    np.testing.assert_allclose(v, np.asarray(gold["values"])[rows], rtol=0, atol=1e-12)
    # a few gradient entries of row 63 by the shift rule on single angles
    ang = W.resolve_angles(spec, params[63:64])[0]
    which = [(0, 0), (1, 0), (59, 0), (300, 0), (353, 0)]
    which = [(g, i) for g, i in which if spec.gates[g].angles]
    ag = orc.angle_grads_param_shift(spec, ang, which=which)
    for g, i in which:
        col = spec.gates[g].angles[i][1]
        assert abs(gold["grads"]["63"][col] - ag[g, i]) < 1e-12
    # the sum rule: each column is fed by exactly one angle in this circuit
    assert sum(1 for gt in spec.gates for a in gt.angles if a[0] == "p") == 240
