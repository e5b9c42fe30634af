"""Writes the stored expected values used by the large-network parity tests.

Calls only the FP64 oracle (and the seeded workload generators for inputs):
  * the amplitude <0|U|0> of the 7x7, depth-8 random U3/CZ grid circuit
    (seeds 1004..1006), by the oracle's loop-nest contraction in its linear
    order, and of the 5x5 variant by both state vector and contraction;
  * the light-cone expectation <Z_25> of the 5x10 RZZ/RX brickwork (seed 1003)
    by the oracle's state vector on the 16-qubit cone;
  * the 20-qubit RY/RZ + CNOT-ladder workload (seed 1002, 64 parameter sets):
    sum_i <Z_i Z_i+1> of every row by the state vector, and the full gradient
    of rows 0 and 63 by the shift rule (Sec. 4.2, Eq. 10), with a SHA-256
    digest of the parameters they were computed from (c3_ladder20.json).
Run:  python tests/golden/make_golden.py [c4] [c3]   (both by default)
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2301_05451_gb300 import workloads as W  # noqa: E402


def params_digest(params):
    """SHA-256 of the float32 parameter array, so a stored value is used only
    with the inputs it was computed from."""
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(params, dtype=np.float32).tobytes()).hexdigest()


def c3():
    import numpy as np
    spec, params, _ = W.ladder20()
    vals = oracle.expvals(spec, W.resolve_angles(spec, params))[:, 0]
    grads = {}
    for b in (0, 63):
        grads[str(b)] = [float(x) for x in oracle.param_grads_param_shift(spec, params[b].astype(np.float64), None)]
    out = {"citation": "values by the FP64 oracle's state vector (tdq_oracle.c), gradients by its shift rule "
                       "(Sec. 4.2, Eq. 10, k = 1/2, s = pi/2); inputs from workloads.ladder20()",
           "params_sha256": params_digest(params), "values": [float(v) for v in vals], "grads": grads}
    with open(os.path.join(HERE, "c3_ladder20.json"), "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


def c4():
    out = {"citation": "values computed by the FP64 oracle (tdq_oracle.c); inputs from workloads.py",
           "grid_u3cz_7x7_d8": {}, "grid_u3cz_5x5_d8": {}, "brickwork_5x10_l4_z25": {}}
    for seed in (1004, 1005, 1006):
        c, p, _ = W.grid_u3cz(seed=seed, rows=7, cols=7, depth=8)
        v, peak = oracle.tn_amplitude(c, W.resolve_angles(c, p)[0], order="linear")
        out["grid_u3cz_7x7_d8"][str(seed)] = [v.real, v.imag]
    c, p, _ = W.grid_u3cz(seed=1004, rows=5, cols=5, depth=8)
    a = W.resolve_angles(c, p)
    v = oracle.amplitudes(c, a)[0, 0]
    out["grid_u3cz_5x5_d8"]["1004"] = [v.real, v.imag]
    c, p, _ = W.grid_brickwork(seed=1003)
    red, kept, qmap = oracle.lightcone(c, [25])
    a = W.resolve_angles(c, p)[:, kept, :]
    out["brickwork_5x10_l4_z25"]["1003"] = float(oracle.expvals(red, a)[0, 0])
    with open(os.path.join(HERE, "c4_values.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


def main(parts):
    for part in parts or ("c4", "c3"):
        {"c4": c4, "c3": c3}[part]()


if __name__ == "__main__":
    main(sys.argv[1:])
