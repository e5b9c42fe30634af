"""Checkpoint and resume of the searched state: a contraction plan (path and
sliced indices, so that a later run skips the path search of Sec. 3.2.2-3.2.3)
and the learned cost model's weights with its feature standardisation.

Files are written atomically (a temporary file renamed over the target).  A
plan file carries a fingerprint of the network it was found for; loading it
for another network, or a file whose statistics no longer match the plan it
describes, raises ValueError."""
import hashlib
import json
import os

import numpy as np

PLAN_FORMAT = "tdq-plan-1"
MODEL_FORMAT = "tdq-costmodel-1"


def _atomic_write(path, data: bytes):
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "wb") as f:
        f.write(data)
    os.replace(tmp, path)


def network_fingerprint(network):
    """SHA-256 of the network's structure: output kind, index count and every
    tensor's kind, gate, conjugation, bit and index list."""
    h = hashlib.sha256()
    h.update(json.dumps([network.output, network.n_tensors, network.n_indices]).encode())
    for i in range(network.n_tensors):
        t = network.tensor(i)
        h.update(json.dumps([t["kind"], t["gate"], t["conj"], t["bit"], t["idx"]]).encode())
    return h.hexdigest()


def save_plan(plan, path):
    pairs, sliced = plan.path()
    doc = {"format": PLAN_FORMAT, "network": network_fingerprint(plan.network),
           "path": [list(p) for p in pairs], "sliced": list(sliced), "stats": plan.stats()}
    _atomic_write(path, json.dumps(doc).encode())


def load_plan(network, path):
    """The plan stored at `path`, rebuilt for `network` (tdq_plan_from_path)."""
    from . import api
    with open(path, "rb") as f:
        doc = json.loads(f.read().decode())
    if doc.get("format") != PLAN_FORMAT:
        raise ValueError("%s: not a plan file" % path)
    if doc["network"] != network_fingerprint(network):
        raise ValueError("%s: the plan was found for another network" % path)
    plan = api.Plan(network, path=[tuple(p) for p in doc["path"]], sliced=doc["sliced"])
    if plan.stats() != doc["stats"]:
        raise ValueError("%s: the stored statistics do not match the rebuilt plan" % path)
    return plan


def save_costmodel(model, path):
    """Weights (packed FP32 vector) and the feature standardisation."""
    doc = {"format": MODEL_FORMAT, "n_features": model.F, "hidden": model.H,
           "params": model.get_params().tolist(), "mean": np.asarray(model.mean).tolist(),
           "std": np.asarray(model.std).tolist()}
    _atomic_write(path, json.dumps(doc).encode())


def load_costmodel(path, device=0):
    from .costmodel import CostModel
    with open(path, "rb") as f:
        doc = json.loads(f.read().decode())
    if doc.get("format") != MODEL_FORMAT:
        raise ValueError("%s: not a cost-model file" % path)
    m = CostModel(doc["n_features"], doc["hidden"], device=device)
    params = np.asarray(doc["params"], np.float32)
    if params.size != m.n_params:
        raise ValueError("%s: %d parameters, the model has %d" % (path, params.size, m.n_params))
    m.set_params(params)
    m.mean = np.asarray(doc["mean"], np.float32)
    m.std = np.asarray(doc["std"], np.float32)
    return m
