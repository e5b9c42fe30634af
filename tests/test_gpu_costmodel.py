"""The learned cost model: K8 kernels against the FP64 oracle MLP, training,
and what ranking by predicted time gains over ranking by FLOPs on held-out
circuits (measured on the GPU)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05451_gb300 import build
    build.build()
    from paper_2301_05451_gb300 import costmodel
    return costmodel


def test_mlp_forward_and_gradients_match_fp64(cm, orc):
    import torch
    r = np.random.default_rng(5)
    M = cm.CostModel(12, 64, seed=3)
    flat = r.normal(0, 0.3, size=M.n_params).astype(np.float32)
    M.set_params(flat)
    X = r.normal(size=(77, 12)).astype(np.float32)
    t = r.normal(size=77).astype(np.float32)
    params = [p.astype(np.float64) for p in M.unpack(flat)]
    y_ref, _ = orc.mlp_forward(params, X)
    # predict() standardises with mean 0 / std 1 here
    np.testing.assert_allclose(M.predict(X), y_ref, rtol=1e-4, atol=1e-4)
    loss, g = M.loss_grad(torch.as_tensor(X).cuda(), torch.as_tensor(t).cuda())
    torch.cuda.synchronize()
    loss_ref, grads_ref = orc.mlp_loss_and_grads(params, X, t)
    assert abs(loss.item() - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
    g = g.cpu().numpy()
    gr = np.concatenate([x.reshape(-1) for x in grads_ref])
    np.testing.assert_allclose(g, gr, rtol=1e-3, atol=1e-4 * np.abs(gr).max())
    # one Adam step against the oracle's
    M.adam_step(1e-2)
    torch.cuda.synchronize()
    new_ref, _, _ = orc.adam_step(params, grads_ref, [np.zeros_like(p) for p in params],
                                  [np.zeros_like(p) for p in params], 1, lr=1e-2)
    np.testing.assert_allclose(M.get_params(), np.concatenate([p.reshape(-1) for p in new_ref]), atol=2e-5)


def test_training_fits_a_smooth_target(cm):
    r = np.random.default_rng(1)
    X = r.normal(size=(4000, 12)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.2 * X[:, 3]).astype(np.float32)
    M = cm.CostModel(12, 64, seed=7)
    losses = M.fit(X, t, epochs=600, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0]


def test_ranking_by_predicted_time_beats_flops(cm):
    """What the trained network gains over the FLOP ranking of Sec. 3.2.2.

    Train on per-launch timings of random 20-50 qubit grid brickwork
    circuits; on held-out circuits, measure every one of 16 candidate plans
    (median of 5 timed runs each), then compare the plan the network picks
    with the plan of fewest FLOPs.  The learned pick must be faster in
    geometric mean over the held-out circuits, and its regret against the
    measured best candidate lower than the FLOP pick's."""
    X, t = cm.collect(48, plans_per_circuit=4, seed=100, reps=2)
    M = cm.CostModel(12, 64, seed=11)
    losses = M.fit(X, t, epochs=1500, lr=3e-3)
    assert losses[-1] < losses[0]
    plan_lists = []
    for c in range(12):
        spec, _, _ = cm.training_circuit(5000 + c)
        _, _, plans = cm.candidates(spec, 16, 5000 + c)
        plan_lists.append(plans)
    pred = cm.rank(M, plan_lists)
    speedup, reg_learned, reg_flops = [], [], []
    for plans, pr in zip(plan_lists, pred):
        meas = np.array([cm.measure(P, reps=5)[0] for P in plans])
        il, iflop = int(np.argmin(pr)), cm.flops_choice(plans)
        speedup.append(meas[iflop] / meas[il])
        reg_learned.append(meas[il] / meas.min() - 1.0)
        reg_flops.append(meas[iflop] / meas.min() - 1.0)
    gm = float(np.exp(np.mean(np.log(speedup))))
    print("learned vs FLOP pick: geomean speed-up %.3f (min %.2f, max %.2f); mean regret vs best: "
          "learned %.3f, FLOP %.3f" % (gm, min(speedup), max(speedup), np.mean(reg_learned), np.mean(reg_flops)))
    assert gm > 1.0
    assert np.mean(reg_learned) < np.mean(reg_flops)


def test_costmodel_checkpoint_round_trip(cm, tmp_path):
    """Saved weights and standardisation reload into a model that predicts
    exactly what the saved one did."""
    from paper_2301_05451_gb300 import checkpoint
    r = np.random.default_rng(7)
    X = r.normal(size=(256, 12)).astype(np.float32)
    t = (X[:, 0] * 0.5 - X[:, 3] ** 2).astype(np.float32)
    M = cm.CostModel(12, 64, seed=3)
    M.fit(X, t, epochs=50, lr=3e-3)
    f = tmp_path / "model.json"
    checkpoint.save_costmodel(M, str(f))
    M2 = checkpoint.load_costmodel(str(f))
    np.testing.assert_array_equal(M2.predict(X[:32]), M.predict(X[:32]))
