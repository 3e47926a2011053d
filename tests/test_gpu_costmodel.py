"""The learned cost model on the GPU, against the FP64 reference in oracle/costmodel.py.

* features: the CUDA features of lattice tetrahedra against the float64 restatement;
* gradients: one training step's gradient against the float64 backward pass (FP32 mode
  to 1e-4, BF16 mode to 2e-2, relative in norm per parameter block);
* forward: tensor-core predictions against the float64 forward pass (BF16 tolerance);
* labels: the per-tetrahedron counts sum to the deposit's own counters, and the
  overlapped-cell counts agree with the oracle's exact overlaps;
* the gain: a trained model predicts the partial clips of unseen tetrahedra with at
  least 10% lower RMSE (of log(1 + clips)) than the best affine fit on the log of the
  bounding-box cell count (the method without the model), and the binned schedule driven
  by it deposits the same masses.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import costmodel as ocm  # noqa: E402
import paper_1612_09491_gb300 as pse  # noqa: E402
from paper_1612_09491_gb300 import costmodel as cm  # noqa: E402
from paper_1612_09491_gb300.metrics import cell_errors  # noqa: E402
from pse_inputs import config_positions, zeldovich_positions, CONFIGS  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1612_09491_gb300 import build
    build.build()
    pse._lib.load()
    yield


def _sample_tets(pos, n, g, ids):
    return [oracle.lattice_tet(pos, n, int(t // 6), int(t % 6)) * g for t in ids]


@pytest.mark.parametrize("case", ["config1", "shell"])
def test_features_match_oracle(case):
    if case == "config1":
        cfg = CONFIGS[1]
        pos, n, g = config_positions(cfg), cfg.n, cfg.grid_n
    else:
        pos, n, g = zeldovich_positions(16, -1.5, 3.0, seed=77), 16, 48
    f = cm.features(torch.from_numpy(pos).cuda(), n, g).cpu().numpy()
    ids = np.random.default_rng(1).choice(6 * n ** 3, 400, replace=False)
    ref = np.array([ocm.features(v) for v in _sample_tets(pos, n, g, ids)])
    got = f[ids]
    # the bounding-box cell count can differ where a float32 vertex sits on a cell plane
    same_box = np.abs(got[:, 6] - ref[:, 6]) < 1e-6
    assert same_box.mean() > 0.99
    lin = [0, 1, 2, 9, 10, 11, 13, 15]
    np.testing.assert_allclose(got[:, lin], ref[:, lin], rtol=1e-4, atol=1e-5)
    frac = np.abs(got[:, 3:6] - ref[:, 3:6])
    assert np.all(np.minimum(frac, 1 - frac) < 1e-4)  # offsets, up to wrapping at 1
    logs = [7, 8, 12, 14]
    np.testing.assert_allclose(got[same_box][:, logs], ref[same_box][:, logs], rtol=0, atol=2e-4)


def _model_and_batch(seed=1, B=512):
    rng = np.random.default_rng(seed)
    p = ocm.init(seed)
    mu = rng.normal(0, 1, 16)
    sigma = rng.uniform(0.5, 2.0, 16)
    f = rng.normal(0, 1, (B, 16)) * sigma + mu
    t = rng.normal(0, 1, (B, 2))
    params = {"mu": mu, "sigma": sigma, **p}
    return params, f, t


@pytest.mark.parametrize("flags,tol", [(pse._lib.PSE_TRAIN_FP32, 1e-4), (0, 2e-2)])
def test_gradient_matches_oracle(flags, tol):
    params, f, t = _model_and_batch()
    m = cm.CostModel(cm.pack(params))
    # the float32 parameters are what both sides evaluate
    p32 = cm.unpack(cm.pack(params))
    pd = {k: p32[k].astype(np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    z = (f.astype(np.float32).astype(np.float64) - p32["mu"]) / p32["sigma"]
    ref = ocm.backward(pd, z, t.astype(np.float32).astype(np.float64))
    m.train_step(torch.from_numpy(f.astype(np.float32)).cuda(), torch.from_numpy(t.astype(np.float32)).cuda(),
                 lr=0.0, flags=flags | pse._lib.PSE_TRAIN_GRAD_ONLY)
    _, g = m.get()
    g = cm.unpack(g)
    for k in ref:
        err = np.linalg.norm(g[k] - ref[k]) / np.linalg.norm(ref[k])
        assert err <= tol, (k, err)
    loss = float(m.loss.item())
    assert loss == pytest.approx(ocm.loss(pd, z, t.astype(np.float32).astype(np.float64)), rel=tol)


def test_forward_matches_oracle():
    params, f, _ = _model_and_batch(seed=2, B=1000)
    m = cm.CostModel(cm.pack(params))
    got = m.predict(torch.from_numpy(f.astype(np.float32)).cuda()).cpu().numpy()
    p32 = cm.unpack(cm.pack(params))
    pd = {k: p32[k].astype(np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    ref, _ = ocm.forward(pd, (f.astype(np.float32).astype(np.float64) - p32["mu"]) / p32["sigma"])
    err = np.abs(got - ref) / (np.abs(ref) + 1.0)
    assert err.max() <= 3e-2 and err.mean() <= 5e-3, (err.max(), err.mean())


def test_adam_step_matches_oracle():
    params, f, t = _model_and_batch(seed=3)
    m = cm.CostModel(cm.pack(params))
    m.train_step(torch.from_numpy(f.astype(np.float32)).cuda(), torch.from_numpy(t.astype(np.float32)).cuda(),
                 lr=1e-2, flags=pse._lib.PSE_TRAIN_FP32)
    got = cm.unpack(m.get()[0])
    p32 = cm.unpack(cm.pack(params))
    pd = {k: p32[k].astype(np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    z = (f.astype(np.float32).astype(np.float64) - p32["mu"]) / p32["sigma"]
    g = ocm.backward(pd, z, t.astype(np.float32).astype(np.float64))
    mo = {k: np.zeros_like(v) for k, v in pd.items()}
    vo = {k: np.zeros_like(v) for k, v in pd.items()}
    ocm.adam(pd, mo, vo, g, step=1, lr=1e-2)
    for k in pd:
        # a first Adam step moves every weight by about lr * sign(g); entries with |g| near
        # float32 rounding may go either way
        d = np.abs(got[k] - pd[k])
        assert np.mean(d < 1e-4) > 0.97, k


def test_labels_sum_to_deposit_counters():
    cfg = CONFIGS[1]
    pos = torch.from_numpy(config_positions(cfg)).cuda()
    c = cm.tet_counts(pos, cfg.n, cfg.grid_n).cpu().numpy().astype(np.int64)
    _, st = pse.deposit_uniform(pos, cfg.n, cfg.grid_n, schedule=pse.PSE_THREAD_PER_TET, stats=True)
    assert c[:, 1].sum() == st["partial_clips"]
    assert np.all(c[:, 0] >= 1)
    # overlapped cells against the oracle's exact overlaps, on a sample
    posh = config_positions(cfg)
    ids = np.random.default_rng(4).choice(cfg.n_tets, 300, replace=False)
    h = np.full(3, 1.0 / cfg.grid_n)
    # the label counts cells whose overlap exceeds 1e-6 of the cell volume
    exact = np.array([np.count_nonzero(oracle.tet_cells(oracle.lattice_tet(posh, cfg.n, int(t // 6), int(t % 6)),
                                                        h)[1] > 1e-6 * h.prod()) for t in ids])
    assert np.mean(c[ids, 0] == exact) > 0.97


def _dataset(pos, n, g):
    p = torch.from_numpy(pos).cuda()
    return cm.features(p, n, g), cm.labels(cm.tet_counts(p, n, g))


def test_trained_model_beats_bbox_estimate_and_keeps_masses():
    # training data: two displacement fields; test data: an unseen one
    train = [_dataset(zeldovich_positions(32, -2.0, 2.0, seed=s), 32, 64) for s in (101, 102)]
    feat = torch.cat([d[0] for d in train])
    targ = torch.cat([d[1] for d in train])
    mu, sd = cm.standardisation(feat.cpu().numpy())
    model = cm.CostModel(cm.pack({**cm.he_init(0), "mu": mu, "sigma": sd}))
    hist = cm.fit(model, feat, targ, steps=3000, batch=4096, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    tf, tt = _dataset(zeldovich_positions(32, -2.0, 2.0, seed=103), 32, 64)
    pred = model.predict(tf).cpu().numpy()
    y = tt.cpu().numpy()[:, 1]
    # the method without the model: the best affine fit of the target on log(bbox cells)
    x_tr = feat.cpu().numpy()[:, 6] * np.log(2.0)
    A = np.stack([x_tr, np.ones_like(x_tr)], 1)
    coef, *_ = np.linalg.lstsq(A, targ.cpu().numpy()[:, 1], rcond=None)
    base = np.stack([tf.cpu().numpy()[:, 6] * np.log(2.0), np.ones(len(y))], 1) @ coef
    rmse_model = float(np.sqrt(np.mean((pred[:, 1] - y) ** 2)))
    rmse_bbox = float(np.sqrt(np.mean((base - y) ** 2)))
    print(f"partial-clip estimate on unseen tetrahedra: RMSE(log1p) model {rmse_model:.4f}, bbox fit {rmse_bbox:.4f}")
    assert rmse_model < 0.9 * rmse_bbox, (rmse_model, rmse_bbox)
    # scheduling by the model leaves the deposit unchanged
    pos = torch.from_numpy(zeldovich_positions(32, -2.0, 2.0, seed=103)).cuda()
    a, sa = pse.deposit_uniform(pos, 32, 64, schedule=pse.PSE_WARP_COOPERATIVE, stats=True)
    b, sb = pse.deposit_uniform(pos, 32, 64, schedule=pse.PSE_BINNED_PERSISTENT, cost_model=model,
                                tuning={"split_cells": 8, "chunk_cells": 16}, stats=True)
    for k in ("tets", "bbox_cells", "inside_cells", "partial_clips", "fp64_redos"):
        assert sa[k] == sb[k], k
    e = cell_errors(b.cpu().numpy(), a.cpu().numpy())
    assert e["max_rel"] <= 2e-6 and e["mass"] <= 1e-13, e
