"""GPU: the learned prefilter's kernels against its FP64 CPU oracle.

* the loss and its gradient from the GPU backward kernels against FP64 finite
  differences of the oracle's forward (relative 1e-3 of the largest entry);
* inference: the FP32 CUDA-core forward within 1e-5 of the oracle, the BF16
  tensor-core forward within BF16 rounding;
* training lowers the loss, and the trained network beats the untrained one
  on held-out pairs;
* the learned path reaches Recall@10 >= 0.99 against the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2606_15476_gb300 as F
    return F


def init_params(rng, D, H, P):
    return [(rng.standard_normal((H, D)) / math.sqrt(D)).astype(np.float32),
            (0.05 * rng.standard_normal(H)).astype(np.float32),
            (rng.standard_normal((P, H)) / math.sqrt(H)).astype(np.float32),
            (0.05 * rng.standard_normal(P)).astype(np.float32)]


def unit(x):
    x = np.asarray(x, np.float64)
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def test_gradient_matches_oracle_finite_differences(F):
    rng = np.random.default_rng(0)
    D, H, P = 40, 64, 64
    params = init_params(rng, D, H, P)
    xq = unit(rng.standard_normal((24, D))).astype(np.float32)
    xd = unit(rng.standard_normal((24, D))).astype(np.float32)
    y = rng.uniform(-0.5, 1.0, 24).astype(np.float32)
    w = rng.uniform(0.5, 2.0, 24).astype(np.float32)
    ctx = F.farm_create(0)
    try:
        F.farm_mlp_set(ctx, *params)
        n = H * D + H + P * H + P
        loss, grad = F.farm_mlp_loss_grad(ctx, xq, xd, y, w, n)
    finally:
        F.farm_destroy(ctx)
    p64 = [p.astype(np.float64) for p in params]
    assert loss == pytest.approx(omlp.loss(p64, xq, xd, y, w), rel=1e-5)
    idx = np.concatenate([rng.choice(H * D, 120, replace=False), H * D + np.arange(H),
                          H * D + H + rng.choice(P * H, 120, replace=False), H * D + H + P * H + np.arange(P)])
    fd = omlp.fd_grad(p64, xq, xd, y, w, idx=idx)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(grad[idx], fd, rtol=0, atol=1e-3 * scale)


def test_inference_matches_oracle_forward(F):
    rng = np.random.default_rng(1)
    D, H, P = 200, 128, 64
    params = init_params(rng, D, H, P)
    x = rng.standard_normal((300, D)).astype(np.float32)
    ctx = F.farm_create(0)
    try:
        F.farm_mlp_set(ctx, *params)
        e32 = F.farm_mlp_embed(ctx, x, P, F.PREC_FP32_SIMT)
        ebf = F.farm_mlp_embed(ctx, x, P, F.PREC_BF16)
    finally:
        F.farm_destroy(ctx)
    ref = omlp.forward([p.astype(np.float64) for p in params], unit(x))
    np.testing.assert_allclose(e32, ref, rtol=0, atol=1e-5)
    # BF16 weights, activations and outputs: a few parts in 2^-8 per entry
    np.testing.assert_allclose(ebf, ref, rtol=0, atol=3e-2)
    assert np.mean(np.abs(ebf - ref)) < 5e-3


def _self_supervised_pairs(F, ctx, sc, scene_id, n_rows, per_row_top, per_row_rand, seed):
    """Proxy queries = a sample of the scene's own descriptors; each is paired with
    its best objects by the library's FP32-accurate cosine and with random ones."""
    rng = np.random.default_rng(seed)
    rows_idx = rng.choice(sc.n, n_rows, replace=False)
    rows = sc.desc[rows_idx]
    S = F.farm_similarity(ctx, scene_id, rows, sc.n, F.PREC_FP32)
    top = np.argpartition(-S, per_row_top, axis=1)[:, :per_row_top]
    rnd = rng.integers(0, sc.n, size=(n_rows, per_row_rand))
    objs = np.concatenate([top, rnd], axis=1)
    pr = np.repeat(np.arange(n_rows), objs.shape[1]).astype(np.int32)
    po = objs.ravel().astype(np.int32)
    y = S[pr, po].astype(np.float32)
    w = np.concatenate([np.full((n_rows, per_row_top), 4.0), np.ones((n_rows, per_row_rand))], axis=1).ravel()
    return rows, pr, po, y, w.astype(np.float32)


def test_training_lowers_loss_and_generalises(F):
    sc = synth.make_scene(31, 4000, 256, extent=(40.0, 40.0, 6.0), n_classes=60, n_views=4)
    rng = np.random.default_rng(2)
    D, H, P = 256, 256, 64
    params = init_params(rng, D, H, P)
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        F.farm_mlp_set(ctx, *params)
        rows, pr, po, y, w = _self_supervised_pairs(F, ctx, sc, 0, 400, 64, 192, seed=3)
        # targets from the library's FP32-accurate similarity agree with the oracle
        for r in range(0, 400, 97):
            ref = oracle.cosines(sc, rows[r])
            sel = pr == r
            np.testing.assert_allclose(y[sel], ref[po[sel]], atol=1e-5)
        hold = _self_supervised_pairs(F, ctx, sc, 0, 100, 64, 192, seed=4)
        xq, xd = unit(hold[0][hold[1]]), sc.desc[hold[2]]
        n = H * D + H + P * H + P
        before, _ = F.farm_mlp_loss_grad(ctx, xq, xd, hold[3], hold[4], n)
        losses = F.farm_mlp_train(ctx, 0, rows, pr, po, y, w, epochs=4, batch=2048, lr=2e-3, seed=5)
        after, _ = F.farm_mlp_loss_grad(ctx, xq, xd, hold[3], hold[4], n)
    finally:
        F.farm_destroy(ctx)
    assert losses[-1] < 0.5 * losses[0], losses
    assert after < 0.5 * before, (before, after)


def test_learned_path_recall_and_gain_over_untrained(F):
    """Training lowers the held-out distillation loss by orders of magnitude and
    raises the recall of each row's exact top-16 within its compressed top-64
    (what decides how few candidates the FP32 rescore needs); the learned path
    then meets Recall@10 >= 0.99 against the FP64 oracle."""
    scenes, qb = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    sub = qb.subset(range(96))
    rng = np.random.default_rng(6)
    D, H, P = 1152, 512, 128
    params = init_params(rng, D, H, P)
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        F.farm_mlp_set(ctx, *params)
        rows_eval = np.concatenate([qb.tgt_emb[:200], qb.c_emb[:200]])
        S = F.farm_similarity(ctx, 0, rows_eval, sc.n, F.PREC_FP32)
        true_top = np.argsort(-S, axis=1)[:, :16]

        def cand_recall():
            ed = F.farm_mlp_embed(ctx, sc.desc, P, F.PREC_BF16)
            eq = F.farm_mlp_embed(ctx, rows_eval, P, F.PREC_BF16)
            ctop = np.argsort(-(eq @ ed.T), axis=1)[:, :64]
            return np.mean([len(set(true_top[i]) & set(ctop[i])) / 16.0 for i in range(len(rows_eval))])

        hold = _self_supervised_pairs(F, ctx, sc, 0, 200, 256, 768, seed=4)
        xq, xd = unit(hold[0][hold[1]]), sc.desc[hold[2]]
        n = H * D + H + P * H + P
        loss_u = F.farm_mlp_loss_grad(ctx, xq, xd, hold[3], hold[4], n)[0]
        rec_u = cand_recall()
        rows, pr, po, y, w = _self_supervised_pairs(F, ctx, sc, 0, 1000, 256, 768, seed=7)
        F.farm_mlp_train(ctx, 0, rows, pr, po, y, w, epochs=2, batch=4096, lr=1e-3, seed=8)
        loss_t = F.farm_mlp_loss_grad(ctx, xq, xd, hold[3], hold[4], n)[0]
        rec_t = cand_recall()
        h = F.farm_query_batch(ctx, sub.scene_of_q, sub.tgt_emb, sub.tgt_cls, sub.c_off, sub.c_pred,
                               sub.c_emb, F.PREC_LEARNED)
        trained = F.farm_topk(ctx, h, 10, sub.n_q)
    finally:
        F.farm_destroy(ctx)
    assert loss_t < 0.05 * loss_u, (loss_u, loss_t)
    assert rec_t >= rec_u + 0.01, (rec_u, rec_t)
    ref = oracle.batch(sc, sub, 10)
    hits = sum(len(set(trained["idx"][q].tolist()) & set(ref["idx"][q].tolist())) for q in range(sub.n_q))
    assert hits / (10.0 * sub.n_q) >= 0.99


@pytest.fixture(scope="module")
def site100k():
    return synth.workload("site_n100k_d1152")


@pytest.mark.parametrize("prec", ["learned", "bf16"])
def test_reduced_paths_recall_100k_objects(F, site100k, prec):
    """The learned prefilter's configured workload (and BF16 on it): the
    100,000-object site, all 16,384 queries in one batch -- after the
    self-supervised training the benchmark runs, for the learned path --
    with Recall@10 >= 0.99 against the FP64 oracle on a seeded sample of 64
    queries."""
    import bench
    scenes, qb = site100k
    sc = scenes[0]
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        code = F.PREC_BF16
        if prec == "learned":
            bench.train_prefilter(F, ctx, sc.dim)
            code = F.PREC_LEARNED
        h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb, code)
        out = F.farm_topk(ctx, h, 10, qb.n_q)
    finally:
        F.farm_destroy(ctx)
    qs = np.sort(np.random.default_rng(29).choice(qb.n_q, size=64, replace=False))
    ref = oracle.batch(sc, qb.subset(qs), 10)
    hits = sum(len(set(out["idx"][q].tolist()) & set(ref["idx"][i].tolist())) for i, q in enumerate(qs))
    assert hits / (10.0 * qs.size) >= 0.99, hits / (10.0 * qs.size)
