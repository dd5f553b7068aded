"""GPU: the reduced-precision paths (BF16 or FP8-E4M3, then FP32 rescore)
against the FP64 oracle.

The reduced-precision stage only chooses which candidates get re-scored; every
kept rank is decided by exact FP32 cosines, so results must match the oracle
(same checker as the FP32 path) wherever the FP32 top-R of a row lies inside
its reduced-precision top-C, and Recall@10 against the oracle's top 10 must be
at least 0.99.
"""
import numpy as np
import pytest

import oracle
from oracle import parity
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


@pytest.fixture(scope="module")
def ctx(F):
    c = F.farm_create(0)
    yield c
    F.farm_destroy(c)


def _run(F, ctx, qb, prec, k=10):
    h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred,
                           qb.c_emb, prec)
    return F.farm_topk(ctx, h, k, qb.n_q)


REDUCED = ["bf16", "fp8"]


def code(F, name):
    return {"bf16": F.PREC_BF16, "fp8": F.PREC_FP8}[name]


@pytest.mark.parametrize("prec,bound,typical", [
    # BF16 keeps 8 significant bits per operand: |error| <= (2 * 2^-8 + 2^-16) sum|u_k d_k| <= 2^-7
    ("bf16", 2.0 ** -7, 1e-4),
    # E4M3 keeps 4: |error| <= (2 * 2^-4 + 2^-8) sum|u_k d_k| <= 0.13
    ("fp8", 0.13, 5e-3)])
def test_reduced_stage_cosine_error(F, ctx, prec, bound, typical):
    scenes, qb = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
    rows = np.concatenate([qb.tgt_emb[:16], qb.c_emb[:16]])
    got = F.farm_similarity(ctx, 0, rows, sc.n, code(F, prec))
    errs = np.concatenate([np.abs(got[r] - oracle.cosines(sc, rows[r])) for r in range(rows.shape[0])])
    assert errs.max() <= bound
    assert np.median(errs) < typical


@pytest.mark.parametrize("prec", REDUCED)
def test_reduced_exact_when_every_object_is_rescored(F, ctx, prec):
    scenes, qb = synth.workload("room_n200_d512")   # n = 200 <= the 256 candidates kept
    sc = scenes[0]
    F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
    out = _run(F, ctx, qb, code(F, prec))
    rep = parity.check_topk(sc, qb, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()


# Queries whose result passes the exact parity check: a true top-R object
# missing from the kept candidates shifts later ranks (and so their
# rank-based scores).  FP8's per-element rounding (2^-4) spans many ranks in
# the 300-member look-alike classes, BF16's (2^-8) rarely does.
CLEAN_FLOOR = {"bf16": 0.9, "fp8": 0.5}


@pytest.mark.parametrize("prec", REDUCED)
def test_reduced_recall_at_10_site_scale(F, ctx, prec):
    scenes, qb = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
    sub = qb.subset(range(128))
    out = _run(F, ctx, sub, code(F, prec))
    ref = oracle.batch(sc, sub, 10)
    hits = sum(len(set(out["idx"][q].tolist()) & set(ref["idx"][q].tolist())) for q in range(sub.n_q))
    recall = hits / (10.0 * sub.n_q)
    assert recall >= 0.99, recall
    rep = parity.check_topk(sc, sub, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    bad_queries = len({f.split(":")[0].split()[0] for f in rep.failures})
    assert 1.0 - bad_queries / sub.n_q >= CLEAN_FLOOR[prec], rep.summary()


@pytest.mark.parametrize("prec", REDUCED)
def test_reduced_matches_fp32_path_on_full_batch(F, ctx, prec):
    scenes, qb = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
    a = _run(F, ctx, qb, F.PREC_FP32)
    b = _run(F, ctx, qb, code(F, prec))
    same = np.mean([len(set(a["idx"][q].tolist()) & set(b["idx"][q].tolist())) / 10.0 for q in range(qb.n_q)])
    assert same >= 0.99, same


@pytest.mark.parametrize("prec", REDUCED)
def test_reduced_recall_at_10_16k_queries(F, ctx, prec):
    """The precision workload as configured: 16,384 queries on the 20,000-object
    site in one graph-captured batch; Recall@10 against the FP64 oracle on a
    seeded sample of 192 queries."""
    scenes, qb = synth.workload("site_n20k_d1152_q16k")
    sc = scenes[0]
    F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
    args = (qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb, code(F, prec))
    F.farm_query_batch(ctx, *args)                   # the batch class's first run: the autotuner
    h = F.farm_query_batch(ctx, *args, graph=True)
    out = F.farm_topk(ctx, h, 10, qb.n_q)
    qs = np.sort(np.random.default_rng(23).choice(qb.n_q, size=192, replace=False))
    ref = oracle.batch(sc, qb.subset(qs), 10)
    hits = sum(len(set(out["idx"][q].tolist()) & set(ref["idx"][i].tolist())) for i, q in enumerate(qs))
    recall = hits / (10.0 * qs.size)
    assert recall >= 0.99, recall
