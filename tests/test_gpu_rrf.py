"""GPU parity of retrieval over several channels (App. D.2 step 3:
reciprocal-rank fusion over four query channels in three embedding spaces),
through the C ABI, against the FP64 oracle with the tie-tolerant checker.

Scenes: the room (200 objects) with two further spaces, a 9,000-object scene
(its target rows take the shared-memory select: fewer 32-object groups than
the channel list length), a 30-object scene (every list holds every object)
and a slice of the 20,000-object site with spaces of 1,024 and 2,048
dimensions.  Queries draw predicates from all fifteen codes (Between pairs included).
"""
import numpy as np
import pytest

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


def _upload(F, ctx, sid, sc, sp):
    F.farm_memory_upload(ctx, sid, sc.desc, sc.cls, sc.box, sc.views)
    for s in range(1, len(sp.desc)):
        F.farm_memory_add_space(ctx, sid, s, sp.desc[s])


def _run(F, ctx, sid, qb, cq, k=10):
    h = F.farm_query_batch_rrf(ctx, sid, cq.channels, cq.tgt, qb.tgt_cls, qb.c_off, qb.c_pred, cq.lm)
    return h, F.farm_topk(ctx, h, k, qb.n_q)


def _case(scene_seed, n, dim, dims, n_q, extent, n_classes=16, distractors=0, m_choices=(0, 1, 2, 3, 4)):
    sc = synth.make_scene(scene_seed, n, dim, extent=extent, n_classes=n_classes, n_views=4,
                          distractor_classes=distractors, distractor_frac=0.3 if distractors else 0.0)
    sp = synth.add_spaces(sc, scene_seed + 50, dims=dims)
    qb = synth.make_queries(scene_seed + 60, sc, n_q, m_choices=m_choices, preds=list(range(15)),
                            distractor_classes=distractors, distractor_target_frac=0.5 if distractors else 0.0)
    cq = synth.channel_queries(scene_seed + 70, sc, sp, qb)
    return sc, sp, qb, cq


@pytest.mark.parametrize("case", ["room", "mid9000", "tiny30"])
def test_fused_parity(F, ctx, case):
    if case == "room":
        sc, sp, qb, cq = _case(700, 200, 512, (256, 384), 96, (10.0, 10.0, 3.0))
    elif case == "mid9000":
        sc, sp, qb, cq = _case(701, 9000, 256, (128, 192), 48, (80.0, 80.0, 8.0), n_classes=180, distractors=9)
    else:
        sc, sp, qb, cq = _case(702, 30, 64, (32, 96), 40, (5.0, 5.0, 3.0), n_classes=4)
    _upload(F, ctx, 70, sc, sp)
    h, out = _run(F, ctx, 70, qb, cq)
    rep = parity.check_topk_mc(sc, sp.desc, qb, cq, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()
    if case != "mid9000":     # (300-object look-alike classes there: every top lies within the tie tolerance)
        assert rep.n_exact > 0


def test_fused_site_slice(F, ctx):
    scenes, _ = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    sp = synth.add_spaces(sc, 801, dims=(1024, 2048))
    qb = synth.make_queries(802, sc, 96, m_choices=(1, 2, 3, 4), distractor_classes=20,
                            distractor_target_frac=0.5, preds=list(range(15)))
    cq = synth.channel_queries(803, sc, sp, qb)
    _upload(F, ctx, 71, sc, sp)
    h, out = _run(F, ctx, 71, qb, cq)
    rep = parity.check_topk_mc(sc, sp.desc, qb, cq, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()


def test_one_channel_matches_the_single_channel_path(F, ctx):
    sc, sp, qb, cq = _case(703, 200, 512, (256, 384), 64, (10.0, 10.0, 3.0))
    _upload(F, ctx, 72, sc, sp)
    h = F.farm_query_batch_rrf(ctx, 72, [(0, 1.0)], [qb.tgt_emb], qb.tgt_cls, qb.c_off, qb.c_pred, [qb.c_emb])
    a = F.farm_topk(ctx, h, 10, qb.n_q)
    h = F.farm_query_batch(ctx, np.full(qb.n_q, 72, np.int32), qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred,
                           qb.c_emb, F.PREC_FP32)
    b = F.farm_topk(ctx, h, 10, qb.n_q)
    # the same ranks and relations; s_sem = cf * (1 / (mu + r)) here against
    # cf / (mu + r) there, one rounding apart
    assert np.allclose(a["score"], b["score"], rtol=1e-6, atol=0)
    same = np.all(a["idx"] == b["idx"], axis=1)
    assert same.mean() > 0.95
    # where an order differs, the scores tie within that rounding
    for q in np.flatnonzero(~same):
        assert np.allclose(np.sort(a["score"][q]), np.sort(b["score"][q]), rtol=1e-6)


def test_fused_invalid_calls(F, ctx):
    sc, sp, qb, cq = _case(704, 200, 512, (256, 384), 8, (10.0, 10.0, 3.0))
    _upload(F, ctx, 73, sc, sp)
    with pytest.raises(F.FarmError):       # space 3 was never uploaded
        F.farm_query_batch_rrf(ctx, 73, [(3, 1.0)], [cq.tgt[0]], qb.tgt_cls, qb.c_off, qb.c_pred, [cq.lm[0]])
    with pytest.raises(F.FarmError):       # non-positive weight
        F.farm_query_batch_rrf(ctx, 73, [(0, 0.0)], [qb.tgt_emb], qb.tgt_cls, qb.c_off, qb.c_pred, [qb.c_emb])
    # FARM_GRAPH is not supported for fused batches (the binding never sets
    # it: call the C entry point directly)
    import ctypes
    h = ctypes.c_uint64()
    ch = (F.FarmChannel * 1)(F.FarmChannel(0, 1.0))
    te = np.ascontiguousarray(qb.tgt_emb)
    st = F.farm._lib.farm_query_batch_rrf(ctx, 73, qb.n_q, 1, ch, te.ctypes.data_as(ctypes.c_void_p),
                                         qb.tgt_cls.ctypes.data_as(ctypes.c_void_p),
                                         qb.c_off.ctypes.data_as(ctypes.c_void_p),
                                         qb.c_pred.ctypes.data_as(ctypes.c_void_p),
                                         qb.c_emb.ctypes.data_as(ctypes.c_void_p), F.GRAPH, ctypes.byref(h))
    assert st == 1 and "FARM_GRAPH" in F.farm_last_error(ctx)
    with pytest.raises(F.FarmError):       # a zero descriptor row
        F.farm_memory_add_space(ctx, 73, 2, np.zeros((sc.n, 8), np.float32))
    # the context stays usable
    h, out = _run(F, ctx, 73, qb, cq)
    rep = parity.check_topk_mc(sc, sp.desc, qb, cq, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()
