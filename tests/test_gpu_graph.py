"""GPU: batches run as CUDA graphs (FARM_GRAPH) give the results of the same
batches run directly, including on replays of a cached graph with new query
contents, after a change of batch shape, and after a scene is re-uploaded."""
import numpy as np
import pytest

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


def _run(F, ctx, qb, prec, graph):
    h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb,
                           prec, graph=graph)
    return F.farm_topk(ctx, h, 10, qb.n_q), F.farm_candidates(ctx, h, qb.n_q, qb.n_c)


def _same(a, b):
    (oa, (ta, la)), (ob, (tb, lb)) = a, b
    for key in ("idx", "score", "pred", "anchor"):
        np.testing.assert_array_equal(oa[key], ob[key], err_msg=key)
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_array_equal(la, lb)


@pytest.fixture(scope="module")
def world(F):
    ctx = F.farm_create(0)
    scenes = {}
    parts = []
    for sid, n in [(50, 3000), (51, 700), (52, 26000)]:
        sc = synth.make_scene(sid, n, 128, extent=(30.0, 30.0, 4.0), n_classes=12, n_views=4)
        F.farm_memory_upload(ctx, sid, sc.desc, sc.cls, sc.box, sc.views)
        scenes[sid] = sc
        parts.append(synth.make_queries(sid + 900, sc, 40, m_choices=(0, 1, 2, 3, 4), scene_id=sid))
    qb = synth.scenes.concat_batches(parts)
    qb = qb.subset(np.random.default_rng(7).permutation(qb.n_q))
    yield ctx, scenes, qb
    F.farm_destroy(ctx)


def _variant(qb, seed):
    """Same shape (scene order, per-scene query and constraint counts), new contents."""
    rng = np.random.default_rng(seed)
    v = qb.subset(np.arange(qb.n_q))
    v.tgt_emb = (v.tgt_emb + 0.05 * rng.standard_normal(v.tgt_emb.shape)).astype(np.float32)
    v.c_emb = (v.c_emb + 0.05 * rng.standard_normal(v.c_emb.shape)).astype(np.float32)
    v.c_pred = rng.integers(0, 5, size=v.c_pred.shape).astype(np.int32)
    v.tgt_cls = np.where(rng.random(v.n_q) < 0.3, -1, v.tgt_cls).astype(np.int32)
    return v


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_graph_matches_direct_and_replays(F, world, prec):
    ctx, scenes, qb = world
    code = {"fp32": F.PREC_FP32, "bf16": F.PREC_BF16, "fp8": F.PREC_FP8}[prec]
    _same(_run(F, ctx, qb, code, graph=True), _run(F, ctx, qb, code, graph=False))
    # replays of the cached graph with new contents of the same shape
    for seed in (1, 2):
        v = _variant(qb, seed)
        _same(_run(F, ctx, v, code, graph=True), _run(F, ctx, v, code, graph=False))


def test_graph_new_shape_and_reupload(F, world):
    ctx, scenes, qb = world
    # another shape: a subset of the queries
    sub = qb.subset(np.arange(0, qb.n_q, 3))
    _same(_run(F, ctx, sub, F.PREC_FP32, graph=True), _run(F, ctx, sub, F.PREC_FP32, graph=False))
    _same(_run(F, ctx, qb, F.PREC_FP32, graph=True), _run(F, ctx, qb, F.PREC_FP32, graph=False))
    # re-upload scene 51 with different descriptors: cached graphs must not be replayed
    sc = scenes[51]
    rng = np.random.default_rng(3)
    desc = (sc.desc + 0.2 * rng.standard_normal(sc.desc.shape)).astype(np.float32)
    F.farm_memory_upload(ctx, 51, desc, sc.cls, sc.box, sc.views)
    try:
        _same(_run(F, ctx, qb, F.PREC_FP32, graph=True), _run(F, ctx, qb, F.PREC_FP32, graph=False))
    finally:
        F.farm_memory_upload(ctx, 51, sc.desc, sc.cls, sc.box, sc.views)


def test_graph_counts_the_same_launches(F, world):
    ctx, scenes, qb = world
    _run(F, ctx, qb, F.PREC_FP32, graph=True)      # captured (or cached) before counting
    F.farm_stage_times(ctx, reset=True)
    h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb,
                           F.PREC_FP32, graph=False)
    _, eager = F.farm_stage_times(ctx, reset=True)
    h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb,
                           F.PREC_FP32, graph=True)
    _, replay = F.farm_stage_times(ctx, reset=True)
    F.farm_sync(ctx)
    assert eager == replay and eager > 0


def test_graph_with_device_inputs(F, world):
    """Device embeddings are read in place: reusing the same buffers replays
    the graph with their current contents; other buffers capture anew."""
    import torch
    ctx, scenes, qb = world
    d_tgt = torch.from_numpy(qb.tgt_emb).cuda()
    d_cemb = torch.from_numpy(qb.c_emb).cuda()

    def dev_run(t, c, graph):
        h = F.farm_query_batch(ctx, qb.scene_of_q, t, qb.tgt_cls, qb.c_off, qb.c_pred, c, F.PREC_FP32,
                               graph=graph)
        return F.farm_topk(ctx, h, 10, qb.n_q), F.farm_candidates(ctx, h, qb.n_q, qb.n_c)

    _same(dev_run(d_tgt, d_cemb, True), _run(F, ctx, qb, F.PREC_FP32, graph=False))
    v = _variant(qb, 11)
    d_tgt.copy_(torch.from_numpy(v.tgt_emb))            # same buffers, new contents
    d_cemb.copy_(torch.from_numpy(v.c_emb))
    torch.cuda.synchronize()
    v.c_pred = qb.c_pred.copy()
    v.tgt_cls = qb.tgt_cls.copy()
    _same(dev_run(d_tgt, d_cemb, True), _run(F, ctx, v, F.PREC_FP32, graph=False))
    d_tgt2, d_cemb2 = d_tgt.clone(), d_cemb.clone()      # other buffers
    _same(dev_run(d_tgt2, d_cemb2, True), _run(F, ctx, v, F.PREC_FP32, graph=False))


@pytest.mark.parametrize("graph", [False, True])
def test_pipelined_host_batches_with_async_topk(F, world, graph):
    """Host embeddings travel on the copy stream into alternating slots and
    FARM_ASYNC leaves the TopK copies enqueued: three batches of new contents
    issued back to back, one farm_sync at the end, must give each batch's
    synchronous result (pinned outputs, one set per batch)."""
    import torch
    ctx, scenes, qb = world
    batches = [_variant(qb, seed) for seed in (21, 22, 23)]
    ref = [_run(F, ctx, v, F.PREC_FP32, graph=False)[0] for v in batches]

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype).pin_memory().numpy()

    outs = []
    for v in batches:
        o = dict(idx=pinned((v.n_q, 10), torch.int32), score=pinned((v.n_q, 10), torch.float32),
                 pred=pinned((v.n_q, 10, 4), torch.float32), anchor=pinned((v.n_q, 10, 4), torch.int32))
        h = F.farm_query_batch(ctx, v.scene_of_q, v.tgt_emb, v.tgt_cls, v.c_off, v.c_pred, v.c_emb, F.PREC_FP32,
                               graph=graph)
        F.farm_topk(ctx, h, 10, v.n_q, o["idx"], o["score"], o["pred"], o["anchor"], asynchronous=True)
        outs.append(o)
    F.farm_sync(ctx)
    for o, r in zip(outs, ref):
        for key in ("idx", "score", "pred", "anchor"):
            np.testing.assert_array_equal(o[key], r[key], err_msg=key)


def _embeddings_only(qb, seed):
    """New embeddings, the same query graphs (scenes, classes, constraints)."""
    rng = np.random.default_rng(seed)
    v = qb.subset(np.arange(qb.n_q))
    v.tgt_emb = (v.tgt_emb + 0.05 * rng.standard_normal(v.tgt_emb.shape)).astype(np.float32)
    v.c_emb = (v.c_emb + 0.05 * rng.standard_normal(v.c_emb.shape)).astype(np.float32)
    return v


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_graph_replay_of_the_same_query_graphs(F, world, prec):
    """Back-to-back graph batches with the same query graphs are replayed
    without planning (host rows still copied into alternating slots): each
    must give its own direct result; an in-place change of a predicate or a
    class in the caller's arrays, or a batch of another shape in between, must
    be planned again."""
    import torch
    ctx, scenes, qb = world
    code = {"fp32": F.PREC_FP32, "bf16": F.PREC_BF16}[prec]
    batches = [_embeddings_only(qb, seed) for seed in (31, 32, 33, 34, 35)]
    ref = [_run(F, ctx, v, code, graph=False)[0] for v in batches]

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype).pin_memory().numpy()

    outs = []
    for v in batches:
        o = dict(idx=pinned((v.n_q, 10), torch.int32), score=pinned((v.n_q, 10), torch.float32),
                 pred=pinned((v.n_q, 10, 4), torch.float32), anchor=pinned((v.n_q, 10, 4), torch.int32))
        h = F.farm_query_batch(ctx, v.scene_of_q, v.tgt_emb, v.tgt_cls, v.c_off, v.c_pred, v.c_emb, code,
                               graph=True)
        F.farm_topk(ctx, h, 10, v.n_q, o["idx"], o["score"], o["pred"], o["anchor"], asynchronous=True)
        outs.append(o)
    F.farm_sync(ctx)
    for o, r in zip(outs, ref):
        for key in ("idx", "score", "pred", "anchor"):
            np.testing.assert_array_equal(o[key], r[key], err_msg=key)
    # the caller's arrays changed in place after a replayable batch
    v = batches[-1]
    _run(F, ctx, v, code, graph=True)
    _run(F, ctx, v, code, graph=True)
    first = int(np.flatnonzero(np.diff(v.c_off) > 0)[0])
    v.c_pred[v.c_off[first]] = (v.c_pred[v.c_off[first]] + 1) % 5
    got = _run(F, ctx, v, code, graph=True)
    _same(got, _run(F, ctx, v, code, graph=False))
    _run(F, ctx, v, code, graph=True)
    _run(F, ctx, v, code, graph=True)
    v.tgt_cls[1] = -1 if v.tgt_cls[1] >= 0 else 0
    got = _run(F, ctx, v, code, graph=True)
    _same(got, _run(F, ctx, v, code, graph=False))
    # another shape in between, then the first again (its staging rewritten)
    sub = v.subset(np.arange(0, v.n_q, 2))
    _run(F, ctx, v, code, graph=True)
    _run(F, ctx, v, code, graph=True)
    _same(_run(F, ctx, sub, code, graph=True), _run(F, ctx, sub, code, graph=False))
    _run(F, ctx, sub, code, graph=True)
    got = _run(F, ctx, v, code, graph=True)
    _same(got, _run(F, ctx, v, code, graph=False))
