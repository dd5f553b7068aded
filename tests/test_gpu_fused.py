"""GPU: the fused rank selection against the unfused path and the oracle.

The fused selection stores only a sample of each similarity row (every s-th
tile of 256 objects), ranks it, and lets the similarity kernel keep only the
entries of the other tiles that reach the sample's R-th value; the row's list
is then merged from the sample's list and the kept entries.  FARM_FUSED fuses
every scene of a batch, FARM_UNFUSED none (the whole block is written and
selected from), and by default the FP32 path fuses the scenes whose sample
holds at least 16 times the target list, so that one batch mixes both
selections.  All see the same
tensor-core values, so their lists -- and everything after them -- must be
bitwise equal, in every precision, graph-captured or not, over scenes of one
tile, a ragged last sample tile, several sample tiles and rows longer than
the shared-memory select.  A scene whose sample tiles hold a class the queries
never ask for overflows the kept-entry buffers on purpose, and one whose
queried class sits in the sample tiles makes the optimistic threshold fall
short on purpose: those rows are recomputed exactly and the result must
still match the oracle.  The learned path's two-pass selection (no sample;
every tile's group maxima) must equal its unfused selection bitwise.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import parity
import synth

pytestmark = pytest.mark.gpu

DIM = 256
# sampling stride of each fused path at the default parameters (tiles of 256
# objects): lists of up to 128 (FP32) 8, up to 256 (BF16) 4
STRIDE = {"fp32": 8, "bf16": 4}


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2606_15476_gb300 as F
    return F


def _code(F, prec):
    return {"fp32": F.PREC_FP32, "bf16": F.PREC_BF16, "fp8": F.PREC_FP8, "learned": F.PREC_LEARNED}[prec]


def _run(F, ctx, qb, code, fused, graph=False):
    h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred, qb.c_emb, code,
                           graph=graph, fused=fused)
    return F.farm_topk(ctx, h, 10, qb.n_q), F.farm_candidates(ctx, h, qb.n_q, qb.n_c)


def _same(a, b, qb=None, qs=None):
    """Bitwise equal results (of the queries qs of batch qb, default all)."""
    if qs is None:
        qs = np.arange(a[0]["idx"].shape[0])
        cs = np.arange(a[1][1].shape[0])
    else:
        cs = np.concatenate([np.arange(qb.c_off[q], qb.c_off[q + 1]) for q in qs]).astype(np.int64)
    for key in ("idx", "score", "pred", "anchor"):
        np.testing.assert_array_equal(a[0][key][qs], b[0][key][qs], err_msg=key)
    np.testing.assert_array_equal(a[1][0][qs], b[1][0][qs])
    np.testing.assert_array_equal(a[1][1][cs], b[1][1][cs])


@pytest.fixture(scope="module")
def world(F):
    ctx = F.farm_create(0)
    scenes, parts = {}, []
    # one tile; a ragged last sample tile; several sample tiles; rows longer
    # than the shared-memory select's 24,576 entries
    for sid, n in [(60, 200), (61, 2100), (62, 9000), (63, 20000), (64, 30001)]:
        sc = synth.make_scene(sid, n, DIM, extent=(40.0, 40.0, 5.0), n_classes=max(8, n // 50), n_views=4,
                              distractor_classes=4, distractor_frac=0.3)
        F.farm_memory_upload(ctx, sid, sc.desc, sc.cls, sc.box, sc.views)
        scenes[sid] = sc
        parts.append(synth.make_queries(sid + 500, sc, 40, m_choices=(0, 1, 2, 3, 4), scene_id=sid,
                                        distractor_classes=4, distractor_target_frac=0.5))
    qb = synth.scenes.concat_batches(parts)
    qb = qb.subset(np.random.default_rng(8).permutation(qb.n_q))
    rng = np.random.default_rng(9)
    H, P = 128, 64
    F.farm_mlp_set(ctx, (rng.standard_normal((H, DIM)) / math.sqrt(DIM)).astype(np.float32),
                   (0.05 * rng.standard_normal(H)).astype(np.float32),
                   (rng.standard_normal((P, H)) / math.sqrt(H)).astype(np.float32),
                   (0.05 * rng.standard_normal(P)).astype(np.float32))
    yield ctx, scenes, qb
    F.farm_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8", "learned"])
def test_fused_equals_unfused(F, world, prec):
    """(FP8 and learned batches are never fused -- E4M3 ties many entries at
    a threshold, and lists of 512 crowd the buffer -- so for them this
    compares the default with the explicit flag.  An unfused BF16 batch runs
    its scenes of fewer than 16,384 objects FP32-accurate, whose lists may
    order near-ties differently from the BF16 stage's FP32 rescore: for BF16
    the larger scenes' queries are compared.)"""
    ctx, scenes, qb = world
    code = _code(F, prec)
    F.farm_select_fallbacks(ctx, reset=True)
    fused = _run(F, ctx, qb, code, True)
    assert F.farm_select_fallbacks(ctx) == 0
    if prec == "bf16":
        qs = np.flatnonzero([scenes[int(s)].n >= 16384 for s in qb.scene_of_q])
        assert qs.size >= 40
        _same(fused, _run(F, ctx, qb, code, False), qb, qs)
    else:
        _same(fused, _run(F, ctx, qb, code, False))


@pytest.mark.parametrize("graph", [False, True])
def test_default_mixes_fused_and_unfused_scenes_bitwise(F, world, graph):
    """The batch's scenes of 200 to 9,000 objects take the unfused selection,
    those of 20,000 and 30,001 the fused one, in the same launches."""
    ctx, scenes, qb = world
    F.farm_select_fallbacks(ctx, reset=True)
    mixed = _run(F, ctx, qb, F.PREC_FP32, None, graph=graph)
    assert F.farm_select_fallbacks(ctx) == 0
    _same(mixed, _run(F, ctx, qb, F.PREC_FP32, False))
    _same(mixed, _run(F, ctx, qb, F.PREC_FP32, True))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fused_graph_replays_bitwise(F, world, prec):
    ctx, scenes, qb = world
    code = _code(F, prec)
    direct = _run(F, ctx, qb, code, True)
    _same(_run(F, ctx, qb, code, True, graph=True), direct)
    _same(_run(F, ctx, qb, code, True, graph=True), direct)     # a replay


def _sample_class_scene(seed, n, fs):
    """Objects of the sample tiles (every fs-th tile of 256) in class 0, all
    others in class 1: a class-1 row's sample ranks only class-0 objects, so
    its threshold lets every class-1 object through."""
    base = synth.make_scene(seed, n, DIM, extent=(30.0, 30.0, 4.0), n_classes=2, n_views=4)
    cls = np.where((np.arange(n) // 256) % fs == 0, 0, 1).astype(np.int32)
    rng = np.random.default_rng(seed + 1)
    desc = base.centroids[cls] + base.noise_sigma * rng.standard_normal((n, DIM))
    desc = (desc / np.linalg.norm(desc, axis=1, keepdims=True)).astype(np.float32)
    return dataclasses.replace(base, desc=desc, cls=cls)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_overflowing_rows_are_recomputed_exactly(F, prec):
    fs = STRIDE[prec]
    sc = _sample_class_scene(71, 4096, fs)
    qb = synth.make_queries(72, sc, 48, m_choices=(1, 2))
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        F.farm_select_fallbacks(ctx, reset=True)
        out, (t, l) = _run(F, ctx, qb, _code(F, prec), True)
        recomputed = F.farm_select_fallbacks(ctx)
    finally:
        F.farm_destroy(ctx)
    # most rows ask for class 1 (all objects but every fs-th tile)
    assert recomputed >= (qb.n_q + qb.n_c) // 2, recomputed
    if prec == "fp32":
        rep = parity.check_topk(sc, qb, 10, out["idx"], out["score"], out["pred"], out["anchor"])
        assert rep.ok(), rep.summary()
        fails = parity.check_candidates(sc, qb, t, l)
        assert not fails, fails[:3]
    else:
        ref = oracle.batch(sc, qb, 10)
        hits = sum(len(set(out["idx"][q].tolist()) & set(ref["idx"][q].tolist())) for q in range(qb.n_q))
        assert hits / (10.0 * qb.n_q) >= 0.99


@pytest.fixture(scope="module")
def big(F):
    """One scene of 70,000 objects (2,188 groups of 32 per row, at least four
    times the learned path's target list of 512: the two-pass selection), one
    of 40,000 (1,250 groups) and one of 9,000 (the unfused learned selection)
    in the same batches."""
    ctx = F.farm_create(0)
    scenes, parts = {}, []
    for sid, n in [(80, 70000), (81, 9000), (82, 40000)]:
        sc = synth.make_scene(sid, n, DIM, extent=(90.0, 90.0, 8.0), n_classes=max(8, n // 50), n_views=4,
                              distractor_classes=4, distractor_frac=0.3)
        F.farm_memory_upload(ctx, sid, sc.desc, sc.cls, sc.box, sc.views)
        scenes[sid] = sc
        parts.append(synth.make_queries(sid + 500, sc, 48, m_choices=(0, 1, 2, 3, 4), scene_id=sid,
                                        distractor_classes=4, distractor_target_frac=0.5))
    qb = synth.scenes.concat_batches(parts)
    qb = qb.subset(np.random.default_rng(18).permutation(qb.n_q))
    rng = np.random.default_rng(19)
    H, P = 128, 64
    F.farm_mlp_set(ctx, (rng.standard_normal((H, DIM)) / math.sqrt(DIM)).astype(np.float32),
                   (0.05 * rng.standard_normal(H)).astype(np.float32),
                   (rng.standard_normal((P, H)) / math.sqrt(H)).astype(np.float32),
                   (0.05 * rng.standard_normal(P)).astype(np.float32))
    yield ctx, scenes, qb
    F.farm_destroy(ctx)


@pytest.mark.parametrize("graph", [False, True])
def test_learned_two_pass_equals_unfused(F, big, graph):
    """The learned path's two-pass selection (every tile's group maxima, the
    threshold from them, every tile keeping the entries that reach it) sees
    the same compressed-space values as the unfused path, which stores them
    all: the candidate lists, the rescored rank lists and the results must be
    bitwise equal, with no row recomputed by the fallback."""
    ctx, scenes, qb = big
    code = _code(F, "learned")
    F.farm_select_fallbacks(ctx, reset=True)
    two = _run(F, ctx, qb, code, None, graph=graph)
    if graph:
        two = _run(F, ctx, qb, code, None, graph=graph)    # (the first batch of a class tunes the tiles)
    assert F.farm_select_fallbacks(ctx) == 0
    _same(two, _run(F, ctx, qb, code, False))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_long_rows_unfused_equal_fused(F, big, prec):
    """Unfused, rows of 1,250 and 2,188 group maxima are keyed by the maxima
    of 2 and 4 consecutive groups in the warp-level select (the groups of the
    keys that reach the R-th largest key are gathered); the lists and results
    must equal the fused selection's bitwise.  (BF16: the queries of the
    scenes of at least 16,384 objects, which run the BF16 stage.)"""
    ctx, scenes, qb = big
    code = _code(F, prec)
    F.farm_select_fallbacks(ctx, reset=True)
    fused = _run(F, ctx, qb, code, True)
    assert F.farm_select_fallbacks(ctx) == 0
    unfused = _run(F, ctx, qb, code, False)
    if prec == "bf16":
        qs = np.flatnonzero([scenes[int(s)].n >= 16384 for s in qb.scene_of_q])
        assert qs.size >= 90
        _same(fused, unfused, qb, qs)
    else:
        _same(fused, unfused)


def test_optimistic_threshold_that_falls_short_is_recomputed(F):
    """The fused selection sets a target row's threshold at the sample's k-th
    entry (k < R), trusting that the rest of the row holds R - k more; a scene
    whose queried class sits almost entirely in the sample tiles breaks that
    trust on purpose: fuse_final must find fewer than R words reaching the
    threshold, leave every such row to the exact fallback, and the results
    must still match the oracle."""
    n, fs = 4096, STRIDE["fp32"]
    base = synth.make_scene(91, n, DIM, extent=(30.0, 30.0, 4.0), n_classes=2, n_views=4)
    rng = np.random.default_rng(92)
    in_sample = (np.arange(n) // 256) % fs == 0
    cls = np.where(in_sample, 0, 1)
    cls[rng.choice(np.flatnonzero(~in_sample), 40, replace=False)] = 0      # a few of the class elsewhere
    cls = cls.astype(np.int32)
    desc = base.centroids[cls] + base.noise_sigma * rng.standard_normal((n, DIM))
    desc = (desc / np.linalg.norm(desc, axis=1, keepdims=True)).astype(np.float32)
    sc = dataclasses.replace(base, desc=desc, cls=cls)
    qb = synth.make_queries(93, sc, 32, m_choices=(1, 2))
    t = base.centroids[0] + base.noise_sigma * rng.standard_normal((qb.n_q, DIM))
    qb.tgt_emb = (t / np.linalg.norm(t, axis=1, keepdims=True)).astype(np.float32)
    qb.tgt_cls = np.zeros(qb.n_q, np.int32)
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        F.farm_select_fallbacks(ctx, reset=True)
        out, (t, l) = _run(F, ctx, qb, F.PREC_FP32, True)
        recomputed = F.farm_select_fallbacks(ctx)
    finally:
        F.farm_destroy(ctx)
    assert recomputed >= qb.n_q, recomputed          # every target row fell short
    rep = parity.check_topk(sc, qb, 10, out["idx"], out["score"], out["pred"], out["anchor"])
    assert rep.ok(), rep.summary()
    fails = parity.check_candidates(sc, qb, t, l)
    assert not fails, fails[:3]
