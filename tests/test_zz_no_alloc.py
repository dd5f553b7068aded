"""farm_rank_rows_noalloc: the ranked object lists of embedding rows, computed
without allocating device memory.

The entry point serves callers that cannot allocate GPU memory while they
answer queries: a robot process whose GPU memory budget is fixed at start-up
(the mapping pipeline and model workers own the rest), or a real-time loop
that must not call cudaMalloc/cudaFree because those calls may synchronise the
device and take unbounded time.  It keeps every intermediate array in one
static device array whose address farm_create resolves.

Through the C ABI, two calls in a row (target rows, then landmark rows, which
reuse the same static array) must return
  * the same ranked lists as the allocating path (farm_query_batch +
    farm_candidates), identical wherever the order is decided by more than
    the cosine tie tolerance of the other parity tests (2e-5);
  * the oracle's ranking: every listed cosine within 1e-5 of the FP64 cosine,
    and the list equal to the oracle's (cosine desc, index asc) order except
    between objects whose FP64 cosines lie within the tie tolerance;
and no call may change the device's free memory or torch's allocations: after
a warm-up call, and on a fresh context whose workspace never grew.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TIE = 2e-5


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
def scene_and_queries():
    sc = synth.make_scene(21, 5000, 256, extent=(40.0, 40.0, 6.0), n_classes=40, n_views=4,
                          distractor_classes=4, distractor_frac=0.3)
    qb = synth.make_queries(22, sc, 48, m_choices=(1, 2, 3), distractor_classes=4,
                            distractor_target_frac=0.5)
    return sc, qb


def _same_ranking(got_idx, ref_idx, sim_rows):
    """Equal lists, or differences only between objects whose cosines are within TIE."""
    for row in range(ref_idx.shape[0]):
        a, b = got_idx[row], ref_idx[row]
        if np.array_equal(a, b):
            continue
        diff = np.flatnonzero(a != b)
        ca = sim_rows[row][a[diff]]
        cb = sim_rows[row][b[diff]]
        assert np.all(np.abs(ca - cb) <= TIE), (row, a[diff][:5], b[diff][:5])
        # the set may differ only at the boundary, by tied objects
        assert abs(sim_rows[row][a[-1]] - sim_rows[row][b[-1]]) <= TIE


def _oracle_lists(sc, emb, r):
    """The oracle's FP64 cosines of each row and its r best objects (cosine desc, index asc)."""
    import oracle
    oracle.build()
    cos = np.stack([oracle.cosines(sc, u) for u in emb])
    idx = np.stack([np.lexsort((np.arange(sc.n), -c))[:r] for c in cos])
    return cos, idx


def _mem_state():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()


@pytest.mark.parametrize("prec_name", ["fp32", "fp32_simt"])
def test_rank_rows_noalloc_matches_batch_path_and_oracle_twice(F, scene_and_queries, prec_name):
    import torch
    prec = {"fp32": F.PREC_FP32, "fp32_simt": F.PREC_FP32_SIMT}[prec_name]
    sc, qb = scene_and_queries
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        h = F.farm_query_batch(ctx, qb.scene_of_q, qb.tgt_emb, qb.tgt_cls, qb.c_off, qb.c_pred,
                               qb.c_emb, prec)
        ref_t, ref_l = F.farm_candidates(ctx, h, qb.n_q, qb.n_c)
        r_t, r_l = ref_t.shape[1], ref_l.shape[1]
        sim_t = F.farm_similarity(ctx, 0, qb.tgt_emb, sc.n, prec)
        sim_l = F.farm_similarity(ctx, 0, qb.c_emb, sc.n, prec)

        emb = torch.from_numpy(qb.tgt_emb).cuda()
        idx1 = torch.full((qb.n_q, r_t), -7, dtype=torch.int32, device="cuda")
        cos1 = torch.zeros((qb.n_q, r_t), dtype=torch.float32, device="cuda")
        emb2 = torch.from_numpy(qb.c_emb).cuda()
        idx2 = torch.full((qb.n_c, r_l), -7, dtype=torch.int32, device="cuda")
        cos2 = torch.zeros((qb.n_c, r_l), dtype=torch.float32, device="cuda")
        # warm-up call, then the measured pair of calls
        F.farm_rank_rows_noalloc(ctx, 0, emb, r_t, prec, idx1, cos1)
        before = _mem_state()
        # call 1: target rows, R candidates each
        F.farm_rank_rows_noalloc(ctx, 0, emb, r_t, prec, idx1, cos1)
        # call 2 (reuses the same static array): landmark rows, K_a candidates each
        F.farm_rank_rows_noalloc(ctx, 0, emb2, r_l, prec, idx2, cos2)
        F.farm_sync(ctx)
        assert _mem_state() == before

        got1, c1 = idx1.cpu().numpy(), cos1.cpu().numpy()
        got2, c2 = idx2.cpu().numpy(), cos2.cpu().numpy()
        # against the allocating path
        _same_ranking(got1, ref_t, sim_t)
        _same_ranking(got2, ref_l, sim_l)
        np.testing.assert_allclose(c1, np.take_along_axis(sim_t, got1, axis=1), rtol=0, atol=1e-5)
        np.testing.assert_allclose(c2, np.take_along_axis(sim_l, got2, axis=1), rtol=0, atol=1e-5)
        assert np.all(np.diff(c1, axis=1) <= 0) and np.all(np.diff(c2, axis=1) <= 0)
        # against the oracle
        for emb_h, got, cg, r in ((qb.tgt_emb, got1, c1, r_t), (qb.c_emb, got2, c2, r_l)):
            ocos, oidx = _oracle_lists(sc, emb_h, r)
            np.testing.assert_allclose(cg, np.take_along_axis(ocos, got, axis=1), rtol=0, atol=1e-5)
            _same_ranking(got, oidx, ocos)
    finally:
        F.farm_destroy(ctx)


def test_rank_rows_noalloc_takes_no_memory_on_a_fresh_context(F, scene_and_queries):
    """The first call on a context whose workspace never grew allocates nothing either."""
    import torch
    sc, qb = scene_and_queries
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        emb = torch.from_numpy(qb.tgt_emb).cuda()
        idx = torch.full((qb.n_q, 16), -7, dtype=torch.int32, device="cuda")
        before = _mem_state()
        for prec in (F.PREC_FP32, F.PREC_FP32_SIMT):
            F.farm_rank_rows_noalloc(ctx, 0, emb, 16, prec, idx)
        F.farm_sync(ctx)
        assert _mem_state() == before
        ocos, oidx = _oracle_lists(sc, qb.tgt_emb, 16)
        _same_ranking(idx.cpu().numpy(), oidx, ocos)
    finally:
        F.farm_destroy(ctx)


def test_rank_rows_noalloc_rejects_oversize(F):
    import torch
    sc = synth.make_scene(23, 20000, 1152, extent=(120.0, 120.0, 10.0), n_classes=50, n_views=2)
    ctx = F.farm_create(0)
    try:
        F.farm_memory_upload(ctx, 0, sc.desc, sc.cls, sc.box, sc.views)
        rows = 1024    # 1024 x 20,000 x 4 B = 82 MB of similarity block > 32 MiB
        emb = torch.randn((rows, 1152), device="cuda")
        out = torch.empty((rows, 10), dtype=torch.int32, device="cuda")
        with pytest.raises(F.FarmError) as e:
            F.farm_rank_rows_noalloc(ctx, 0, emb, 10, F.PREC_FP32, out)
        assert e.value.status == 1 and "FARM_NOALLOC_SCRATCH_BYTES" in str(e.value)
    finally:
        F.farm_destroy(ctx)
