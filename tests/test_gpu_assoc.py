"""GPU parity of the mapping-side association (App. D.1 steps 3-5: Hellinger
neighbour search, union-find correspondence, sufficient-statistics fusion)
through the C ABI against the FP64 oracle.

Detections whose outcome the arithmetic could flip -- a feature cosine
within 1e-5 of tau_f, a Hellinger distance within 1e-5 of the budget, or two
kept distances within 1e-5 of one another -- are counted first; the seeded
cases here have none, so match lists, components and winners must agree
exactly and the fused moments within FP32 rounding.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TAU, HMAX, MM = 0.8, 0.9, 8


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


def _full(c):
    ix = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    m = np.zeros((3, 3))
    for k, (i, j) in enumerate(ix):
        m[i, j] = m[j, i] = c[k]
    return m


def _ambiguous(ent, det, ref, hmax=HMAX):
    """Detections whose match list depends on a decision within 1e-5."""
    ef = ent["feat"].astype(np.float64)
    df = det["feat"].astype(np.float64)
    cos = (df / np.linalg.norm(df, axis=1, keepdims=True)) @ (ef / np.linalg.norm(ef, axis=1, keepdims=True)).T
    amb = set(np.flatnonzero(np.any(np.abs(cos - TAU) < 1e-5, axis=1)).tolist())
    for d in range(df.shape[0]):
        hs = ref["match_h"][d][ref["match_h"][d] >= 0]
        if np.any(np.abs(hs - hmax) < 1e-5) or np.any(np.diff(hs) < 1e-5):
            amb.add(d)
        if ref["match_cnt"][d] > MM:     # the (max_m + 1)-th could tie with the last kept
            amb.add(d)
    return amb


def _check(ent, det, got, ref, hmax=HMAX):
    assert not _ambiguous(ent, det, ref, hmax)
    assert np.array_equal(got["match_cnt"], ref["match_cnt"])
    assert np.array_equal(got["match_idx"], ref["match_idx"])
    kept = ref["match_idx"] >= 0
    assert np.allclose(got["match_h"][kept], ref["match_h"][kept], atol=1e-5)
    assert np.array_equal(got["parent"], ref["parent"])
    assert np.allclose(got["w"], ref["w"], rtol=1e-6, atol=0)
    assert np.allclose(got["mu"], ref["mu"], rtol=0, atol=2e-5)
    assert np.allclose(got["cov"], ref["cov"], rtol=1e-4, atol=1e-7)
    assert np.allclose(got["feat"], ref["feat"], rtol=0, atol=2e-6)


@pytest.mark.parametrize("seed", [11, 12])
def test_room_association(F, ctx, seed):
    scenes, _ = synth.workload("room_n200_d512")
    ent, det = synth.make_association(seed, scenes[0], 256, feat_dim=64, bridge_frac=0.15)
    ref = oracle.associate(ent, det, TAU, HMAX, MM)
    got = F.farm_associate(ctx, ent, det, TAU, HMAX, MM)
    assert np.sum(ref["parent"][:200] != np.arange(200)) > 0      # some entities merge
    assert np.sum(ref["match_cnt"] == 0) > 0                       # and some detections are new
    _check(ent, det, got, ref)


def test_site_association_and_device_pointers(F, ctx):
    import torch
    scenes, _ = synth.workload("site_n20k_d1152")
    ent, det = synth.make_association(13, scenes[0], 512, feat_dim=256, bridge_frac=0.1)
    ref = oracle.associate(ent, det, TAU, HMAX, MM)
    got = F.farm_associate(ctx, ent, det, TAU, HMAX, MM)
    _check(ent, det, got, ref)
    dent = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in ent.items()}
    ddet = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in det.items()}
    gd = F.farm_associate(ctx, dent, ddet, TAU, HMAX, MM)
    F.farm_sync(ctx)          # device outputs are written on the context's stream
    for k in ("match_cnt", "match_idx", "parent"):
        assert np.array_equal(gd[k].cpu().numpy(), got[k])
    assert np.allclose(gd["mu"].cpu().numpy(), got["mu"], atol=2e-5)


def test_association_beyond_shared_memory_labels(F, ctx):
    """Over 51,200 nodes (100,000 entities): the components kernel keeps its
    labels in global memory instead of shared memory.  A looser budget lets
    bridging detections merge entities at this scene's sparser classes."""
    scenes, _ = synth.workload("site_n100k_d1152")
    hmax = 0.97
    ent, det = synth.make_association(15, scenes[0], 256, feat_dim=64, bridge_frac=0.3)
    n = ent["mu"].shape[1]
    assert n + det["mu"].shape[1] > 51200
    ref = oracle.associate(ent, det, TAU, hmax, MM)
    assert np.sum(ref["parent"][:n] != np.arange(n)) > 0      # a component holds two entities
    got = F.farm_associate(ctx, ent, det, TAU, hmax, MM)
    _check(ent, det, got, ref, hmax)


def test_association_invalid_arguments(F, ctx):
    scenes, _ = synth.workload("room_n200_d512")
    ent, det = synth.make_association(14, scenes[0], 16, feat_dim=16)
    with pytest.raises(F.FarmError):
        F.farm_associate(ctx, ent, det, TAU, HMAX, 0)
    with pytest.raises(F.FarmError):
        F.farm_associate(ctx, ent, det, TAU, 1.5, MM)
    bad = dict(ent)
    bad["w"] = -np.ones_like(ent["w"])
    with pytest.raises(F.FarmError):
        F.farm_associate(ctx, bad, det, TAU, HMAX, MM)
    got = F.farm_associate(ctx, ent, det, TAU, HMAX, MM)       # the context stays usable
    assert got["parent"].shape[0] == ent["mu"].shape[1] + det["mu"].shape[1]
