"""Pins of the oracle's mapping-side association (App. D.1 steps 3-5):
Hellinger neighbour search, union-find correspondence and the
sufficient-statistics fusion.

* the Hellinger distance: 0 for equal Gaussians; equal to 1 minus the
  box-moment Near of App. D.2's Hellinger form for axis-aligned covariances;
  unchanged by a common rotation; and Monte Carlo estimates of the
  Bhattacharyya coefficient E_p[sqrt(q / p)];
* the neighbour lists against a numpy brute force (cosines, numpy.linalg
  determinants and solves);
* the components against a breadth-first search of the match graph, and the
  winner rule (largest weight, lower index on ties);
* the fused moments against the paper's M1 = w mu, M2 = w (S + mu mu') form
  and a hand-built scene.
"""
import math
from collections import deque

import numpy as np
import pytest

import oracle
from oracle import NEAR_H
import synth
from synth import Scene

pytestmark = pytest.mark.usefixtures("oracle_lib")

IX = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def full(c):
    m = np.zeros((3, 3))
    for k, (i, j) in enumerate(IX):
        m[i, j] = m[j, i] = c[k]
    return m


def packed(m):
    return np.asarray([m[i, j] for i, j in IX])


def rand_cov(rng):
    a = rng.standard_normal((3, 3))
    return packed(a @ a.T * 0.1 + 0.02 * np.eye(3))


def test_hellinger_identities():
    rng = np.random.default_rng(0)
    for _ in range(20):
        mu, c = rng.standard_normal(3), rand_cov(rng)
        assert oracle.hellinger(mu, c, mu, c) == pytest.approx(0.0, abs=2e-8)
    # axis-aligned: the box-moment Hellinger Near of the predicate set
    for _ in range(20):
        c = rng.uniform(0, 3, (2, 3))
        s = rng.lognormal(-1, 0.5, (2, 3))
        box = np.zeros((6, 2), np.float32)
        box[:3] = c.T
        box[3:] = s.T
        sc = Scene(desc=np.eye(2, dtype=np.float32), cls=np.zeros(2, np.int32), box=box,
                   views=np.zeros((6, 0, 2), np.float32))
        b = box.astype(np.float64)
        cv = lambda j: np.asarray([b[3, j] ** 2 / 12, 0, 0, b[4, j] ** 2 / 12, 0, b[5, j] ** 2 / 12])  # noqa: E731
        h = oracle.hellinger(b[:3, 0], cv(0), b[:3, 1], cv(1))
        assert h == pytest.approx(1.0 - oracle.relation(sc, NEAR_H, 0, 1), abs=1e-9)
    # a common rotation changes nothing
    for _ in range(20):
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        m1, m2 = rng.standard_normal(3), rng.standard_normal(3)
        c1, c2 = rand_cov(rng), rand_cov(rng)
        r1, r2 = packed(q @ full(c1) @ q.T), packed(q @ full(c2) @ q.T)
        assert oracle.hellinger(q @ m1, r1, q @ m2, r2) == pytest.approx(oracle.hellinger(m1, c1, m2, c2), abs=1e-9)


def test_hellinger_monte_carlo():
    from scipy.stats import multivariate_normal as mvn
    rng = np.random.default_rng(1)
    for _ in range(6):
        m1, m2 = rng.standard_normal(3) * 0.3, rng.standard_normal(3) * 0.3
        c1, c2 = rand_cov(rng), rand_cov(rng)
        p, q = mvn(m1, full(c1)), mvn(m2, full(c2))
        x = p.rvs(size=400000, random_state=rng)
        ratio = np.exp(0.5 * (q.logpdf(x) - p.logpdf(x)))
        bc = ratio.mean()
        se = ratio.std() / math.sqrt(len(x))
        h = oracle.hellinger(m1, c1, m2, c2)
        assert 1.0 - h * h == pytest.approx(bc, abs=6 * se + 1e-4)


def _np_hellinger(m1, c1, m2, c2):
    S1, S2 = full(c1), full(c2)
    S = 0.5 * (S1 + S2)
    d = np.asarray(m1) - np.asarray(m2)
    bc = (np.linalg.det(S1) ** 0.25 * np.linalg.det(S2) ** 0.25 / math.sqrt(np.linalg.det(S))
          * math.exp(-0.125 * d @ np.linalg.solve(S, d)))
    return math.sqrt(max(0.0, 1.0 - bc))


def _case(seed=3, n_det=96):
    scenes, _ = synth.workload("room_n200_d512")
    ent, det = synth.make_association(seed, scenes[0], n_det, feat_dim=32, bridge_frac=0.2)
    return ent, det


def test_neighbour_lists_match_a_brute_force():
    ent, det = _case()
    tau, hmax, mm = 0.8, 0.8, 6
    out = oracle.associate(ent, det, tau, hmax, mm)
    ef = ent["feat"].astype(np.float64)
    df = det["feat"].astype(np.float64)
    cos = (df / np.linalg.norm(df, axis=1, keepdims=True)) @ (ef / np.linalg.norm(ef, axis=1, keepdims=True)).T
    for d in range(df.shape[0]):
        hs = []
        for e in range(ef.shape[0]):
            if not ent["active"][e] or cos[d, e] < tau:
                continue
            h = _np_hellinger(det["mu"][:, d].astype(np.float64), det["cov"][:, d].astype(np.float64),
                              ent["mu"][:, e].astype(np.float64), ent["cov"][:, e].astype(np.float64))
            if h <= hmax:
                hs.append((h, e))
        hs.sort()
        assert out["match_cnt"][d] == len(hs)
        got = [int(x) for x in out["match_idx"][d] if x >= 0]
        assert got == [e for _, e in hs[:mm]]
        assert np.allclose(out["match_h"][d][: len(got)], [h for h, _ in hs[:mm]], atol=1e-9)


def test_components_and_winners():
    ent, det = _case(4, 128)
    out = oracle.associate(ent, det, 0.8, 0.9, 6)
    N, B = ent["mu"].shape[1], det["mu"].shape[1]
    adj = [[] for _ in range(N + B)]
    for d in range(B):
        for e in out["match_idx"][d]:
            if e >= 0:
                adj[N + d].append(int(e))
                adj[int(e)].append(N + d)
    seen = np.full(N + B, -1)
    merges = 0
    for s0 in range(N + B):
        if seen[s0] >= 0:
            continue
        comp, dq = [], deque([s0])
        seen[s0] = s0
        while dq:
            x = dq.popleft()
            comp.append(x)
            for y in adj[x]:
                if seen[y] < 0:
                    seen[y] = s0
                    dq.append(y)
        ents = [x for x in comp if x < N]
        if ents:
            w = ent["w"]
            win = min(ents, key=lambda e: (-w[e], e))
            merges += len(ents) - 1
        else:
            assert len(comp) == 1
            win = comp[0]
        for x in comp:
            assert out["parent"][x] == win
    assert merges > 0       # the bridging detections do merge entities here


def test_fusion_equals_the_sufficient_statistics_form():
    ent, det = _case(5, 128)
    out = oracle.associate(ent, det, 0.8, 0.9, 6)
    N, B = ent["mu"].shape[1], det["mu"].shape[1]
    T = N + B
    mu_all = np.concatenate([ent["mu"], det["mu"]], axis=1).astype(np.float64)
    cv_all = np.concatenate([ent["cov"], det["cov"]], axis=1).astype(np.float64)
    w_all = np.concatenate([ent["w"], np.ones(B)]).astype(np.float64)
    f_all = np.concatenate([ent["feat"], det["feat"]]).astype(np.float64)
    for g in np.unique(out["parent"]):
        mem = np.flatnonzero(out["parent"] == g)
        w = w_all[mem].sum()
        M1 = (w_all[mem] * mu_all[:, mem]).sum(axis=1)
        M2 = sum(w_all[x] * (full(cv_all[:, x]) + np.outer(mu_all[:, x], mu_all[:, x])) for x in mem)
        mu = M1 / w
        S = M2 / w - np.outer(mu, mu)
        assert out["w"][g] == pytest.approx(w, rel=1e-12)
        assert np.allclose(out["mu"][:, g], mu, rtol=1e-12, atol=1e-12)
        assert np.allclose(full(out["cov"][:, g]), S, rtol=1e-7, atol=1e-9)
        assert np.allclose(out["feat"][g], (w_all[mem, None] * f_all[mem]).sum(axis=0) / w, atol=1e-12)
    gone = np.flatnonzero(out["parent"] != np.arange(T))
    assert np.all(out["w"][gone] == 0.0)


def test_hand_built_association():
    """Entities 0 (w 3) and 1 (w 5), 2 m apart, one class; entity 2 elsewhere.
    Detection 0 re-observes entity 0, detection 1 spans entities 0 and 1
    (bridging them), detection 2 is a new object far away.  Entity 1 wins
    the merged component (larger weight); entity 2 is untouched."""
    f = np.zeros((3, 4), np.float32)
    f[:, 0] = 1.0
    ent = dict(mu=np.asarray([[0.0, 2.0, 9.0], [0.0, 0.0, 9.0], [0.5, 0.5, 0.5]], np.float32),
               cov=np.tile(np.asarray([0.04, 0, 0, 0.04, 0, 0.04], np.float32)[:, None], (1, 3)),
               feat=f, w=np.asarray([3.0, 5.0, 2.0], np.float32), active=np.ones(3, np.int32))
    det = dict(mu=np.asarray([[0.02, 1.0, 20.0], [0.0, 0.0, 20.0], [0.5, 0.5, 0.5]], np.float32),
               cov=np.asarray([[0.04, 1.2, 0.04], [0, 0, 0], [0, 0, 0], [0.04, 0.3, 0.04], [0, 0, 0],
                               [0.04, 0.3, 0.04]], np.float32),
               feat=np.asarray([[1, 0, 0, 0]] * 3, np.float32))
    out = oracle.associate(ent, det, 0.9, 0.9, 4)
    assert out["match_idx"][0][0] == 0
    assert sorted(int(x) for x in out["match_idx"][1] if x >= 0) == [0, 1]
    assert out["match_cnt"][2] == 0
    assert out["parent"].tolist() == [1, 1, 2, 1, 1, 5]
    # w = 3 + 5 + 1 + 1; mu = (3*0 + 5*2 + 0.02 + 1) / 10 along x
    assert out["w"][1] == pytest.approx(10.0)
    assert out["mu"][0, 1] == pytest.approx((3 * 0 + 5 * 2 + 0.02 + 1.0) / 10.0, rel=1e-6)
    assert out["w"][0] == 0.0 and out["w"][3] == 0.0 and out["w"][4] == 0.0
    assert out["w"][5] == 1.0 and out["w"][2] == 2.0
