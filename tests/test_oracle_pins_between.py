"""Pins of the oracle's Between relation (App. B: a ternary predicate that
couples only the variables it mentions; exact binding of the pair by bucket
elimination).  The paper gives no evaluator; the reading pinned here is
sig(t / 0.1) sig((1 - t) / 0.1) exp(-d^2 / (2 sigma_near^2)) with t the
position of e's centre along the segment from a_p to a_q and d its distance
from the line.

* closed forms at the midpoint, at an end, off the line, past the segment;
* swapping the two landmarks changes nothing; coincident landmarks score 0;
* a query with a Between pair and a second relation, against a brute force
  over every (a_p, a_q, a) binding: the pair is one factor of the geometric
  mean, and both of its constraints report its score and the bound pair;
* malformed pair encodings are rejected.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import ABOVE, BETWEEN, BETWEEN_AND, NEAR, OracleParams
from synth import Scene

pytestmark = pytest.mark.usefixtures("oracle_lib")

P = OracleParams()
SIG = lambda x: 1.0 / (1.0 + math.exp(-x))   # noqa: E731


def boxes(centres):
    n = len(centres)
    box = np.zeros((6, n), np.float32)
    box[:3] = np.asarray(centres, np.float32).T
    box[3:] = 0.3
    return Scene(desc=np.eye(n, max(n, 2), dtype=np.float32), cls=np.zeros(n, np.int32), box=box,
                 views=np.zeros((6, 0, n), np.float32))


def test_between_closed_forms():
    sc = boxes([[1.0, 0.0, 0.5], [0.0, 0.0, 0.5], [2.0, 0.0, 0.5]])        # e midway between a_p and a_q
    assert oracle.between(sc, 0, 1, 2) == pytest.approx(SIG(5.0) ** 2, rel=1e-12)
    sc = boxes([[0.0, 0.0, 0.5], [0.0, 0.0, 0.5], [2.0, 0.0, 0.5]])        # e at a_p: t = 0
    assert oracle.between(sc, 0, 1, 2) == pytest.approx(0.5 * SIG(10.0), rel=1e-12)
    sc = boxes([[1.0, 0.4, 0.5], [0.0, 0.0, 0.5], [2.0, 0.0, 0.5]])        # 0.4 m off the line at t = 1/2
    assert oracle.between(sc, 0, 1, 2) == pytest.approx(SIG(5.0) ** 2 * math.exp(-0.16 / 0.5), rel=1e-6)
    sc = boxes([[3.0, 0.0, 0.5], [0.0, 0.0, 0.5], [2.0, 0.0, 0.5]])        # past a_q: t = 1.5
    assert oracle.between(sc, 0, 1, 2) == pytest.approx(SIG(15.0) * SIG(-5.0), rel=1e-9)
    sc = boxes([[1.0, 0.0, 0.5], [2.0, 0.0, 0.5], [2.0, 0.0, 0.5]])        # coincident landmarks
    assert oracle.between(sc, 0, 1, 2) == 0.0


def test_between_is_symmetric_in_its_landmarks():
    rng = np.random.default_rng(4)
    for _ in range(50):
        sc = boxes(rng.uniform(0, 4, (3, 3)))
        assert oracle.between(sc, 0, 1, 2) == pytest.approx(oracle.between(sc, 0, 2, 1), rel=1e-12, abs=1e-300)


def _scene(seed, n=9):
    rng = np.random.default_rng(seed)
    c = rng.integers(-3, 4, (n, 4)).astype(np.float32)
    c[np.all(c == 0, axis=1)] = 1
    box = np.zeros((6, n), np.float32)
    box[:3] = rng.uniform(0, 3, (3, n))
    box[3:] = rng.uniform(0.1, 0.6, (3, n))
    return Scene(desc=c, cls=rng.integers(0, 2, n).astype(np.int32), box=box,
                 views=np.zeros((6, 0, n), np.float32))


def test_brute_force_with_a_between_pair():
    p = OracleParams(k_anchor=3)
    for seed in range(6):
        sc = _scene(seed)
        rng = np.random.default_rng(100 + seed)
        preds = [BETWEEN, BETWEEN_AND, NEAR] if seed % 2 else [ABOVE, BETWEEN, BETWEEN_AND]
        u0 = rng.integers(-3, 4, 4).astype(np.float32)
        if not np.any(u0):
            u0[0] = 1
        uc = rng.integers(-3, 4, (3, 4)).astype(np.float32)
        uc[np.all(uc == 0, axis=1)] = 1
        c_t = -1 if seed % 3 else 1
        out = oracle.query_all(sc, u0, c_t, np.asarray(preds, np.int32), uc, params=p)
        ranks = [oracle.ranks(oracle.cosines(sc, uc[i])) for i in range(3)]
        lists = [sorted(range(sc.n), key=lambda j: r[j])[: p.k_anchor] for r in ranks]
        r0 = oracle.ranks(oracle.cosines(sc, u0))
        pair = 0 if preds[0] == BETWEEN else 1
        other = 2 if pair == 0 else 0
        for e in range(sc.n):
            cf = p.class_mis if (c_t >= 0 and sc.cls[e] != c_t) else 1.0
            ssem = cf / (p.mu + r0[e])
            best, arg = None, None
            for ap, aq, a in itertools.product(lists[pair], lists[pair + 1], lists[other]):
                if e in (ap, aq, a) or ap == aq:
                    continue
                tb = oracle.between(sc, e, ap, aq, p)
                to = oracle.relation(sc, preds[other], e, a, p)
                g = 0.0 if min(tb, to) <= 0 else math.sqrt(tb * to)      # two factors: the pair and the other
                v = ssem * ((1 - p.w) + p.w * g)
                if best is None or v > best:
                    best = v
            assert out["s"][e] == pytest.approx(best, rel=1e-12), (seed, e)
            # both constraints of the pair carry its score and bound pair
            assert out["t"][pair][e] == out["t"][pair + 1][e]
            ap, aq = out["anchor"][pair][e], out["anchor"][pair + 1][e]
            if ap >= 0:
                assert ap != aq and e not in (ap, aq)
                assert ap in lists[pair] and aq in lists[pair + 1]
                assert out["t"][pair][e] == pytest.approx(oracle.between(sc, e, ap, aq, p), rel=1e-15)
                for x, y in itertools.product(lists[pair], lists[pair + 1]):
                    if e not in (x, y) and x != y:
                        assert oracle.between(sc, e, x, y, p) <= out["t"][pair][e] + 1e-15


def test_malformed_pairs_are_rejected():
    sc = _scene(0)
    u0 = np.ones(4, np.float32)
    for preds in ([BETWEEN], [BETWEEN_AND], [BETWEEN_AND, BETWEEN], [BETWEEN, NEAR]):
        with pytest.raises(ValueError):
            oracle.query_all(sc, u0, -1, np.asarray(preds, np.int32), np.ones((len(preds), 4), np.float32))


def test_bounds_cover_the_pair_at_zero_tolerance():
    p = OracleParams(k_anchor=3)
    sc = _scene(7)
    preds = np.asarray([BETWEEN, BETWEEN_AND], np.int32)
    rng = np.random.default_rng(8)
    u0 = rng.standard_normal(4).astype(np.float32)
    uc = rng.standard_normal((2, 4)).astype(np.float32)
    ex = oracle.query_all(sc, u0, -1, preds, uc, params=p)
    b = oracle.query_bounds(sc, u0, -1, preds, uc, tau=0.0, params=p)
    assert np.allclose(b["s_lo"], ex["s"], rtol=1e-14) and np.allclose(b["s_hi"], ex["s"], rtol=1e-14)
    assert np.allclose(b["t_lo"], ex["t"], rtol=1e-14) and np.allclose(b["t_hi"], ex["t"], rtol=1e-14)


def test_a_pair_binds_two_distinct_landmarks():
    """Two landmarks at one point: every pair scores 0, and the bound pair is
    still two distinct objects (the lower-index pair (1, 2), never (1, 1))."""
    p = OracleParams(k_anchor=2)
    box = np.zeros((6, 3), np.float32)
    box[:3] = np.asarray([[0.0, 0.0, 0.5], [1.0, 1.0, 0.5], [1.0, 1.0, 0.5]], np.float32).T
    box[3:] = 0.3
    desc = np.asarray([[1, 0, 0], [0, 1, 0], [0, 1, 0.01]], np.float32)
    sc = Scene(desc=desc, cls=np.zeros(3, np.int32), box=box, views=np.zeros((6, 0, 3), np.float32))
    uc = np.asarray([[0, 1, 0], [0, 1, 0]], np.float32)
    out = oracle.query_all(sc, np.asarray([1, 0, 0], np.float32), -1, np.asarray([BETWEEN, BETWEEN_AND], np.int32),
                           uc, params=p)
    assert out["t"][0][0] == 0.0
    assert (out["anchor"][0][0], out["anchor"][1][0]) == (1, 2)
