"""Pins of the oracle's several-channel retrieval (App. D.2 step 3:
reciprocal-rank fusion over query channels in several embedding spaces; the
landmarks retrieved the same way).

* one channel of weight 1 is the single-channel oracle, value for value;
* a channel repeated with weights a and b fuses like one channel of weight
  a + b;
* a hand-built two-space scene whose per-channel ranks, fused scores and
  composite are worked out by hand;
* a brute force over every anchor tuple, with ranks taken from exact
  rational dot products of small integer vectors;
* relabelling the objects relabels the result (TopK invariance);
* the tie-tolerant bounds collapse to the exact result at tau = 0.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import ABOVE, BELOW, NEAR, LEFT_OF, OracleParams
import synth
from synth import Scene

pytestmark = pytest.mark.usefixtures("oracle_lib")

P = OracleParams()


def _small(seed=0, n=40, dims=(24, 16, 32)):
    sc = synth.make_scene(seed, n, dims[0], extent=(6.0, 6.0, 3.0), n_classes=5, n_views=3)
    sp = synth.add_spaces(sc, seed + 100, dims=dims[1:])
    qb = synth.make_queries(seed + 200, sc, 6, m_choices=(0, 1, 2, 3), preds=list(range(15)))
    cq = synth.channel_queries(seed + 300, sc, sp, qb)
    return sc, sp, qb, cq


def _q(qb, cq, q):
    m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
    return ([t[q] for t in cq.tgt], int(qb.tgt_cls[q]), qb.c_pred[m0:m1], [l[m0:m1] for l in cq.lm])


def test_one_channel_is_the_single_channel_oracle():
    sc, sp, qb, cq = _small()
    for q in range(qb.n_q):
        m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
        got = oracle.query_mc(sc, sp.desc, [(0, 1.0)], [qb.tgt_emb[q]], int(qb.tgt_cls[q]), qb.c_pred[m0:m1],
                              [qb.c_emb[m0:m1]])
        ref = oracle.query_all(sc, qb.tgt_emb[q], int(qb.tgt_cls[q]), qb.c_pred[m0:m1], qb.c_emb[m0:m1])
        assert np.array_equal(got["fused"], 1.0 / (P.mu + ref["rank0"]))
        # cf * (1 / (mu + r)) against cf / (mu + r): one rounding apart
        assert np.allclose(got["s_sem"], ref["s_sem"], rtol=1e-15, atol=0)
        assert np.array_equal(got["t"], ref["t"]) and np.array_equal(got["anchor"], ref["anchor"])
        assert np.allclose(got["s"], ref["s"], rtol=1e-15, atol=0)


def test_repeated_channel_adds_its_weights():
    sc, sp, qb, cq = _small(1)
    for q in range(qb.n_q):
        u0, ct, pr, uc = _q(qb, cq, q)
        two = oracle.query_mc(sc, sp.desc, [(1, 0.25), (1, 0.5)], [u0[0], u0[0]], ct, pr, [uc[0], uc[0]])
        one = oracle.query_mc(sc, sp.desc, [(1, 0.75)], [u0[0]], ct, pr, [uc[0]])
        assert np.allclose(two["fused"], one["fused"], rtol=1e-15, atol=0)
        assert np.array_equal(two["anchor"], one["anchor"])
        assert np.allclose(two["s"], one["s"], rtol=1e-14, atol=0)


def _hand_scene():
    """Four objects; space 0 is 2-d, space 1 is 3-d.  Target channels:
    channel A (space 0, w = 1) ranks the objects 0, 1, 2, 3; channel B
    (space 1, w = 0.5) ranks them 2, 0, 3, 1."""
    d0 = np.array([[1, 0], [3, 1], [1, 1], [0, 1]], np.float32)      # cos to (1, 0): 1, .949, .707, 0
    d1 = np.array([[4, 2, 0], [0, 0, 1], [1, 0, 0], [1, 1, 1]], np.float32)  # cos to (1,0,0): .894, 0, 1, .577
    box = np.zeros((6, 4), np.float32)
    box[0] = [0.0, 0.0, 5.0, 3.0]
    box[1] = [0.0, 0.0, 0.0, 0.0]
    box[2] = [1.0, 0.0, 1.0, 0.2]        # heights: objects 0, 2 low (1.0), 1 (0.0), 3 high (0.2)
    box[3:] = 0.3
    views = np.zeros((6, 0, 4), np.float32)
    sc = Scene(desc=d0, cls=np.array([0, 0, 0, 1], np.int32), box=box, views=views)
    return sc, [d0, d1]


def test_hand_built_fusion():
    sc, spaces = _hand_scene()
    ch = [(0, 1.0), (1, 0.5)]
    out = oracle.query_mc(sc, spaces, ch, [np.array([1, 0], np.float32), np.array([1, 0, 0], np.float32)],
                          -1, [], [np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32)])
    # ranks A: 1, 2, 3, 4; ranks B: 2, 4, 1, 3
    want = [1 / 6 + 0.5 / 7, 1 / 7 + 0.5 / 9, 1 / 8 + 0.5 / 6, 1 / 9 + 0.5 / 8]
    assert np.allclose(out["fused"], want, rtol=1e-15, atol=0)
    assert np.allclose(out["s"], want, rtol=1e-15, atol=0)          # m = 0: s = s_sem
    # with a target class 0, object 3 (class 1) takes the 0.3 factor
    out = oracle.query_mc(sc, spaces, ch, [np.array([1, 0], np.float32), np.array([1, 0, 0], np.float32)],
                          0, [], [np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32)])
    assert out["s"][3] == pytest.approx(0.3 * want[3], rel=1e-15)
    # one constraint "above the landmark" whose two channels rank object 1
    # first in A (u = (3, 1)) and object 3 first in B (u = (1, 1, 1)); with
    # K_a = 1 the landmark is the object of largest fused landmark score:
    # object 1 scores 1/6 + 0.5/(5+r_B(1)), object 3 scores 1/(5+r_A(3)) + 0.5/6
    p1 = OracleParams(k_anchor=1)
    lmA, lmB = np.array([[3, 1]], np.float32), np.array([[1, 1, 1]], np.float32)
    out = oracle.query_mc(sc, spaces, ch, [np.array([1, 0], np.float32), np.array([1, 0, 0], np.float32)],
                          -1, [ABOVE], [lmA, lmB], params=p1)
    cA = oracle.cosines(Scene(desc=spaces[0], cls=sc.cls, box=sc.box, views=sc.views), lmA[0])
    cB = oracle.cosines(Scene(desc=spaces[1], cls=sc.cls, box=sc.box, views=sc.views), lmB[0])
    rA, rB = oracle.ranks(cA), oracle.ranks(cB)
    assert rA[1] == 1 and rB[3] == 1
    F1, F3 = 1 / (5 + rA[1]) + 0.5 / (5 + rB[1]), 1 / (5 + rA[3]) + 0.5 / (5 + rB[3])
    lm = 1 if F1 > F3 else 3
    for e in range(4):
        assert out["anchor"][0][e] == (lm if e != lm else -1)
    # Above: sig((z_e - z_lm) / tau_v)
    for e in range(4):
        if e != lm:
            dz = float(sc.box[2, e]) - float(sc.box[2, lm])
            assert out["t"][0][e] == pytest.approx(1 / (1 + np.exp(-dz / P.tau_v)), rel=1e-12)


def _exact_ranks(vecs, u):
    """Ranks by exact rational cosine (ties: lower index first)."""
    def cos(v):
        dot = sum(Fraction(int(a)) * int(b) for a, b in zip(v, u))
        nv = sum(int(a) * int(a) for a in v)
        nu = sum(int(b) * int(b) for b in u)
        # compare dot / sqrt(nv nu) exactly through the sign and the square
        return (1 if dot > 0 else (-1 if dot < 0 else 0), Fraction(dot * dot, nv * nu))

    def key(j):
        sg, sq = cos(vecs[j])
        return (-(sg * sq), j)
    order = sorted(range(len(vecs)), key=key)
    r = np.zeros(len(vecs), np.int64)
    for pos, j in enumerate(order):
        r[j] = pos + 1
    return r


def test_brute_force_over_anchor_tuples():
    """Every binding (one anchor per constraint among its fused top K_a)
    scored directly; the best per target equals the oracle's composite."""
    rng = np.random.default_rng(5)
    n = 7
    p = OracleParams(k_anchor=3)
    for trial in range(6):
        s0 = rng.integers(-3, 4, (n, 3)).astype(np.float32)
        s1 = rng.integers(-3, 4, (n, 4)).astype(np.float32)
        s0[np.all(s0 == 0, axis=1)] = 1
        s1[np.all(s1 == 0, axis=1)] = 1
        box = np.zeros((6, n), np.float32)
        box[:3] = rng.uniform(0, 3, (3, n))
        box[3:] = rng.uniform(0.1, 0.8, (3, n))
        sc = Scene(desc=s0, cls=rng.integers(0, 2, n).astype(np.int32), box=box,
                   views=np.zeros((6, 0, n), np.float32))
        ch = [(0, 1.0), (1, 0.5), (1, 0.75)]
        u0 = [rng.integers(-3, 4, 3).astype(np.float32), rng.integers(-3, 4, 4).astype(np.float32),
              rng.integers(-3, 4, 4).astype(np.float32)]
        for u in u0:
            if not np.any(u):
                u[0] = 1
        preds = [ABOVE, NEAR, BELOW][: 1 + trial % 3]
        m = len(preds)
        uc = [rng.integers(-3, 4, (m, 3)).astype(np.float32), rng.integers(-3, 4, (m, 4)).astype(np.float32),
              rng.integers(-3, 4, (m, 4)).astype(np.float32)]
        for a in uc:
            a[np.all(a == 0, axis=1)] = 1
        c_t = -1 if trial % 2 == 0 else 1
        spaces = [s0, s1]
        got = oracle.query_mc(sc, spaces, ch, u0, c_t, preds, uc, params=p)

        def fused(embs):
            F = np.zeros(n)
            for (sp, w), u in zip(ch, embs):
                F += w / (p.mu + _exact_ranks(spaces[sp], u))
            return F
        F0 = fused(u0)
        lms = []
        for i in range(m):
            Fi = fused([uc[c][i] for c in range(len(ch))])
            order = sorted(range(n), key=lambda j: (-Fi[j], j))
            lms.append(order[: p.k_anchor])
        for e in range(n):
            cf = p.class_mis if (c_t >= 0 and sc.cls[e] != c_t) else 1.0
            best = None
            for tup in itertools.product(*lms):
                if any(a == e for a in tup):
                    continue
                t = [oracle.relation(sc, preds[i], e, a, p) for i, a in enumerate(tup)]
                g = 0.0 if min(t) <= 0 else float(np.exp(np.mean(np.log(t))))
                v = cf * F0[e] * ((1 - p.w) + p.w * g)
                best = v if best is None else max(best, v)
            if best is None:        # e is in every candidate list of size 1...: no full binding
                continue
            assert got["s"][e] == pytest.approx(best, rel=1e-12), (trial, e)
        assert np.allclose(got["fused"], F0, rtol=1e-14, atol=0)


def test_relabelling_objects_relabels_the_result():
    sc, sp, qb, cq = _small(2)
    perm = np.random.default_rng(9).permutation(sc.n)
    inv = np.argsort(perm)
    psc = Scene(desc=np.ascontiguousarray(sc.desc[perm]), cls=sc.cls[perm],
                box=np.ascontiguousarray(sc.box[:, perm]), views=np.ascontiguousarray(sc.views[:, :, perm]))
    psp = [np.ascontiguousarray(d[perm]) for d in sp.desc]
    for q in range(qb.n_q):
        u0, ct, pr, uc = _q(qb, cq, q)
        a = oracle.query_mc(sc, sp.desc, cq.channels, u0, ct, pr, uc)
        b = oracle.query_mc(psc, psp, cq.channels, u0, ct, pr, uc)
        assert np.allclose(b["s"][inv], a["s"], rtol=1e-13, atol=0)
        k = 5
        ta = oracle.topk(a["s"], k)
        tb = perm[oracle.topk(b["s"], k)]
        assert np.allclose(a["s"][ta], a["s"][tb], rtol=1e-13, atol=0)


def test_bounds_collapse_at_zero_tolerance():
    sc, sp, qb, cq = _small(3)
    for q in range(qb.n_q):
        u0, ct, pr, uc = _q(qb, cq, q)
        ex = oracle.query_mc(sc, sp.desc, cq.channels, u0, ct, pr, uc)
        b = oracle.query_bounds_mc(sc, sp.desc, cq.channels, u0, ct, pr, uc, tau=0.0)
        assert np.array_equal(b["F_lo"], ex["fused"]) and np.array_equal(b["F_hi"], ex["fused"])
        # closest / farthest and tied fused scores may leave ranges open; the
        # exact value always lies inside them
        assert np.all(b["s_lo"] <= ex["s"] * (1 + 1e-12)) and np.all(ex["s"] <= b["s_hi"] * (1 + 1e-12))
        b2 = oracle.query_bounds_mc(sc, sp.desc, cq.channels, u0, ct, pr, uc, tau=1e-3)
        assert np.all(b2["s_lo"] <= b["s_lo"] * (1 + 1e-12)) and np.all(b["s_hi"] <= b2["s_hi"] * (1 + 1e-12))
