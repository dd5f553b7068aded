"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
example of App. C (hand-derived expectations in tests/golden/), closed forms of
the App. D.2 evaluators, exact rational arithmetic, brute-force enumeration of
bindings (the star decomposition of App. B), textbook special cases, and
invariants (symmetry, permutation, the [1-w, 1] blend bound of App. D.2).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import ABOVE, BELOW, LEFT_OF, NEAR, RIGHT_OF, OracleParams
import synth
from scenes_util import golden_case, load_golden, single_query, tiny_scene
from synth import Scene

pytestmark = pytest.mark.usefixtures("oracle_lib")

P = OracleParams()


def two_objects(pe, pa, views_e=None):
    """Scene of two objects e=0, a=1 with the given centres and views of e."""
    box = np.zeros((6, 2), np.float32)
    box[:3, 0], box[:3, 1] = pe, pa
    box[3:] = 0.5
    vs = views_e or []
    views = np.zeros((6, max(len(vs), 1), 2), np.float32)
    for v, (o, f) in enumerate(vs):
        views[:3, v, 0] = o
        views[3:, v, 0] = f
    if not vs:
        views = np.zeros((6, 0, 2), np.float32)
    desc = np.eye(2, 4, dtype=np.float32)
    return Scene(desc=desc, cls=np.zeros(2, np.int32), box=box, views=views)


# --- closed forms of the evaluators (App. D.2 step 4) -----------------------

def test_sigmoid_closed_forms():
    assert oracle.sigmoid(0.0) == 0.5
    assert oracle.sigmoid(math.log(3.0)) == pytest.approx(0.75, abs=1e-15)
    assert oracle.sigmoid(-math.log(3.0)) == pytest.approx(0.25, abs=1e-15)
    assert oracle.sigmoid(math.log(9.0)) == pytest.approx(0.9, abs=1e-15)
    assert oracle.sigmoid(-800.0) == 0.0 and oracle.sigmoid(800.0) == 1.0


def test_above_below_closed_form():
    dz = P.tau_v * math.log(3.0)
    sc = two_objects([1.0, 2.0, 1.0 + dz], [1.0, 2.0, 1.0])
    assert oracle.relation(sc, ABOVE, 0, 1) == pytest.approx(0.75, abs=1e-6)
    assert oracle.relation(sc, BELOW, 0, 1) == pytest.approx(0.25, abs=1e-6)
    flat = two_objects([0.0, 0.0, 2.0], [5.0, -3.0, 2.0])
    assert oracle.relation(flat, ABOVE, 0, 1) == 0.5
    assert oracle.relation(flat, BELOW, 0, 1) == 0.5


def test_above_is_below_swapped_bitwise():
    sc, _ = synth.workload("room_n200_d512")
    s = sc[0]
    rng = np.random.default_rng(1)
    for e, a in rng.integers(0, s.n, size=(200, 2)):
        assert oracle.relation(s, ABOVE, e, a) == oracle.relation(s, BELOW, a, e)


def test_near_closed_form_and_symmetry():
    d_half = P.sigma_near * math.sqrt(2.0 * math.log(2.0))
    sc = two_objects([0.0, 0.0, 0.0], [d_half, 0.0, 0.0])
    assert oracle.relation(sc, NEAR, 0, 1) == pytest.approx(0.5, abs=1e-7)
    d_e = P.sigma_near * math.sqrt(2.0)
    sc = two_objects([1.0, 1.0, 1.0], [1.0, 1.0 + d_e, 1.0])
    assert oracle.relation(sc, NEAR, 0, 1) == pytest.approx(math.exp(-1.0), abs=1e-7)
    assert oracle.relation(sc, NEAR, 0, 0) == 1.0
    sc, _ = synth.workload("room_n200_d512")
    rng = np.random.default_rng(2)
    for e, a in rng.integers(0, sc[0].n, size=(200, 2)):
        assert oracle.relation(sc[0], NEAR, e, a) == oracle.relation(sc[0], NEAR, a, e)


SOUTH = ([5.0, 3.0, 1.0], [0.0, 1.0, 0.0])   # 2 m south of (5,5,1), looking north; right = +x
NORTH = ([5.0, 7.0, 1.0], [0.0, -1.0, 0.0])  # 2 m north, looking south; right = -x


def test_left_right_hand_computed_single_view():
    # a sits tau_h*ln3*2 m east of e; seen from the south at depth 2 m its image
    # coordinate is tau_h*ln3, e's is 0, so left_of = sig(ln 3) = 0.75.
    dx = 2.0 * P.tau_h * math.log(3.0)
    sc = two_objects([5.0, 5.0, 1.0], [5.0 + dx, 5.0, 1.0], [SOUTH])
    assert oracle.relation(sc, LEFT_OF, 0, 1) == pytest.approx(0.75, abs=1e-6)
    assert oracle.relation(sc, RIGHT_OF, 0, 1) == pytest.approx(0.25, abs=1e-6)


def test_left_right_mean_over_views():
    dx = 2.0 * P.tau_h * math.log(3.0)
    sc = two_objects([5.0, 5.0, 1.0], [5.0 + dx, 5.0, 1.0], [SOUTH, NORTH])
    # the northern view sees a on the left: mean(0.75, 0.25) = 0.5
    assert oracle.relation(sc, LEFT_OF, 0, 1) == pytest.approx(0.5, abs=1e-6)
    sc3 = two_objects([5.0, 5.0, 1.0], [5.0 + dx, 5.0, 1.0], [SOUTH, SOUTH, NORTH])
    assert oracle.relation(sc3, LEFT_OF, 0, 1) == pytest.approx((0.75 * 2 + 0.25) / 3, abs=1e-6)


def test_left_right_no_valid_view_is_half():
    # a behind the only camera
    sc = two_objects([5.0, 5.0, 1.0], [5.5, 2.5, 1.0], [SOUTH])
    assert oracle.relation(sc, LEFT_OF, 0, 1) == 0.5
    assert oracle.relation(sc, RIGHT_OF, 0, 1) == 0.5
    # camera looking straight down has no horizontal image axis
    sc = two_objects([5.0, 5.0, 1.0], [6.0, 5.0, 1.0], [([5.0, 5.0, 3.0], [0.0, 0.0, -1.0])])
    assert oracle.relation(sc, LEFT_OF, 0, 1) == 0.5
    # no stored views at all
    sc = two_objects([5.0, 5.0, 1.0], [6.0, 5.0, 1.0])
    assert oracle.relation(sc, LEFT_OF, 0, 1) == 0.5
    # one invalid view does not dilute a valid one
    dx = 2.0 * P.tau_h * math.log(3.0)
    behind = ([5.0 + dx, 5.5, 1.0], [0.0, 1.0, 0.0])   # a is behind this camera
    sc = two_objects([5.0, 5.0, 1.0], [5.0 + dx, 5.0, 1.0], [SOUTH, behind])
    assert oracle.relation(sc, LEFT_OF, 0, 1) == pytest.approx(0.75, abs=1e-6)


def test_left_plus_right_is_one():
    sc, _ = synth.workload("room_n200_d512")
    rng = np.random.default_rng(3)
    for e, a in rng.integers(0, sc[0].n, size=(300, 2)):
        l = oracle.relation(sc[0], LEFT_OF, e, a)
        r = oracle.relation(sc[0], RIGHT_OF, e, a)
        assert l + r == pytest.approx(1.0, abs=1e-12)


def test_mirror_swaps_left_and_right_exactly():
    sc, _ = synth.workload("room_n200_d512")
    s = sc[0]
    m = Scene(desc=s.desc, cls=s.cls, box=s.box.copy(), views=s.views.copy())
    m.box[0] *= -1.0
    m.views[0] *= -1.0
    m.views[3] *= -1.0
    rng = np.random.default_rng(4)
    for e, a in rng.integers(0, s.n, size=(300, 2)):
        assert oracle.relation(m, LEFT_OF, e, a) == oracle.relation(s, RIGHT_OF, e, a)
        assert oracle.relation(m, RIGHT_OF, e, a) == oracle.relation(s, LEFT_OF, e, a)


# --- cosines and ranks (App. D.2 step 3) -------------------------------------

def _exact_order_key(u, d):
    """Exact cosine as a comparable key: sign(dot) * dot^2 / (|u|^2 |d|^2)."""
    dot = sum(Fraction(int(x)) * Fraction(int(y)) for x, y in zip(u, d))
    nn = sum(Fraction(int(x)) ** 2 for x in u) * sum(Fraction(int(y)) ** 2 for y in d)
    return (1 if dot > 0 else -1 if dot < 0 else 0) * dot * dot / nn


def test_ranks_match_exact_rational_order():
    rng = np.random.default_rng(5)
    for trial in range(20):
        n, dim = 40, 5
        base = rng.integers(-3, 4, size=(n, dim))
        base[base.sum(axis=1) == 0, 0] += 1
        base[np.abs(base).sum(axis=1) == 0, 0] = 1
        # exact duplicates and positive multiples share a cosine: lower index must win
        base[7] = base[3]
        base[11] = 2 * base[5]
        u = rng.integers(-3, 4, size=dim)
        u[0] = u[0] if np.any(u) else 1
        if not np.any(u):
            u[0] = 1
        sc = Scene(desc=base.astype(np.float32), cls=np.zeros(n, np.int32),
                   box=np.zeros((6, n), np.float32), views=np.zeros((6, 0, n), np.float32))
        c = oracle.cosines(sc, u.astype(np.float32))
        r = oracle.ranks(c)
        keys = [_exact_order_key(u, base[j]) for j in range(n)]
        expect = sorted(range(n), key=lambda j: (-keys[j], j))
        # only distinct exact keys are ordered by the exact arithmetic; equal
        # keys must be ordered by index
        got = sorted(range(n), key=lambda j: r[j])
        assert [keys[j] for j in got] == [keys[j] for j in expect]
        for a, b in zip(got, got[1:]):
            if keys[a] == keys[b]:
                assert a < b


def test_cosines_match_library_matmul():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    d = s.desc.astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    u = qb.tgt_emb[0].astype(np.float64)
    u /= np.linalg.norm(u)
    np.testing.assert_allclose(oracle.cosines(s, qb.tgt_emb[0]), d @ u, rtol=0, atol=1e-14)


def test_zero_embedding_is_rejected():
    sc, _ = synth.workload("room_n200_d512")
    with pytest.raises(ValueError):
        oracle.cosines(sc[0], np.zeros(sc[0].dim, np.float32))


# --- special cases with a textbook answer ------------------------------------

def test_no_constraints_no_class_is_topk_of_cosine():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    d = s.desc.astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for q in range(8):
        u = qb.tgt_emb[q].astype(np.float64)
        c = d @ (u / np.linalg.norm(u))
        expect = np.lexsort((np.arange(s.n), -c))[:10]
        one = single_query(qb.tgt_emb[q], -1, [], np.zeros((0, s.dim)), s.dim)
        got = oracle.batch(s, one, 10)
        assert list(got["idx"][0]) == list(expect)
        np.testing.assert_allclose(got["score"][0], 1.0 / (5.0 + np.arange(1, 11)), rtol=0, atol=1e-15)


def test_class_factor_scales_mismatches_only():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    q = 0
    m0, m1 = qb.c_off[q], qb.c_off[q + 1]
    out = oracle.query_all(s, qb.tgt_emb[q], qb.tgt_cls[q], qb.c_pred[m0:m1], qb.c_emb[m0:m1])
    cf = out["s_sem"] * (5.0 + out["rank0"])
    mism = s.cls != qb.tgt_cls[q]
    np.testing.assert_allclose(cf[mism], 0.3, rtol=1e-15)
    np.testing.assert_allclose(cf[~mism], 1.0, rtol=1e-15)


def test_blend_bound_half_to_one():
    """App. D.2 'Why soft, not hard?': the spatial factor stays in [1-w, 1]."""
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    for q in range(10):
        m0, m1 = qb.c_off[q], qb.c_off[q + 1]
        out = oracle.query_all(s, qb.tgt_emb[q], qb.tgt_cls[q], qb.c_pred[m0:m1], qb.c_emb[m0:m1])
        ratio = out["s"] / out["s_sem"]
        assert np.all(ratio >= 0.5 - 1e-15) and np.all(ratio <= 1.0 + 1e-15)


# --- the star decomposition against brute-force enumeration (App. B) ---------

def _brute_force_scores(s, u0, c_t, preds, u_c, k_anchor, params):
    """max over all anchor tuples of Verify(eta), by explicit enumeration."""
    n = s.n
    d = s.desc.astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)

    def order(u):
        u = np.asarray(u, np.float64)
        c = d @ (u / np.linalg.norm(u))
        return np.lexsort((np.arange(n), -c))

    o0 = order(u0)
    rank0 = np.empty(n, np.int64)
    rank0[o0] = np.arange(1, n + 1)
    cands = [list(order(u_c[i])[:min(k_anchor, n)]) for i in range(len(preds))]
    rel = {}
    best = np.zeros(n)
    for e in range(n):
        cf = params.class_mis if (c_t >= 0 and s.cls[e] != c_t) else 1.0
        s_sem = cf / (params.mu + rank0[e])
        pools = [[a for a in L if a != e] for L in cands]
        if any(len(p) == 0 for p in pools):
            best[e] = s_sem * (1 - params.w) if preds else s_sem
            continue
        top = -1.0
        for tup in itertools.product(*pools):
            vals = []
            for i, a in enumerate(tup):
                key = (int(preds[i]), e, a)
                if key not in rel:
                    rel[key] = oracle.relation(s, int(preds[i]), e, a, params)
                vals.append(rel[key])
            g = float(np.prod(vals)) ** (1.0 / len(vals)) if vals else 1.0
            top = max(top, s_sem * ((1 - params.w) + params.w * g))
        best[e] = top
    return best


@pytest.mark.parametrize("m", [0, 1, 2, 3])
def test_per_constraint_max_equals_joint_enumeration(m):
    rng = np.random.default_rng(10 + m)
    params = OracleParams(k_anchor=3)
    for trial in range(3):
        s = tiny_scene(rng, 9, 6)
        u0 = rng.standard_normal(6).astype(np.float32)
        preds = rng.integers(0, 5, size=m).astype(np.int32)
        u_c = rng.standard_normal((m, 6)).astype(np.float32)
        c_t = int(rng.integers(-1, 3))
        out = oracle.query_all(s, u0, c_t, preds, u_c, params)
        brute = _brute_force_scores(s, u0, c_t, preds, u_c, params.k_anchor, params)
        np.testing.assert_allclose(out["s"], brute, rtol=1e-12, atol=0)


# --- invariants ---------------------------------------------------------------

def test_topk_invariant_to_object_permutation():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    perm = np.random.default_rng(6).permutation(s.n)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(s.n)
    ps = Scene(desc=np.ascontiguousarray(s.desc[perm]), cls=s.cls[perm],
               box=np.ascontiguousarray(s.box[:, perm]), views=np.ascontiguousarray(s.views[:, :, perm]))
    sub = qb.subset(range(16))
    a = oracle.batch(s, sub, 10)
    b = oracle.batch(ps, sub, 10)
    np.testing.assert_array_equal(perm[b["idx"]], a["idx"])
    np.testing.assert_array_equal(b["score"], a["score"])


@pytest.mark.parametrize("with_class", [True, False])
def test_topk_lies_within_rank_bound(with_class):
    """A candidate of target rank r scores at most 1/(mu+r), while K objects
    score at least (1-w)*S_K, S_K >= cf_min/(mu+K): so every TopK member has
    rank <= (mu+K)/((1-w)*cf_min) - mu (95 for K=10 with a class, 25 without)."""
    sc, _ = synth.workload("room_n200_d512")
    s = sc[0]
    qb = synth.make_queries(77, s, 24, m_choices=(1, 2, 3, 4), with_class=with_class)
    k = 10
    cf_min = 0.3 if with_class else 1.0
    r_max = (5.0 + k) / (0.5 * cf_min) - 5.0
    for q in range(qb.n_q):
        m0, m1 = qb.c_off[q], qb.c_off[q + 1]
        out = oracle.query_all(s, qb.tgt_emb[q], qb.tgt_cls[q], qb.c_pred[m0:m1], qb.c_emb[m0:m1])
        top = oracle.topk(out["s"], k)
        assert np.all(out["rank0"][top] <= r_max + 1e-9)


def test_batch_agrees_with_single_query_path():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    sub = qb.subset(range(6))
    b = oracle.batch(s, sub, 10)
    for q in range(sub.n_q):
        m0, m1 = sub.c_off[q], sub.c_off[q + 1]
        out = oracle.query_all(s, sub.tgt_emb[q], sub.tgt_cls[q], sub.c_pred[m0:m1], sub.c_emb[m0:m1])
        top = oracle.topk(out["s"], 10)
        np.testing.assert_array_equal(b["idx"][q], top)
        np.testing.assert_array_equal(b["score"][q], out["s"][top])
        for i in range(m1 - m0):
            np.testing.assert_array_equal(b["t"][q, :, i], out["t"][i][top])
            np.testing.assert_array_equal(b["anchor"][q, :, i], out["anchor"][i][top])
        assert np.all(b["anchor"][q, :, m1 - m0:] == -1)


def test_bounds_collapse_at_zero_tolerance_and_contain_the_value():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    for q in range(4):
        m0, m1 = qb.c_off[q], qb.c_off[q + 1]
        args = (s, qb.tgt_emb[q], qb.tgt_cls[q], qb.c_pred[m0:m1], qb.c_emb[m0:m1])
        out = oracle.query_all(*args)
        b0 = oracle.query_bounds(*args, tau=0.0)
        np.testing.assert_array_equal(b0["s_lo"], out["s"])
        np.testing.assert_array_equal(b0["s_hi"], out["s"])
        b = oracle.query_bounds(*args, tau=1e-2)
        assert np.all(b["s_lo"] <= out["s"]) and np.all(out["s"] <= b["s_hi"])
        assert np.any(b["s_lo"] < b["s_hi"])


def test_batch_rejects_bad_inputs():
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    with pytest.raises(ValueError):
        oracle.batch(s, qb.subset([0]), s.n + 1)
    bad = qb.subset([0])
    bad.tgt_emb[:] = 0.0
    with pytest.raises(ValueError):
        oracle.batch(s, bad, 5)


# --- the worked example (App. C) ------------------------------------------------

@pytest.mark.parametrize("which", ["both", "left_of_only", "below_only", "none"])
def test_worked_scene_lamp_below_dartboard_left_of_poster(which):
    g = load_golden("lamp_below_dartboard_left_of_poster.json")
    sc, qb = golden_case(g, which)
    gp = g["params"]
    params = OracleParams(**gp)
    exp = g["expected"][which]
    names = [o["name"] for o in g["objects"]]
    out = oracle.batch(sc, qb, 3, params)
    assert names[out["idx"][0, 0]] == exp["top1"]
    assert out["score"][0, 0] == pytest.approx(exp["top1_score"], abs=exp["score_tol"])
    if "anchors" in exp:
        assert [names[a] for a in out["anchor"][0, 0, :2]] == exp["anchors"]
