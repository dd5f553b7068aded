"""Pins of the oracle's further predicates (App. D.2 step 4): NextTo, On,
InFrontOf / Behind and Closest / Farthest.

Closed forms on hand-built geometry, exact identities (complements,
symmetry, the NextTo / Near scale relation), and a brute force of the whole
query over every anchor tuple in which Closest / Farthest are computed here,
independently of the C code, from their definition.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import (ABOVE, BEHIND, CLOSEST, FARTHEST, IN_FRONT_OF, NEAR, NEXT_TO, ON, OracleParams)
import synth
from scenes_util import tiny_scene
from synth import Scene

pytestmark = pytest.mark.usefixtures("oracle_lib")

P = OracleParams()
SIG = lambda x: 1.0 / (1.0 + math.exp(-x))   # noqa: E731


def boxes(centres, sizes, views_of_first=()):
    """Scene of len(centres) objects; object 0 carries the given views."""
    n = len(centres)
    box = np.zeros((6, n), np.float32)
    box[:3] = np.asarray(centres, np.float32).T
    box[3:] = np.asarray(sizes, np.float32).T
    vs = list(views_of_first)
    views = np.zeros((6, len(vs), n), np.float32)
    for v, (o, f) in enumerate(vs):
        views[:3, v, 0] = o
        views[3:, v, 0] = f
    desc = np.eye(n, max(n, 2), dtype=np.float32)
    return Scene(desc=desc, cls=np.zeros(n, np.int32), box=box, views=views)


# --- NextTo ---------------------------------------------------------------------

def test_next_to_closed_form_symmetry_and_scale():
    d = math.sqrt(2.0 * math.log(2.0)) * P.sigma_next
    sc = boxes([[1.0, 2.0, 1.0], [1.0 + d, 2.0, 1.0]], [[0.5] * 3] * 2)
    assert oracle.relation(sc, NEXT_TO, 0, 1) == pytest.approx(0.5, abs=1e-7)
    assert oracle.relation(sc, NEXT_TO, 0, 1) == oracle.relation(sc, NEXT_TO, 1, 0)
    same = boxes([[1.0, 2.0, 1.0], [1.0, 2.0, 1.0]], [[0.5] * 3] * 2)
    assert oracle.relation(same, NEXT_TO, 0, 1) == 1.0
    # sigma_next = 2 sigma_near: NextTo at distance d equals Near at d / 2
    rng = np.random.default_rng(0)
    for _ in range(20):
        p0 = rng.uniform(0, 5, 3)
        dv = rng.standard_normal(3)
        far = boxes([p0, p0 + dv], [[0.5] * 3] * 2)
        half = boxes([p0, p0 + dv / 2], [[0.5] * 3] * 2)
        assert oracle.relation(far, NEXT_TO, 0, 1) == pytest.approx(oracle.relation(half, NEAR, 0, 1), rel=1e-6)


# --- On -------------------------------------------------------------------------

def test_on_resting_on_top_is_the_gate_alone():
    # a: 1.0 x 0.6 x 0.8 box centred at z = 0.4 (top at 0.8); e: 0.2 m cube whose
    # bottom is exactly at 0.8, 0.1 m off a's centre: gap 0, rho = 0.5, d_xy = 0.1
    sc = boxes([[0.1, 0.0, 0.9], [0.0, 0.0, 0.4]], [[0.2, 0.2, 0.2], [1.0, 0.6, 0.8]])
    assert oracle.relation(sc, ON, 0, 1) == pytest.approx(SIG(0.4 / P.on_gate), abs=1e-7)


def test_on_band_half_width_and_gate_edge():
    g = math.sqrt(2.0 * math.log(2.0)) * P.on_band
    # raised by g above the top: band = 1/2; centred horizontally: gate = sig(rho / on_gate)
    sc = boxes([[0.0, 0.0, 0.9 + g], [0.0, 0.0, 0.4]], [[0.2, 0.2, 0.2], [1.0, 0.6, 0.8]])
    assert oracle.relation(sc, ON, 0, 1) == pytest.approx(0.5 * SIG(0.5 / P.on_gate), abs=1e-6)
    # at the rim (d_xy = rho) the gate is 1/2
    sc = boxes([[0.5, 0.0, 0.9], [0.0, 0.0, 0.4]], [[0.2, 0.2, 0.2], [1.0, 0.6, 0.8]])
    assert oracle.relation(sc, ON, 0, 1) == pytest.approx(0.5, abs=1e-6)
    # e below a: the band vanishes
    sc = boxes([[0.0, 0.0, -1.0], [0.0, 0.0, 0.4]], [[0.2, 0.2, 0.2], [1.0, 0.6, 0.8]])
    assert oracle.relation(sc, ON, 0, 1) < 1e-20


# --- InFrontOf / Behind ---------------------------------------------------------

SOUTH = ([5.0, 3.0, 1.0], [0.0, 1.0, 0.0])   # 2 m south of (5, 5), looking north


def test_front_behind_hand_computed_single_view():
    # e at depth 2, a at depth 2.5 in the camera of e: e is in front of a
    sc = boxes([[5.0, 5.0, 1.0], [5.0, 5.5, 1.0]], [[0.5] * 3] * 2, [SOUTH])
    assert oracle.relation(sc, IN_FRONT_OF, 0, 1) == pytest.approx(SIG(0.5 / P.tau_d), abs=1e-7)
    assert oracle.relation(sc, BEHIND, 0, 1) == pytest.approx(SIG(-0.5 / P.tau_d), abs=1e-7)


def test_front_behind_no_valid_view_is_half():
    sc = boxes([[5.0, 5.0, 1.0], [5.0, 2.0, 1.0]], [[0.5] * 3] * 2, [SOUTH])   # a behind the camera
    assert oracle.relation(sc, IN_FRONT_OF, 0, 1) == 0.5
    assert oracle.relation(sc, BEHIND, 0, 1) == 0.5
    down = ([5.0, 5.0, 3.0], [0.0, 0.0, -1.0])                                 # no horizontal image axis
    sc = boxes([[5.0, 5.0, 1.0], [5.0, 5.0, 0.0]], [[0.5] * 3] * 2, [down])
    assert oracle.relation(sc, IN_FRONT_OF, 0, 1) == 0.5


def test_front_plus_behind_is_one():
    sc, _ = synth.workload("room_n200_d512")
    rng = np.random.default_rng(4)
    for e, a in rng.integers(0, sc[0].n, size=(300, 2)):
        f = oracle.relation(sc[0], IN_FRONT_OF, e, a)
        b = oracle.relation(sc[0], BEHIND, e, a)
        assert f + b == pytest.approx(1.0, abs=1e-12)


# --- Closest / Farthest ---------------------------------------------------------

def test_closest_farthest_on_a_line():
    # a = object 0 at x = 0; set members at x = 1, 2, 3 (objects 1, 2, 3); object 4 outside the set
    xs = [0.0, 1.0, 2.0, 3.0, 0.5]
    sc = boxes([[x, 0.0, 0.0] for x in xs], [[0.2] * 3] * 5)
    cset = [0, 1, 2, 3]                       # a itself is in the set but never ranked
    assert oracle.relation_in(sc, CLOSEST, 1, 0, cset) == 1.0
    assert oracle.relation_in(sc, CLOSEST, 2, 0, cset) == 0.5
    assert oracle.relation_in(sc, CLOSEST, 3, 0, cset) == pytest.approx(1 / 3)
    assert oracle.relation_in(sc, FARTHEST, 3, 0, cset) == 1.0
    assert oracle.relation_in(sc, FARTHEST, 1, 0, cset) == pytest.approx(1 / 3)
    assert oracle.relation_in(sc, CLOSEST, 4, 0, cset) == 0.0      # not a member
    assert oracle.relation_in(sc, FARTHEST, 4, 0, cset) == 0.0


def test_closest_ties_go_to_the_lower_index():
    xs = [0.0, 1.0, -1.0]                     # objects 1 and 2 equally far from a = 0
    sc = boxes([[x, 0.0, 0.0] for x in xs], [[0.2] * 3] * 3)
    assert oracle.relation_in(sc, CLOSEST, 1, 0, [1, 2]) == 1.0
    assert oracle.relation_in(sc, CLOSEST, 2, 0, [1, 2]) == 0.5


def _python_rank_score(centres, pred, e, a, cset):
    if e not in cset or e == a:
        return 0.0
    members = [j for j in cset if j != a]
    d = lambda j: float(np.sum((centres[j] - centres[a]) ** 2))   # noqa: E731
    order = sorted(members, key=lambda j: (d(j), j))
    rank = order.index(e) + 1
    return 1.0 / rank if pred == CLOSEST else 1.0 / (len(members) - rank + 1)


def _brute_force(s, u0, c_t, preds, u_c, params):
    n = s.n
    d = s.desc.astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centres = s.box[:3].T.astype(np.float64)

    def order(u):
        u = np.asarray(u, np.float64)
        c = d @ (u / np.linalg.norm(u))
        return np.lexsort((np.arange(n), -c))

    o0 = order(u0)
    rank0 = np.empty(n, np.int64)
    rank0[o0] = np.arange(1, n + 1)
    cset = [int(j) for j in o0[:min(params.k_closest, n)]]
    cands = [list(order(u_c[i])[:min(params.k_anchor, n)]) for i in range(len(preds))]
    best = np.zeros(n)
    for e in range(n):
        cf = params.class_mis if (c_t >= 0 and s.cls[e] != c_t) else 1.0
        s_sem = cf / (params.mu + rank0[e])
        pools = [[a for a in L if a != e] for L in cands]
        if any(len(pl) == 0 for pl in pools):
            best[e] = s_sem * (1 - params.w) if preds else s_sem
            continue
        top = -1.0
        for tup in itertools.product(*pools):
            vals = []
            for i, a in enumerate(tup):
                p = int(preds[i])
                if p in (CLOSEST, FARTHEST):
                    vals.append(_python_rank_score(centres, p, e, int(a), cset))
                else:
                    vals.append(oracle.relation(s, p, e, int(a), params))
            g = float(np.prod(vals)) ** (1.0 / len(vals)) if vals else 1.0
            top = max(top, s_sem * ((1 - params.w) + params.w * g))
        best[e] = top
    return best


@pytest.mark.parametrize("m", [1, 2, 3])
def test_every_predicate_per_constraint_max_equals_joint_enumeration(m):
    rng = np.random.default_rng(40 + m)
    params = OracleParams(k_anchor=3, k_closest=5)
    for trial in range(4):
        s = tiny_scene(rng, 9, 6, n_views=3)
        u0 = rng.standard_normal(6).astype(np.float32)
        preds = rng.integers(0, 11, size=m).astype(np.int32)
        preds[trial % m] = (CLOSEST, FARTHEST, ON, IN_FRONT_OF)[trial]
        u_c = rng.standard_normal((m, 6)).astype(np.float32)
        c_t = int(rng.integers(-1, 3))
        out = oracle.query_all(s, u0, c_t, preds, u_c, params)
        brute = _brute_force(s, u0, c_t, preds, u_c, params)
        np.testing.assert_allclose(out["s"], brute, rtol=1e-12, atol=0)


@pytest.mark.parametrize("pred", [NEXT_TO, ON, IN_FRONT_OF, BEHIND, CLOSEST, FARTHEST])
def test_bounds_collapse_at_zero_tolerance_and_contain_the_value(pred):
    sc, qb = synth.workload("room_n200_d512")
    s = sc[0]
    rng = np.random.default_rng(pred)
    for q in range(4):
        preds = np.array([pred, ABOVE], np.int32)
        u_c = qb.c_emb[2 * q:2 * q + 2]
        ex = oracle.query_all(s, qb.tgt_emb[q], int(qb.tgt_cls[q]), preds, u_c)
        b0 = oracle.query_bounds(s, qb.tgt_emb[q], int(qb.tgt_cls[q]), preds, u_c, tau=0.0)
        np.testing.assert_allclose(b0["s_lo"], ex["s"], rtol=1e-12)
        np.testing.assert_allclose(b0["s_hi"], ex["s"], rtol=1e-12)
        b = oracle.query_bounds(s, qb.tgt_emb[q], int(qb.tgt_cls[q]), preds, u_c, tau=2e-5)
        assert np.all(b["s_lo"] <= ex["s"] * (1 + 1e-12)) and np.all(ex["s"] <= b["s_hi"] * (1 + 1e-12))
    del rng


# --- Near, Hellinger form (Sec. 2.3) -------------------------------------------

def _bc_by_quadrature(c0, s0, c1, s1):
    """Bhattacharyya coefficient of the two box-moment Gaussians, integrated
    numerically axis by axis (the densities factorise over the axes)."""
    from scipy import integrate
    bc = 1.0
    for k in range(3):
        v0, v1 = s0[k] ** 2 / 12.0, s1[k] ** 2 / 12.0
        g0 = lambda x, m=c0[k], v=v0: math.exp(-(x - m) ** 2 / (2 * v)) / math.sqrt(2 * math.pi * v)  # noqa: E731
        g1 = lambda x, m=c1[k], v=v1: math.exp(-(x - m) ** 2 / (2 * v)) / math.sqrt(2 * math.pi * v)  # noqa: E731
        lo = min(c0[k], c1[k]) - 12 * max(s0[k], s1[k])
        hi = max(c0[k], c1[k]) + 12 * max(s0[k], s1[k])
        val, _ = integrate.quad(lambda x: math.sqrt(g0(x) * g1(x)), lo, hi, points=[c0[k], c1[k]],
                                limit=200, epsabs=1e-13, epsrel=1e-11)
        bc *= val
    return bc


def test_near_h_matches_the_integral_of_the_densities():
    from oracle import NEAR_H
    pytest.importorskip("scipy")
    rng = np.random.default_rng(7)
    for _ in range(12):
        c0, c1 = rng.uniform(0, 2, 3), rng.uniform(0, 2, 3)
        s0, s1 = rng.lognormal(-1, 0.5, 3), rng.lognormal(-1, 0.5, 3)
        sc = boxes([c0, c1], [s0, s1])
        # the scene stores float32 geometry: integrate the stored values
        bc = _bc_by_quadrature(sc.box[:3, 0].astype(np.float64), sc.box[3:, 0].astype(np.float64),
                               sc.box[:3, 1].astype(np.float64), sc.box[3:, 1].astype(np.float64))
        want = 1.0 - math.sqrt(max(0.0, 1.0 - bc))
        assert oracle.relation(sc, NEAR_H, 0, 1) == pytest.approx(want, abs=1e-7)


def test_near_h_identities():
    from oracle import NEAR_H
    # identical Gaussians: H = 0
    same = boxes([[1.0, 2.0, 0.5], [1.0, 2.0, 0.5]], [[0.4, 0.3, 0.8]] * 2)
    assert oracle.relation(same, NEAR_H, 0, 1) == 1.0
    # equal boxes offset by d along x: BC = exp(-d^2 / (8 var)), var = s^2 / 12
    s, d = 0.6, 0.25
    sc = boxes([[0.0, 0.0, 0.0], [d, 0.0, 0.0]], [[s, s, s]] * 2)
    bc = math.exp(-d * d / (8.0 * s * s / 12.0))
    assert oracle.relation(sc, NEAR_H, 0, 1) == pytest.approx(1.0 - math.sqrt(1.0 - bc), abs=1e-7)
    # concentric boxes differing in one size only: BC = sqrt(2 s0 s1 / (s0^2 + s1^2))
    sc = boxes([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]], [[0.5, 0.5, 0.5], [0.5, 0.5, 2.0]])
    bc = math.sqrt(2 * 0.5 * 2.0 / (0.25 + 4.0))
    assert oracle.relation(sc, NEAR_H, 0, 1) == pytest.approx(1.0 - math.sqrt(1.0 - bc), abs=1e-7)
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.uniform(0, 3, (2, 3))
        sz = rng.lognormal(-1, 0.5, (2, 3))
        sc = boxes(c, sz)
        r01, r10 = oracle.relation(sc, NEAR_H, 0, 1), oracle.relation(sc, NEAR_H, 1, 0)
        assert r01 == r10                       # symmetric, bit for bit
        assert 0.0 <= r01 <= 1.0
    # moving one box away never raises the score
    vals = [oracle.relation(boxes([[0, 0, 0], [x, 0.2, 0]], [[0.4, 0.4, 0.4], [0.5, 0.3, 0.6]]), NEAR_H, 0, 1)
            for x in np.linspace(0.0, 3.0, 31)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))


def test_near_h_degenerate_axes():
    from oracle import NEAR_H
    # two flat boxes (zero height) at the same height: that axis contributes 1
    flat = boxes([[0.0, 0.0, 1.0], [0.3, 0.0, 1.0]], [[0.5, 0.5, 0.0], [0.5, 0.5, 0.0]])
    bc = math.exp(-0.09 / (8.0 * 0.25 / 12.0))
    assert oracle.relation(flat, NEAR_H, 0, 1) == pytest.approx(1.0 - math.sqrt(1.0 - bc), abs=1e-7)
    # ... at different heights: BC = 0
    apart = boxes([[0.0, 0.0, 1.0], [0.0, 0.0, 1.5]], [[0.5, 0.5, 0.0], [0.5, 0.5, 0.0]])
    assert oracle.relation(apart, NEAR_H, 0, 1) == 0.0
    # zero extent against positive extent on one axis: BC = 0
    mixed = boxes([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]], [[0.5, 0.5, 0.0], [0.5, 0.5, 0.4]])
    assert oracle.relation(mixed, NEAR_H, 0, 1) == 0.0


# --- Inside (App. D.2 step 4, containment) ---------------------------------------

def test_inside_closed_forms():
    from oracle import INSIDE
    big = [2.0, 2.0, 2.0]
    # fully inside, touching the walls, fully outside
    assert oracle.relation(boxes([[0.1, -0.2, 0.3], [0, 0, 0]], [[0.5, 0.5, 0.5], big]), INSIDE, 0, 1) == 1.0
    assert oracle.relation(boxes([[0.75, 0, 0], [0, 0, 0]], [[0.5, 0.5, 0.5], big]), INSIDE, 0, 1) == 1.0
    assert oracle.relation(boxes([[3.0, 0, 0], [0, 0, 0]], [[0.5, 0.5, 0.5], big]), INSIDE, 0, 1) == 0.0
    # half out along x, a quarter out along y: 0.5 * 0.75
    sc = boxes([[1.0, 0.875, 0.0], [0, 0, 0]], [[0.5, 0.5, 0.5], big])
    assert oracle.relation(sc, INSIDE, 0, 1) == pytest.approx(0.5 * 0.75, abs=1e-7)
    # not symmetric: the big box is mostly outside the small one
    sc = boxes([[0, 0, 0], [0, 0, 0]], [big, [0.5, 0.5, 0.5]])
    assert oracle.relation(sc, INSIDE, 0, 1) == pytest.approx(0.25 ** 3, abs=1e-9)
    # a point (zero size) inside / outside
    assert oracle.relation(boxes([[0.2, 0.2, 0.2], [0, 0, 0]], [[0, 0, 0], big]), INSIDE, 0, 1) == 1.0
    assert oracle.relation(boxes([[1.2, 0.2, 0.2], [0, 0, 0]], [[0, 0, 0], big]), INSIDE, 0, 1) == 0.0


def test_inside_is_the_volume_fraction_on_a_grid():
    from oracle import INSIDE
    rng = np.random.default_rng(11)
    g = (np.arange(40) + 0.5) / 40.0 - 0.5          # cell centres of a 40^3 grid over a unit box
    for _ in range(10):
        c = rng.uniform(0, 1, (2, 3))
        sz = rng.uniform(0.2, 1.0, (2, 3))
        sc = boxes(c, sz)
        ce, se = sc.box[:3, 0].astype(np.float64), sc.box[3:, 0].astype(np.float64)
        ca, sa = sc.box[:3, 1].astype(np.float64), sc.box[3:, 1].astype(np.float64)
        frac = 1.0
        for k in range(3):
            x = ce[k] + g * se[k]
            frac *= np.mean(np.abs(x - ca[k]) <= sa[k] / 2)
        # the midpoint rule over 40 cells per axis is within 1/40 per axis
        assert oracle.relation(sc, INSIDE, 0, 1) == pytest.approx(frac, abs=3 * 1.0 / 40 + 1e-9)
