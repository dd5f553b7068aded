"""Comparison of a TopK result (from any implementation) with the FP64 oracle.

TEST INFRASTRUCTURE.  The result under test arrives as plain numpy arrays;
everything expected comes from the oracle.

Cosines computed in FP32 may order two objects whose exact cosines differ by
less than the arithmetic error either way, and such an order changes the
object's rank-based score by a whole rank.  So for every query the oracle
gives, at tie tolerance `tau`, bounds [s_lo, s_hi] on the score each object
may take under any admissible order (oracle.query_bounds), and the check is:

  * exact part: when no object near the top has s_lo < s_hi and the oracle's
    k-th and (k+1)-th scores differ by more than rtol, the indices must equal
    the oracle's TopK and every score must be within rtol (relative);
  * otherwise (ambiguous): indices distinct, scores non-increasing, each
    returned score inside its object's [s_lo, s_hi] (widened by rtol), and no
    object left out whose lower bound beats the k-th returned score;
  * breakdown: each returned per-constraint score t_i lies in [t_lo, t_hi];
    the returned anchor is an admissible landmark candidate, not the target,
    and its relation score (evaluated by the oracle) equals t_i -- for
    Closest / Farthest, evaluated within the query's candidate set (skipped
    when that set is itself tie-ambiguous), up to near-equal distances.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import os

import numpy as np

from . import oracle as O


@dataclasses.dataclass
class ParityReport:
    n_queries: int = 0
    n_exact: int = 0
    n_ambiguous: int = 0
    max_rel_err_exact: float = 0.0
    failures: list = dataclasses.field(default_factory=list)

    def ok(self) -> bool:
        return not self.failures

    def summary(self) -> str:
        s = (f"{self.n_queries} queries: {self.n_exact} exact, {self.n_ambiguous} tie-ambiguous, "
             f"max rel err {self.max_rel_err_exact:.3g}")
        if self.failures:
            s += f"; {len(self.failures)} FAILED, first: {self.failures[0]}"
        return s


def _rank_score_range(scene, pred, e, a, cset, dtol=1e-5):
    """Closest / farthest of e to anchor a within the candidate set `cset`:
    the range of scores when squared distances within a relative dtol may be
    ordered either way (e outside the set scores 0)."""
    if e not in cset or e == a:
        return 0.0, 0.0
    c = np.asarray(scene.box[:3], np.float64).T
    d = lambda j: float(np.sum((c[j] - c[a]) ** 2))   # noqa: E731
    de = d(e)
    members = [j for j in cset if j != a]
    c_lo = sum(1 for j in members if j != e and d(j) < de * (1 - dtol))
    c_hi = sum(1 for j in members if j != e and d(j) <= de * (1 + dtol))
    r_lo, r_hi = 1 + c_lo, 1 + c_hi
    if pred == O.CLOSEST:
        return 1.0 / r_hi, 1.0 / r_lo
    return 1.0 / (len(members) - r_lo + 1), 1.0 / (len(members) - r_hi + 1)


def _check_one(scene, qb, q, k, idx, score, t, anchor, params, tau, rtol, atol_t):
    m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
    args = (scene, qb.tgt_emb[q], int(qb.tgt_cls[q]), qb.c_pred[m0:m1], qb.c_emb[m0:m1])
    b = O.query_bounds(*args, tau=tau, params=params)
    ex = O.query_all(*args, params=params)
    # the Closest / Farthest candidate set: target ranks 1..k_closest, when
    # the tie tolerance leaves it unambiguous
    kc = min(params.k_closest, scene.n)
    cset_certain = not np.any((b["rank_lo"] <= kc) & (b["rank_hi"] > kc))
    cset = set(np.flatnonzero(b["rank_hi"] <= kc).tolist()) if cset_certain else None
    return _judge(scene, qb, q, k, idx, score, t, anchor, params, rtol, atol_t, b, ex, cset)


def _topk_sets(lo, hi, K):
    """Objects certainly / possibly among the K largest when each value is
    only known to lie in [lo, hi]."""
    n = lo.shape[0]
    hs, ls = np.sort(hi), np.sort(lo)
    reach = n - np.searchsorted(hs, lo, side="left") - 1          # others with hi >= my lo
    beat = n - np.searchsorted(ls, hi, side="right")              # others with lo > my hi
    return reach < K, beat < K


def _check_one_mc(scene, spaces, qb, cq, q, k, idx, score, t, anchor, params, tau, rtol, atol_t):
    m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
    args = (scene, spaces, cq.channels, [x[q] for x in cq.tgt], int(qb.tgt_cls[q]), qb.c_pred[m0:m1],
            [x[m0:m1] for x in cq.lm])
    b = O.query_bounds_mc(*args, tau=tau, params=params)
    ex = O.query_mc(*args, params=params)
    kc = min(params.k_closest, scene.n)
    certain, possible = _topk_sets(b["F_lo"], b["F_hi"], kc)
    cset = set(np.flatnonzero(certain).tolist()) if np.array_equal(certain, possible) else None
    return _judge(scene, qb, q, k, idx, score, t, anchor, params, rtol, atol_t, b, ex, cset)


def _judge(scene, qb, q, k, idx, score, t, anchor, params, rtol, atol_t, b, ex, cset):
    fails = []
    m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
    m = m1 - m0
    s_lo, s_hi = b["s_lo"], b["s_hi"]
    n = scene.n
    idx = np.asarray(idx, np.int64)
    score = np.asarray(score, np.float64)
    if np.any(idx < 0) or np.any(idx >= n) or len(set(idx.tolist())) != k:
        return [f"q{q}: bad index list {idx.tolist()}"], False, 0.0
    if np.any(np.diff(score) > 0):
        fails.append(f"q{q}: scores not non-increasing")
    top = O.topk(ex["s"], min(k + 1, n))
    s_sorted = ex["s"][top]
    s_k = float(score[-1])
    near_top = s_hi >= s_k * (1 - 4 * rtol)
    gap_ok = k >= n or (s_sorted[k - 1] - s_sorted[k]) > rtol * s_sorted[k - 1]
    exact = gap_ok and bool(np.all(s_lo[near_top] == s_hi[near_top]))
    rel = 0.0
    if exact:
        if idx.tolist() != top[:k].tolist():
            fails.append(f"q{q}: indices {idx.tolist()} != oracle {top[:k].tolist()}")
        else:
            rel = float(np.max(np.abs(score - ex["s"][idx]) / np.maximum(ex["s"][idx], 1e-30)))
            if rel > rtol:
                fails.append(f"q{q}: score rel err {rel:.3g} > {rtol}")
    else:
        lo = s_lo[idx] * (1 - rtol)
        hi = s_hi[idx] * (1 + rtol)
        bad = np.flatnonzero((score < lo) | (score > hi))
        if bad.size:
            j = int(bad[0])
            fails.append(f"q{q}: score {score[j]:.9g} of object {idx[j]} outside "
                         f"[{s_lo[idx[j]]:.9g}, {s_hi[idx[j]]:.9g}]")
        missing = np.ones(n, bool)
        missing[idx] = False
        beat = np.flatnonzero(missing & (s_lo > s_k * (1 + rtol)))
        if beat.size:
            fails.append(f"q{q}: object {int(beat[0])} (s_lo {s_lo[beat[0]]:.9g}) missing, "
                         f"k-th returned {s_k:.9g}")
    if t is not None and anchor is not None:
        for r, e in enumerate(idx.tolist()):
            for i in range(4):
                tv, av = float(t[r][i]), int(anchor[r][i])
                if i >= m:
                    if tv != -1.0 or av != -1:
                        fails.append(f"q{q}: slot {i} beyond m={m} not empty")
                    continue
                tl, th = b["t_lo"][i][e], b["t_hi"][i][e]
                if tv < tl - atol_t or tv > th * (1 + rtol) + atol_t:
                    fails.append(f"q{q} e{e} c{i}: t {tv:.9g} outside [{tl:.9g}, {th:.9g}]")
                if av < 0:
                    if th > 0:
                        fails.append(f"q{q} e{e} c{i}: no anchor although witnesses exist")
                    continue
                if av == e or not b["in_p"][i][av]:
                    fails.append(f"q{q} e{e} c{i}: anchor {av} not an admissible landmark")
                    continue
                pred = int(qb.c_pred[m0 + i])
                if pred == O.BETWEEN_AND:
                    continue                # checked with its first landmark
                if pred == O.BETWEEN:
                    aq = int(anchor[r][i + 1])
                    if aq < 0 or aq == e or aq == av or not b["in_p"][i + 1][aq]:
                        fails.append(f"q{q} e{e} c{i}: Between pair ({av}, {aq}) not admissible")
                        continue
                    rv = O.between(scene, e, av, aq, params)
                    if abs(rv - tv) > rtol * abs(rv) + atol_t:
                        fails.append(f"q{q} e{e} c{i}: pair ({av}, {aq}) scores {rv:.9g}, reported t {tv:.9g}")
                    continue
                if pred in (O.CLOSEST, O.FARTHEST):
                    if cset is None:
                        continue            # the set itself is ambiguous: the t bounds above decide
                    rl, rh = _rank_score_range(scene, pred, e, av, cset)
                    if tv < rl * (1 - rtol) - atol_t or tv > rh * (1 + rtol) + atol_t:
                        fails.append(f"q{q} e{e} c{i}: anchor {av} scores [{rl:.9g}, {rh:.9g}], reported t {tv:.9g}")
                    continue
                rv = O.relation(scene, pred, e, av, params)
                if abs(rv - tv) > rtol * abs(rv) + atol_t:
                    fails.append(f"q{q} e{e} c{i}: anchor {av} scores {rv:.9g}, reported t {tv:.9g}")
    return fails, exact, rel


def check_topk(scene, qb, k, idx, score, t=None, anchor=None, params=None, tau=2e-5, rtol=1e-5,
               atol_t=2e-6, queries=None, threads=None) -> ParityReport:
    """Check TopK rows `queries` (default: all) of a result against the oracle."""
    params = params or O.OracleParams()
    qs = list(range(qb.n_q)) if queries is None else [int(x) for x in queries]
    rep = ParityReport(n_queries=len(qs))
    threads = threads or max(1, min(32, os.cpu_count() or 1))

    def one(q):
        return _check_one(scene, qb, q, k, idx[q], score[q], None if t is None else t[q],
                          None if anchor is None else anchor[q], params, tau, rtol, atol_t)

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for fails, exact, rel in ex.map(one, qs):
            rep.failures.extend(fails)
            if exact:
                rep.n_exact += 1
                rep.max_rel_err_exact = max(rep.max_rel_err_exact, rel)
            else:
                rep.n_ambiguous += 1
    return rep


def check_topk_mc(scene, spaces, qb, cq, k, idx, score, t=None, anchor=None, params=None, tau=2e-5, rtol=1e-5,
                  atol_t=2e-6, queries=None, threads=None) -> ParityReport:
    """check_topk for a batch over several channels: `spaces` the scene's
    descriptor spaces, `cq` the per-channel embeddings (synth.ChannelQueries)."""
    params = params or O.OracleParams()
    qs = list(range(qb.n_q)) if queries is None else [int(x) for x in queries]
    rep = ParityReport(n_queries=len(qs))
    threads = threads or max(1, min(32, os.cpu_count() or 1))

    def one(q):
        return _check_one_mc(scene, spaces, qb, cq, q, k, idx[q], score[q], None if t is None else t[q],
                             None if anchor is None else anchor[q], params, tau, rtol, atol_t)

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for fails, exact, rel in ex.map(one, qs):
            rep.failures.extend(fails)
            if exact:
                rep.n_exact += 1
                rep.max_rel_err_exact = max(rep.max_rel_err_exact, rel)
            else:
                rep.n_ambiguous += 1
    return rep


def check_candidates(scene, qb, tgt_idx, lm_idx, tau=2e-5, queries=None, params=None):
    """Rank lists against the oracle's admissible rank ranges.

    Returns a list of failure strings (empty when every listed target
    candidate at position r has rank_lo <= r+1 <= rank_hi and every landmark
    list holds exactly admissible objects)."""
    params = params or O.OracleParams()
    fails = []
    qs = range(qb.n_q) if queries is None else queries
    for q in qs:
        m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
        args = (scene, qb.tgt_emb[q], int(qb.tgt_cls[q]), qb.c_pred[m0:m1], qb.c_emb[m0:m1])
        b = O.query_bounds(*args, tau=tau, params=params)
        row = [int(x) for x in tgt_idx[q] if x >= 0]
        for r, e in enumerate(row):
            if not (b["rank_lo"][e] <= r + 1 <= b["rank_hi"][e]):
                fails.append(f"q{q}: object {e} at rank {r + 1}, admissible "
                             f"[{b['rank_lo'][e]}, {b['rank_hi'][e]}]")
                break
        for i in range(m1 - m0):
            lm = [int(x) for x in lm_idx[m0 + i] if x >= 0]
            if (len(lm) != min(params.k_anchor, scene.n) or len(set(lm)) != len(lm)
                    or not all(b["in_p"][i][a] for a in lm)):
                fails.append(f"q{q} c{i}: landmark list {lm} not admissible")
    return fails
