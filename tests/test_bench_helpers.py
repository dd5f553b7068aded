"""The benchmark's bookkeeping (CPU): operand rows per scene, the split of a
reduced-precision batch into the scenes that run the reduced arithmetic and
those that run FP32-accurate, the statement of the bytes each step streams,
and the rule that a captured traffic figure is reported only for the kernel
source it was captured on."""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import synth  # noqa: E402


def _two_scene_batch():
    small = synth.make_scene(3, 900, 64, extent=(10.0, 10.0, 3.0), n_classes=8, n_views=2)
    large = synth.make_scene(4, 17000, 64, extent=(60.0, 60.0, 6.0), n_classes=40, n_views=2)
    parts = [synth.make_queries(13, small, 7, m_choices=(0, 1, 2), scene_id=0),
             synth.make_queries(14, large, 5, m_choices=(1, 3), scene_id=1)]
    return [small, large], synth.scenes.concat_batches(parts)


def test_rows_per_scene_counts_targets_and_constraints():
    scenes, qb = _two_scene_batch()
    rows = bench.rows_per_scene(scenes, qb)
    m = np.diff(qb.c_off)
    for sid in (0, 1):
        mine = qb.scene_of_q == sid
        assert rows[sid] == mine.sum() + m[mine].sum()
    assert rows.sum() == qb.n_q + qb.n_c


def test_reduced_split_follows_the_object_bound():
    scenes, qb = _two_scene_batch()
    assert bench.reduced_split("fp32", scenes, qb) is None
    sp = bench.reduced_split("bf16", scenes, qb)
    assert (sp["scenes_reduced"], sp["scenes_fp32_accurate"]) == (1, 1)
    assert sp["queries_reduced"] == int(np.sum(qb.scene_of_q == 1))
    assert sp["queries_fp32_accurate"] == int(np.sum(qb.scene_of_q == 0))


def test_l2_statement_counts_the_stored_similarity_columns():
    scenes, qb = _two_scene_batch()
    args = argparse.Namespace(precision="bf16", fused="default")
    rows = bench.rows_per_scene(scenes, qb)
    stored = sum(4 * int(r) * (-(-sc.n // 32) * 32) for r, sc in zip(rows, scenes))
    text = bench.l2_statement(args, scenes, qb, 64, False)
    assert f"similarity block {stored / 1e6:.0f} MB" in text
    args.precision = "fp32"
    assert "stored sample" in bench.l2_statement(args, scenes, qb, 64, False)


def test_traffic_is_reported_for_the_captured_source_only(monkeypatch):
    key = next(iter(bench.SIM_TRAFFIC))
    workload, prec, variant, fused = key
    assert bench.sim_traffic(workload, prec, [variant], fused) == bench.SIM_TRAFFIC[key]
    assert bench.sim_traffic(workload, prec, [variant, variant + 1], fused) is None     # two variants ran
    assert bench.sim_traffic(workload, prec, [variant], not fused) is None
    monkeypatch.setattr(bench, "SIM_TRAFFIC_SOURCE", "0" * 16)                         # another source
    assert bench.sim_traffic(workload, prec, [variant], fused) is None


def test_code_digest_ignores_comments_only():
    src = "// header\n__global__ void k(float *x) {\n    x[0] = 1.f;   // one\n    /* block\n comment */ x[1] = 2.f;\n}\n"
    reworded = "// another header\n__global__ void k(float *x) {\n  x[0] = 1.f;\n  /* other */ x[1] = 2.f;   // two\n}\n"
    changed = src.replace("2.f", "3.f")
    assert bench.code_digest(src) == bench.code_digest(reworded)
    assert bench.code_digest(src) != bench.code_digest(changed)
