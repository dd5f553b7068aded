"""Benchmark: relational queries/s on one GB300 for the 20,000-object site scene.

Workload (default): one 120x120x10 m scene, N = 20,000 objects, D = 1152
FP32 descriptors over 400 classes (30% in 20 look-alike classes), 8 stored
views per object; 4,096 queries with 1-4 constraints; TopK = 10.  A step is
one farm_query_batch + farm_topk over the whole batch (similarity, rank
select, relations, composite, TopK).

Prints one JSON line.  `value` times device-resident inputs with CUDA events on
the library's stream; `e2e` times the same steps through host buffers (pinned
H2D of the embeddings and query metadata, D2H of the TopK records) by wall
clock.  `roofline` reports the dominant kernel (the similarity contraction)
from the library's own stage events over the timed region.  `cpu_baseline` is
the FP64 oracle on the host cores on a bounded query sample.

--impl reference times the oracle itself, as it stands, on the host cores.
Under torchrun every rank runs its own replica (weak scaling, no collective on
the data path; one barrier and a max over ranks for the timing).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "site_n20k_d1152"
K_TOP = 10


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    nvidia-smi takes a while to start, so entering waits (at most 5 s) for its
    first line; it then samples every 5 ms, and leaving waits (at most 1 s)
    until at least one sample was taken after the region began, so that a
    region of a few tens of milliseconds still has one.  The summary uses the
    samples from the region's start on."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.n0 = 0

    def __enter__(self):
        if self.index < 0:          # not sampled
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "5"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return self
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
            time.sleep(0.005)
        self.n0 = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            t0 = time.time()
            while len(self.lines) <= self.n0 and self.proc.poll() is None and time.time() - t0 < 1.0:
                time.sleep(0.002)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.n0:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, dist=None, device=None):
    """Element-wise max of per-rank timings (ms) over the process group.

    Replicas only: ranks exchange nothing but these timings, after the timed
    region.  Without a process group the values are returned unchanged."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def rows_per_scene(scenes, qb):
    """Operand rows (targets and constraints) each scene contributes to a batch."""
    rows = np.bincount(qb.scene_of_q, minlength=len(scenes)).astype(np.int64)
    m = np.diff(qb.c_off.astype(np.int64))
    rows += np.bincount(qb.scene_of_q, weights=m, minlength=len(scenes)).astype(np.int64)
    return rows


# scenes below this many objects run FP32-accurate inside BF16 and FP8 batches
REDUCED_FROM_OBJECTS = 16384


def l2_statement(args, scenes, qb, dim, multi_ch):
    """Why no L2 flush is needed between steps: the bytes each step streams
    (tensor-core operand copies of descriptors and query rows, and the stored
    similarity columns) against the 129 MB L2."""
    rows_s = rows_per_scene(scenes, qb)
    rows = int(rows_s.sum())
    n_obj = sum(x.n for x in scenes)
    per = {"fp32": 4, "bf16": 2, "fp8": 1, "learned": 2, "fp32_simt": 4}[args.precision]
    # the learned path's operands are its 128-d BF16 embeddings
    operands = (n_obj + rows) * (128 if args.precision == "learned" else dim) * per
    fused = args.precision in ("fp32", "bf16") and (
        args.fused == "on" or (args.fused == "default" and args.precision == "fp32"))
    # the similarity block of the rows that store theirs (32-column aligned)
    stored = 0 if fused else int(sum(4 * int(r) * (-(-sc.n // 32) * 32) for r, sc in zip(rows_s, scenes)))
    if multi_ch:
        return "inputs larger than L2 (four descriptor spaces and their similarity blocks)"
    what = f"operand copies {operands / 1e6:.0f} MB"
    if stored:
        what += f", similarity block {stored / 1e6:.0f} MB written and re-read"
    elif fused:
        what += " (plus a stored sample of the similarity block)"
    return f"inputs larger than L2 ({what}; L2 129 MB)"


def job_rate(n_units_per_rank, world, ms_per_step):
    """Whole-job throughput: units all ranks processed / the slowest rank's step time."""
    return world * n_units_per_rank / (ms_per_step * 1e-3)


def cpu_baseline(scenes, qb, k, n_sample, seed=0, budget_s=15.0):
    """The oracle on a seeded query sample: its rate, and its TopK for recall.

    Queries of the seeded sample are scored in chunks of 64 until about
    budget_s seconds of wall time have passed or n_sample queries are done."""
    import oracle
    order = np.random.default_rng(seed).permutation(qb.n_q)[:min(n_sample, qb.n_q)]
    done = []
    refs = []
    t0 = time.perf_counter()
    for c0 in range(0, len(order), 64):
        chunk = np.sort(order[c0:c0 + 64])
        ref = np.zeros((len(chunk), k), np.int64)
        for sid in np.unique(qb.scene_of_q[chunk]):
            pos = np.flatnonzero(qb.scene_of_q[chunk] == sid)
            out = oracle.batch(scenes[int(sid)], qb.subset(chunk[pos]), k)
            ref[pos] = out["idx"]
        done.append(chunk)
        refs.append(ref)
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    qs = np.concatenate(done)
    return {"value": len(qs) / dt, "unit": "queries/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{len(qs)} of the {qb.n_q} queries (seeded, in chunks of 64 until about "
                      f"{budget_s:.0f} s), FP64 oracle, OpenMP over queries, {dt:.1f} s wall"}, qs, \
        np.concatenate(refs)


def cpu_baseline_mc(scene, spaces, qb, cq, k, n_sample, seed=0, budget_s=15.0):
    """The oracle of the several-channel batch on a seeded query sample (a
    thread per host core, each scoring one query at a time)."""
    import concurrent.futures as cf
    import oracle
    order = np.random.default_rng(seed).permutation(qb.n_q)[:min(n_sample, qb.n_q)]
    threads = os.cpu_count() or 1

    def one(q):
        m0, m1 = int(qb.c_off[q]), int(qb.c_off[q + 1])
        out = oracle.query_mc(scene, spaces.desc, cq.channels, [x[q] for x in cq.tgt], int(qb.tgt_cls[q]),
                              qb.c_pred[m0:m1], [x[m0:m1] for x in cq.lm])
        return oracle.topk(out["s"], k)

    done, refs = [], []
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for c0 in range(0, len(order), threads):
            chunk = order[c0:c0 + threads]
            refs.extend(ex.map(one, chunk.tolist()))
            done.extend(chunk.tolist())
            if time.perf_counter() - t0 >= budget_s:
                break
    dt = time.perf_counter() - t0
    return {"value": len(done) / dt, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(done)} of the {qb.n_q} queries (seeded, {threads} at a time until about "
                      f"{budget_s:.0f} s), FP64 oracle over {len(cq.channels)} channels, {dt:.1f} s wall"}, \
        np.asarray(done), np.asarray(refs)


# DRAM bytes of the similarity stage per step (both launches when the
# selection is fused), captured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) for the kernel source whose code digest follows
# (code_digest: the source without its comments):
# (workload, precision, tile variant, fused) -> bytes
SIM_TRAFFIC = {
    ("site_n20k_d1152", "fp32", 2, True): (90.488320e6 + 120.849664e6) + (623.171328e6 + 18.991104e6),
}
SIM_TRAFFIC_SOURCE = "02fcefe394fc0788"


def code_digest(text):
    """sha256 prefix of a CUDA source's code: comments removed and white space
    collapsed, so that an edit of the comments alone keeps a capture valid."""
    import hashlib
    code = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    code = re.sub(r"//[^\n]*", " ", code)
    code = " ".join(code.split())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def sim_traffic(workload, precision, variants, fused):
    """Captured bytes per step, or None when the run differs from the capture."""
    with open(os.path.join(ROOT, "paper_2606_15476_gb300", "csrc", "k_sim_tc.cu")) as f:
        if code_digest(f.read()) != SIM_TRAFFIC_SOURCE:
            return None
    if len(variants) != 1:
        return None
    return SIM_TRAFFIC.get((workload, precision, variants[0], fused))


def reduced_split(prec, scenes, qb):
    """Which scenes of a BF16 or FP8 batch ran that precision and which ran
    the FP32-accurate similarity (scenes below REDUCED_FROM_OBJECTS objects;
    a batch of such scenes only runs as FP32); None for the other paths."""
    if prec not in ("bf16", "fp8"):
        return None
    used = np.bincount(qb.scene_of_q, minlength=len(scenes)) > 0
    small = np.array([sc.n < REDUCED_FROM_OBJECTS for sc in scenes])
    q_small = int(np.sum(small[qb.scene_of_q]))
    return {"scenes_reduced": int(np.sum(used & ~small)), "scenes_fp32_accurate": int(np.sum(used & small)),
            "queries_reduced": int(qb.n_q - q_small), "queries_fp32_accurate": q_small,
            "rule": f"scenes under {REDUCED_FROM_OBJECTS:,} objects run the FP32-accurate similarity"}


def similarity_flops(scenes, qb):
    """2 D N per (row, object) over every scene's rows: the algorithmic work of the similarity stage."""
    rows = np.bincount(qb.scene_of_q, minlength=len(scenes)).astype(np.float64)
    m = np.diff(qb.c_off.astype(np.int64))
    rows += np.bincount(qb.scene_of_q, weights=m, minlength=len(scenes))
    return float(sum(2.0 * rows[i] * sc.n * sc.dim for i, sc in enumerate(scenes)))


PREFILTER_SCENE_BASE = 4000     # scene ids the training scenes occupy while the network trains


def prefilter_training_pairs(F, ctx, dim, seed=0, n_scenes=2, pairs=2_000_000, top=256, rand=768):
    """(descriptor, query, score) tuples from seeded scenes of the 20,000-object
    site's recipe that are NOT the memory the network is then used on: each
    training scene's relational queries give query rows (target and landmark
    embeddings), each paired with its `top` best objects by the library's
    FP32-accurate cosine (weight 4) and `rand` random ones (weight 1).  The
    scenes are uploaded under ids PREFILTER_SCENE_BASE + k."""
    import synth
    rng = np.random.default_rng(seed)
    per_row = top + rand
    rows_per_scene = -(-pairs // (per_row * n_scenes))
    rows_l, pr_l, ps_l, po_l, y_l, w_l = [], [], [], [], [], []
    row0 = 0
    for k in range(n_scenes):
        sc = synth.make_scene(7001 + 13 * k + seed, 20000, dim, extent=(120.0, 120.0, 10.0), n_classes=400,
                              n_views=2, distractor_classes=20, distractor_frac=0.30)
        sid = PREFILTER_SCENE_BASE + k
        F.farm_memory_upload(ctx, sid, sc.desc, sc.cls, sc.box, sc.views)
        qb = synth.make_queries(7101 + 13 * k + seed, sc, rows_per_scene, m_choices=(1, 2, 3, 4),
                                distractor_classes=20, distractor_target_frac=0.5)
        q_rows = np.concatenate([qb.tgt_emb, qb.c_emb])[rng.permutation(qb.n_q + qb.n_c)[:rows_per_scene]]
        for c0 in range(0, len(q_rows), 256):
            blk = q_rows[c0:c0 + 256]
            S = F.farm_similarity(ctx, sid, blk, sc.n, F.PREC_FP32)
            t = np.argpartition(-S, top, axis=1)[:, :top]
            r = rng.integers(0, sc.n, size=(len(blk), rand))
            objs = np.concatenate([t, r], axis=1)
            loc = np.repeat(np.arange(len(blk)), per_row)
            pr_l.append(row0 + c0 + loc)
            ps_l.append(np.full(loc.size, k))
            po_l.append(objs.ravel())
            y_l.append(S[loc, objs.ravel()])
            w_l.append(np.concatenate([np.full((len(blk), top), 4.0), np.ones((len(blk), rand))], axis=1).ravel())
        rows_l.append(q_rows)
        row0 += len(q_rows)
    cat = lambda xs, dt: np.concatenate(xs).astype(dt)
    return ([PREFILTER_SCENE_BASE + k for k in range(n_scenes)], np.concatenate(rows_l), cat(pr_l, np.int32),
            cat(ps_l, np.int32), cat(po_l, np.int32), cat(y_l, np.float32), cat(w_l, np.float32))


def train_prefilter(F, ctx, dim, seed=0, epochs=2, pairs=2_000_000, hidden=512, out_dim=128):
    """The learned prefilter of the configuration: a 2-layer MLP dim -> 512 ->
    128 trained by the library's BF16 tensor-core kernels on 2,000,000 tuples
    from two separate seeded scenes of the site's recipe (never on the memory
    it is evaluated on).  The training scenes are released afterwards."""
    rng = np.random.default_rng(seed)
    params = [(rng.standard_normal((hidden, dim)) / np.sqrt(dim)).astype(np.float32),
              (0.05 * rng.standard_normal(hidden)).astype(np.float32),
              (rng.standard_normal((out_dim, hidden)) / np.sqrt(hidden)).astype(np.float32),
              (0.05 * rng.standard_normal(out_dim)).astype(np.float32)]
    F.farm_mlp_set(ctx, *params)
    t0 = time.perf_counter()
    sids, rows, pr, ps, po, y, w = prefilter_training_pairs(F, ctx, dim, seed=seed, pairs=pairs)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = F.farm_mlp_train(ctx, sids, rows, pr, po, y, w, epochs=epochs, batch=4096, lr=1e-3, seed=seed + 1,
                              pair_scene=ps)
    t_train = time.perf_counter() - t0
    for sid in sids:
        F.farm_memory_release(ctx, sid)
    return {"pairs": int(len(y)), "scenes": len(sids), "epochs": epochs, "seconds": t_train,
            "data_seconds": t_data, "arithmetic": "bf16 tensor cores, fp32 master weights",
            "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1])}


def run_reference(args):
    """The oracle on the host cores: the only reference implementation there is."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.build()
    import synth
    scenes, qb = synth.workload(args.workload)
    sc = scenes[0]
    n_per_step = args.ref_queries
    rng = np.random.default_rng(1)

    def one_step(count):
        qs = np.sort(rng.choice(qb.n_q, size=count, replace=False))
        for sid in np.unique(qb.scene_of_q[qs]):
            pos = qs[qb.scene_of_q[qs] == sid]
            oracle.batch(scenes[int(sid)], qb.subset(pos), K_TOP)

    for _ in range(args.warmup):
        one_step(8)
    t0 = time.perf_counter()
    for s in range(args.steps):
        one_step(n_per_step)
    dt = time.perf_counter() - t0
    value = n_per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": "relational queries/s", "value": value, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "scenes": len(scenes),
                   "n_objects": int(sum(x.n for x in scenes)), "dim": sc.dim,
                   "queries_per_step": n_per_step, "top_k": K_TOP},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{n_per_step} seeded queries of {args.workload} per step"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


ASSOC_TAU, ASSOC_HMAX, ASSOC_MAXM = 0.8, 0.9, 8


def run_associate(args, F, synth, torch, dist, rank, world, local):
    """Mapping-side association: B detections against the site's N entities.
    A step is one farm_associate call (feature cosines, Hellinger neighbour
    search, components, fusion)."""
    scenes, _ = synth.workload("site_n20k_d1152")
    sc = scenes[0]
    B, feat = 4096, 256
    ent, det = synth.make_association(31, sc, B, feat_dim=feat, bridge_frac=0.1)
    N = sc.n
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = F.farm_create(local, stream)
    dent = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in ent.items()}
    ddet = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in det.items()}
    out = F.farm_associate(ctx, dent, ddet, ASSOC_TAU, ASSOC_HMAX, ASSOC_MAXM)

    def step():
        F.farm_associate(ctx, dent, ddet, ASSOC_TAU, ASSOC_HMAX, ASSOC_MAXM, out=out)

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks([ev0.elapsed_time(ev1) / args.steps], dist, "cuda" if dist else None)[0]
    # end to end through host arrays
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F.farm_associate(ctx, ent, det, ASSOC_TAU, ASSOC_HMAX, ASSOC_MAXM)
    e2e_ms = max_over_ranks([(time.perf_counter() - t0) * 1e3 / args.steps], dist, "cuda" if dist else None)[0]
    T = N + B
    h2d = sum(np.asarray(v).nbytes for v in ent.values()) + sum(np.asarray(v).nbytes for v in det.values())
    d2h = B * 4 + B * ASSOC_MAXM * 8 + T * 4 * (1 + 1 + 3 + 6 + feat)
    # the similarity block is written once and read once by the search; the
    # features and Gaussians are read: the step's algorithmic bytes
    bytes_step = 2.0 * B * N * 4 + (N + B) * feat * 4 * 2 + (N + B) * 10 * 4 + T * (10 + feat) * 4 * 2
    peaks, peak_kind = _peaks()
    line = {
        "metric": "detections associated/s", "value": world * B / (ms * 1e-3), "unit": "detections/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "site_n20k_assoc_b4096_f256", "entities": N, "detections": B, "feature_dim": feat,
                   "tau_f": ASSOC_TAU, "h_max": ASSOC_HMAX, "max_matches": ASSOC_MAXM,
                   "parallelism": f"replicas{world}", "l2": "the similarity block (328 MB) exceeds L2"},
        "e2e": {"value": world * B / (e2e_ms * 1e-3), "unit": "detections/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 12 * args.steps,
        "roofline": {"bound": "hbm", "achieved": bytes_step / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": bytes_step / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "whole association step", "peak_source": f"{peak_kind} HBM copy bandwidth"},
        "clocks": clk.summary(),
        "merges": int(np.sum(out["parent"].cpu().numpy()[:N] != np.arange(N))),
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sub = 64
        t0 = time.perf_counter()
        oracle.associate(ent, {k: np.ascontiguousarray(v[..., :sub] if k != "feat" else v[:sub])
                               for k, v in det.items()}, ASSOC_TAU, ASSOC_HMAX, ASSOC_MAXM)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sub / dt, "unit": "detections/s", "cores": 1, "kind": "oracle",
                                "sample": f"{sub} of the {B} detections against all {N} entities, FP64, one thread, "
                                          f"{dt:.1f} s"}
    F.farm_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_retrieval(args, F, synth, torch, dist, rank, world, local, workload, steps, extra_paths, cpu_budget_s):
    """One retrieval workload: the device-timed steps of args.precision (and
    of extra_paths, under 'paths'), their stage breakdown, roofline and
    end-to-end rate; with cpu_budget_s > 0 the oracle's rate and the
    Recall@10 of every path on a seeded query sample.  Returns the JSON line."""
    scenes, qb = synth.workload(workload)
    if args.queries > 0:
        qb = qb.subset(np.arange(min(args.queries, qb.n_q)))
    sc = scenes[0]
    PREC = {"fp32": F.PREC_FP32, "fp32_simt": F.PREC_FP32_SIMT, "bf16": F.PREC_BF16,
            "fp8": F.PREC_FP8, "learned": F.PREC_LEARNED}
    stream = torch.cuda.Stream()          # the library and the timing events share it
    torch.cuda.set_stream(stream)
    ctx = F.farm_create(local, stream)
    if args.tile_variant >= 0:
        F.farm_sim_variant_pin(ctx, args.tile_variant)
    for sid, scn in enumerate(scenes):
        F.farm_memory_upload(ctx, sid, scn.desc, scn.cls, scn.box, scn.views)
    multi_ch = args.channels == "paper"
    # the headline comparison: the reduced-precision and learned paths timed in
    # the same run on the same workload (one scene-set, one channel)
    extra = [] if (multi_ch or args.precision != "fp32") else list(extra_paths)
    training = None
    if args.precision == "learned" or "learned" in extra:
        training = train_prefilter(F, ctx, sc.dim)
    n_q, n_c = qb.n_q, qb.n_c
    if multi_ch:
        if len(scenes) != 1 or args.precision != "fp32":
            raise SystemExit("--channels paper runs one scene in FP32")
        spaces = synth.add_spaces(sc, 9001, dims=(1024, 2048))
        for s_i in range(1, len(spaces.desc)):
            F.farm_memory_add_space(ctx, 0, s_i, spaces.desc[s_i])
        cq = synth.channel_queries(9002, sc, spaces, qb)
        # the channels' embeddings laid end to end, as the call takes them
        flat_t = np.concatenate([x.ravel() for x in cq.tgt])
        flat_l = np.concatenate([x.ravel() for x in cq.lm])
        d_tgts, d_lms = torch.from_numpy(flat_t).cuda(), torch.from_numpy(flat_l).cuda()
        h_tgts = torch.from_numpy(flat_t).pin_memory().numpy()
        h_lms = torch.from_numpy(flat_l).pin_memory().numpy()
    d_tgt = torch.from_numpy(qb.tgt_emb).cuda()
    d_cemb = torch.from_numpy(qb.c_emb).cuda()
    o_idx = torch.empty((n_q, K_TOP), dtype=torch.int32, device="cuda")
    o_score = torch.empty((n_q, K_TOP), dtype=torch.float32, device="cuda")
    o_pred = torch.empty((n_q, K_TOP, 4), dtype=torch.float32, device="cuda")
    o_anc = torch.empty((n_q, K_TOP, 4), dtype=torch.int32, device="cuda")
    h_tgt = torch.from_numpy(qb.tgt_emb).pin_memory().numpy()
    h_cemb = torch.from_numpy(qb.c_emb).pin_memory().numpy()
    graph = not args.no_graph and not multi_ch
    FUSE = {"default": None, "on": True, "off": False}[args.fused]

    def timed(fn, sample_clocks):
        """K steps between CUDA events on the library's stream, barrier and synchronize on both sides."""
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local if sample_clocks else -1) as clk:
            ev0.record(stream)
            for _ in range(steps):
                fn()
            ev1.record(stream)
            torch.cuda.synchronize()
        F.farm_sync(ctx)
        return ev0.elapsed_time(ev1), clk

    def measure(prec):
        """One path: the K device-timed steps (graphs), a directly run pass with
        the stage events, and the K end-to-end steps through host buffers."""
        host_s = [0.0]

        def step_device(use_graph=graph):
            t0 = time.perf_counter()
            if multi_ch:
                h = F.farm_query_batch_rrf(ctx, 0, cq.channels, d_tgts, qb.tgt_cls, qb.c_off, qb.c_pred, d_lms)
            else:
                h = F.farm_query_batch(ctx, qb.scene_of_q, d_tgt, qb.tgt_cls, qb.c_off, qb.c_pred, d_cemb, prec,
                                       graph=use_graph, fused=FUSE)
            host_s[0] += time.perf_counter() - t0
            F.farm_topk(ctx, h, K_TOP, n_q, o_idx, o_score, o_pred, o_anc)

        for _ in range(args.warmup):
            step_device()
        F.farm_sync(ctx)
        F.farm_stage_times(ctx, reset=True)
        F.farm_select_fallbacks(ctx, reset=True)
        host_s[0] = 0.0
        ms, clk = timed(step_device, True)
        host_ms = host_s[0] * 1e3 / steps
        fallbacks = F.farm_select_fallbacks(ctx, reset=True)
        _, launches = F.farm_stage_times(ctx, reset=True)
        ms_step = max_over_ranks([ms / steps], dist, "cuda" if dist else None)[0]
        # the host's own time per call (planning, staging, graph launch), the GPU idle before each call
        plan_s = []
        for _ in range(min(steps, 20)):
            F.farm_sync(ctx)
            t0 = time.perf_counter()
            step_device()
            plan_s.append(time.perf_counter() - t0)
        F.farm_sync(ctx)
        host_plan_ms = statistics.median(plan_s) * 1e3
        # the same steps run directly with the library's stage events: the stage
        # breakdown and the similarity kernel's time for the roofline
        for _ in range(min(args.warmup, 3)):
            step_device(False)
        F.farm_sync(ctx)
        F.farm_stage_times(ctx, reset=True)
        F.farm_set_profiling(ctx, True)
        ms_prof, _ = timed(lambda: step_device(False), False)
        stage_ms, _ = F.farm_stage_times(ctx, reset=True)
        F.farm_set_profiling(ctx, False)
        if dist:
            dist.barrier()
        # ---- end to end through host buffers (pinned), same steps
        h_out = dict(idx=torch.empty((n_q, K_TOP), dtype=torch.int32).pin_memory().numpy(),
                     score=torch.empty((n_q, K_TOP), dtype=torch.float32).pin_memory().numpy(),
                     pred=torch.empty((n_q, K_TOP, 4), dtype=torch.float32).pin_memory().numpy(),
                     anchor=torch.empty((n_q, K_TOP, 4), dtype=torch.int32).pin_memory().numpy())

        def step_host(asynchronous):
            if multi_ch:
                h = F.farm_query_batch_rrf(ctx, 0, cq.channels, h_tgts, qb.tgt_cls, qb.c_off, qb.c_pred, h_lms)
            else:
                h = F.farm_query_batch(ctx, qb.scene_of_q, h_tgt, qb.tgt_cls, qb.c_off, qb.c_pred, h_cemb, prec,
                                       graph=graph, fused=FUSE)
            F.farm_topk(ctx, h, K_TOP, n_q, h_out["idx"], h_out["score"], h_out["pred"], h_out["anchor"],
                        asynchronous=asynchronous)

        # a serving loop: each step copies its rows in and its TopK records out
        # (pinned host buffers); with the asynchronous TopK (default) a step's
        # input copy overlaps the previous step's kernels, and the last
        # step's records are read after the closing farm_sync
        asynchronous = not args.e2e_sync
        for _ in range(args.warmup):
            step_host(False)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            step_host(asynchronous)
        F.farm_sync(ctx)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
        e2e_ms = max_over_ranks([e2e_ms], dist, "cuda" if dist else None)[0]
        return {"ms_step": ms_step, "clk": clk, "launches": int(launches), "stage_ms": stage_ms,
                "ms_prof": ms_prof, "e2e_ms": e2e_ms, "h_out": h_out, "host_ms": host_ms,
                "fallbacks": fallbacks / steps, "host_plan_ms": host_plan_ms}

    if multi_ch:
        h2d = flat_t.nbytes + flat_l.nbytes + 4 * (2 * n_q + 1 + n_c)
    else:
        h2d = (n_q + n_c) * sc.dim * 4 + 4 * (3 * n_q + 1 + n_c)
    d2h = n_q * K_TOP * (4 + 4 + 16 + 16)
    peaks, peak_kind = _peaks()
    flops_full = similarity_flops(scenes, qb)
    if multi_ch:
        dims = spaces.dims
        flops_full = sum(2.0 * (n_q + n_c) * sc.n * dims[sp] for sp, _ in cq.channels)

    def roofline(pname, r):
        """The similarity contraction (stage 1) over the timed steps against
        its peak: burst for a region under a second (the stage then runs at
        the maximum SM clock), sustained otherwise."""
        flops_step = flops_full * (128.0 / sc.dim if pname == "learned" else 1.0)
        gemm_ms = r["stage_ms"][1] / steps
        region_s = r["ms_step"] * steps * 1e-3
        pk_key, pk_word = ("bf16_tflops", "burst") if region_s < 1.0 else ("bf16_tflops_sustained", "sustained")
        bound, unit = "tensor", "TFLOP/s"
        if pname == "fp32":
            # three FP16 products per FP32-accurate product; FP16 dense peak = bf16 dense peak
            peak = peaks[pk_key] / 3.0
            note = f"{peak_kind} {pk_word} bf16 (= fp16 dense) / 3 (three-term FP16 split)"
        elif pname == "bf16":
            peak, note = peaks[pk_key], f"{peak_kind} {pk_word} bf16"
        elif pname == "learned":
            peak, note = peaks[pk_key], f"{peak_kind} {pk_word} bf16 (128-d learned embeddings)"
        elif pname == "fp8":
            peak = peaks[pk_key] * (4.5 / 2.25)
            note = f"{peak_kind} {pk_word} bf16 x 4.5/2.25 (FP8 dense)"
        else:
            sm_mhz = peaks.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
            bound, note = "alu", "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"
        if pname in ("bf16", "fp8") and not multi_ch:
            # scenes under REDUCED_FROM_OBJECTS objects ran FP32-accurate: the
            # peak is the one that does the batch's flops in the least time,
            # each scene's at its own arithmetic's peak
            rows_s = rows_per_scene(scenes, qb)
            f_small = sum(2.0 * int(r) * x.n * x.dim for r, x in zip(rows_s, scenes) if x.n < REDUCED_FROM_OBJECTS)
            if f_small > 0:
                t_ideal = (flops_step - f_small) / peak + f_small / (peaks[pk_key] / 3.0)
                peak = flops_step / t_ideal
                note += f"; {f_small / flops_step:.0%} of the flops FP32-accurate (peak / 3), combined"
        achieved = flops_step / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else 0.0
        return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak if peak else None,
                # the whole step against the same peak: the similarity's flops over ms_per_step
                "step_frac": flops_step / (r["ms_step"] * 1e-3) / 1e12 / peak if peak else None,
                "timed_region_s": region_s,
                "traffic": sim_traffic(workload, pname,
                                       [args.tile_variant] if args.tile_variant >= 0
                                       else sorted({d[3] for d in F.farm_sim_tuning(ctx)
                                                    if d[0] % 10 == {"fp32": 0, "fp8": 2}.get(pname, 1)}),
                                       pname in ("fp32", "bf16") and (args.fused == "on" or (
                                           args.fused == "default" and pname == "fp32"))),
                "traffic_unit": "bytes per step of the similarity stage",
                "kernel": "similarity", "peak_source": note}

    def stages(r):
        sm = r["stage_ms"]
        return {"prepare": sm[0] / steps, "similarity": sm[1] / steps, "select": sm[2] / steps,
                "compose": sm[3] / steps, "direct_ms_per_step": r["ms_prof"] / steps,
                "host_ms_per_query_batch_call": r["host_ms"],
                "host_ms_per_step_gpu_idle": r["host_plan_ms"],
                "exact_fallback_rows_per_step": r["fallbacks"]}

    main_r = measure(PREC[args.precision])
    extra_r = {x: measure(PREC[x]) for x in extra}

    line = {
        "metric": "relational queries/s", "value": job_rate(n_q, world, main_r["ms_step"]),
        "unit": "queries/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": main_r["ms_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32_simt": "f32", "bf16": "bf16", "fp8": "f8e4m3",
                  "learned": "bf16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload, "scenes": len(scenes),
                   "n_objects": int(sum(x.n for x in scenes)), "dim": sc.dim, "n_views": sc.n_views,
                   "queries": n_q, "constraint_rows": n_c, "top_k": K_TOP,
                   "precision": args.precision, "parallelism": f"replicas{world}",
                   "channels": ([{"space": sp, "dim": spaces.dims[sp], "weight": w} for sp, w in cq.channels]
                                if multi_ch else 1),
                   "cuda_graph": graph, "fused_selection": args.fused,
                   "l2": l2_statement(args, scenes, qb, sc.dim, multi_ch),
                   "reduced_precision_scenes": reduced_split(args.precision, scenes, qb)},
        "e2e": {"value": job_rate(n_q, world, main_r["e2e_ms"]), "unit": "queries/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipelined": not args.e2e_sync},
        "gpu_launches": main_r["launches"],
        "autotuned_tiles": [{"mode": d[0] % 10, "fused_selection": (d[0] // 10) % 2 == 1,
                             "with_fp32_accurate_scenes": d[0] >= 20, "log2_rows": d[1], "log2_objects": d[2],
                             "variant": d[3], "tile_n": 128 if d[3] == 1 else 256,
                             "tile_m": 256 if d[3] == 2 else 128, "cta_pair": d[3] == 2}
                            for d in F.farm_sim_tuning(ctx)],
        "pinned_tile_variant": args.tile_variant if args.tile_variant >= 0 else None,
        "stage_ms_per_step": stages(main_r),
        "roofline": roofline(args.precision, main_r),
        "clocks": main_r["clk"].summary(),
    }
    if extra_r:
        line["paths"] = {}
        for x, r in extra_r.items():
            line["paths"][x] = {
                "value": job_rate(n_q, world, r["ms_step"]), "unit": "queries/s", "ms_per_step": r["ms_step"],
                "e2e": {"value": job_rate(n_q, world, r["e2e_ms"]), "unit": "queries/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "speedup_vs_fp32": main_r["ms_step"] / r["ms_step"],
                "e2e_speedup_vs_fp32": main_r["e2e_ms"] / r["e2e_ms"],
                "gpu_launches": r["launches"], "stage_ms_per_step": stages(r),
                "roofline": roofline(x, r), "clocks": r["clk"].summary(),
                "dtype": "bf16"}
    if rank == 0 and cpu_budget_s > 0:
        import oracle
        oracle.build()
        if multi_ch:
            base, qs, ref_idx = cpu_baseline_mc(sc, spaces, qb, cq, K_TOP, args.cpu_sample, budget_s=cpu_budget_s)
        else:
            base, qs, ref_idx = cpu_baseline(scenes, qb, K_TOP, args.cpu_sample, budget_s=cpu_budget_s)
        line["cpu_baseline"] = base

        def recall(h_out):
            got = h_out["idx"][qs]
            hits = sum(len(set(got[i].tolist()) & set(ref_idx[i].tolist())) for i in range(len(qs)))
            return {"value": hits / (K_TOP * len(qs)), "queries": int(len(qs))}

        line["recall_at_10_vs_oracle"] = recall(main_r["h_out"])
        for x, r in extra_r.items():
            line["paths"][x]["recall_at_10_vs_oracle"] = recall(r["h_out"])
    if training:
        line["prefilter_training"] = training
    F.farm_destroy(ctx)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_simt", "bf16", "fp8", "learned"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-sample", type=int, default=4096,
                    help="most queries the oracle baseline scores (it stops after about 15 s)")
    ap.add_argument("--ref-queries", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile-variant", type=int, default=-1,
                    help="pin the similarity kernel's tile variant (0-2) instead of autotuning it")
    ap.add_argument("--paths", default="bf16,learned",
                    help="further paths timed in the same run of an FP32 one-channel workload and reported under "
                         "'paths' (comma list of bf16, fp8, learned; 'none' for none)")
    ap.add_argument("--prefilter-workload", default="site_n100k_d1152",
                    help="the default one-GPU run also times the FP32, BF16 and learned paths on this workload "
                         "(the learned prefilter's configuration, 100,000 objects) and reports them under "
                         "'prefilter_workload'; 'none' to skip")
    ap.add_argument("--e2e-sync", action="store_true",
                    help="end-to-end steps wait for each step's TopK records (no overlap of a step's input copy "
                         "with the previous step's kernels)")
    ap.add_argument("--fused", default="default", choices=["default", "on", "off"],
                    help="the fused rank selection: the library's default (FP32 fused, BF16 not), on (FARM_FUSED) "
                         "or off (FARM_UNFUSED)")
    ap.add_argument("--no-graph", action="store_true",
                    help="run the timed steps directly instead of as CUDA graphs (FARM_GRAPH)")
    ap.add_argument("--task", default="retrieve", choices=["retrieve", "associate"],
                    help="'associate': the mapping-side association (detections/s) of 4,096 detections "
                         "against the 20,000-object site's entities, 256-d features")
    ap.add_argument("--queries", type=int, default=0,
                    help="time only the workload's first N queries (profiling captures of a smaller case)")
    ap.add_argument("--channels", default="one", choices=["one", "paper"],
                    help="'paper': reciprocal-rank fusion over four query channels in three descriptor "
                         "spaces (the scene's, a 1,024-d and a 2,048-d one; weights 1.0 / 0.5 / 0.75 / 1.0)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist:
        dist.barrier()
    import paper_2606_15476_gb300 as F
    import synth

    if args.task == "associate":
        run_associate(args, F, synth, torch, dist, rank, world, local)
        return

    extra = [] if args.paths == "none" else [x for x in args.paths.split(",") if x]
    line = run_retrieval(args, F, synth, torch, dist, rank, world, local, args.workload, args.steps, extra,
                         0.0 if args.no_cpu_baseline else 15.0)
    if (args.prefilter_workload != "none" and args.workload == WORKLOAD and args.precision == "fp32"
            and args.channels == "one" and args.queries == 0 and args.tile_variant < 0 and world == 1):
        # the learned prefilter's own configuration (100,000 objects): the
        # learned and BF16 paths against the FP32 path, timed in the same run
        sub = run_retrieval(args, F, synth, torch, dist, rank, world, local, args.prefilter_workload,
                            min(args.steps, 10), ["bf16", "learned"], 0.0 if args.no_cpu_baseline else 6.0)
        line["prefilter_workload"] = {
            k: sub[k] for k in ("config", "value", "unit", "ms_per_step", "e2e", "stage_ms_per_step", "roofline",
                                "clocks", "paths", "recall_at_10_vs_oracle", "cpu_baseline", "prefilter_training",
                                "steps") if k in sub}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()

if __name__ == "__main__":
    main()
