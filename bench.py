#!/usr/bin/env python3
"""FGraft build benchmark on one GB300 (or N replicas under torchrun).

One step is one pass of the whole hot path over the paper-scale angular
workload (n = 1,183,514 unit vectors, d = 100, 256 vMF-like clusters with
Zipf(1.1) sizes): SAT scaffold (T = 8), the B = 8 harvest blocks (R = 64,
ef_h = 100; one CUDA graph), the final graph, a 10,000-query search
(ef_s = 64, top-10) and 64 dense 1024-point intra-cluster blocks (top-64 per
row, BF16 tensor-core filter with float32 rerank).  The headline value is
points built per second over the whole step; L2 is flushed (a 256 MiB
write) before every timed step, whose duration is taken with CUDA events on
the launching stream.  The in-cache workload (n = 100,000, 40 MB of vectors,
L2-resident) is measured after it as a labelled extra.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the
plain C restatement of the method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FGraft build pts/s & dist-evals/s vs dense-block ceiling, 1 GB300; recall@10"
WORKLOAD = "paper-angular-n1183514-d100"
SPEC = dict(workload=WORKLOAD, n=1_183_514, d=100, k=256, sizes="zipf", kappa=20.0, T=8, B=8,
            R=64, ef_h=100, alpha=1.2, nq=10_000, ef_s=64, topk=10, dense_blocks=64,
            block_size=1024, dense_k=64, seed=0)
INCACHE = dict(workload="incache-angular-n100k-d100", n=100_000, d=100, k=64, sizes="equal",
               kappa=20.0, T=8, B=8, R=32, ef_h=64, alpha=1.2, nq=10_000, ef_s=64, topk=10,
               dense_blocks=64, block_size=1024, dense_k=32, seed=0)
CPU_SAMPLE_N = 20_000
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dims", action="store_true", help="skip the dimension sweep extra")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip every extra after the headline (paper arms, dimension sweep, "
                         "in-cache run): for profiling the step alone")
    ap.add_argument("--tune-table", default=None,
                    help="autotuner table (JSON): loaded when the file exists, otherwise "
                         "written after tuning (a profiled run then reuses the settings of "
                         "the plain run instead of tuning under the profiler)")
    ap.add_argument("--n", type=int, default=None, help="override n (smaller runs)")
    ap.add_argument("--batch", type=int, default=64, help="builds of --mode batched")
    ap.add_argument("--arms", default="32x1,8x1,8x2,8x4,8x8,8x16",
                    help="--mode paper: the TxB arms to build")
    ap.add_argument("--tunes", default="0x0",
                    help="--mode paper: harvest launch settings to try per arm, "
                         "hash_log2 x warps per CTA (0 keeps the default)")
    ap.add_argument("--dims", default="32,64,128,256,512,960,128u8",
                    help="--mode dims: dimensions (suffix u8 for byte vectors)")
    ap.add_argument("--no-ladder", action="store_true", help="--mode paper: skip recall")
    ap.add_argument("--schedule", default="auto", choices=["auto", "coherent", "id"],
                    help="order in which each block's searches are claimed: tree-0 preorder "
                         "(coherent), point id, or the preorder when X exceeds L2 (auto)")
    ap.add_argument("--mode", default="step",
                    choices=["step", "dims", "paper", "batched", "cap", "dense", "lockstep", "tc"],
                    help="step: the benchmark line; dims: adaptive vs dense cost per evaluation "
                         "across d; paper: the paper-scale angular arms; batched: many "
                         "independent builds harvested together; cap: the scaffold degree "
                         "cap ablation; dense: the dense-block ceiling alone; lockstep: the "
                         "visited-set overlap of the GPU harvest (Section 5.5); tc: the two "
                         "tensor-core Gram kernels alone (Gram-only dense blocks, exact k-NN), "
                         "for profiling")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def make_inputs(spec):
    from paper_2609_30493_gb300 import synth
    ps = synth.vmf_like(spec["n"], spec["d"], spec["k"], spec["seed"], spec["kappa"],
                        sizes=spec["sizes"])
    Q = synth.queries(ps, spec["nq"], spec["seed"] + 1)
    blocks = synth.intra_cluster_blocks(ps.labels, spec["dense_blocks"], spec["block_size"],
                                        spec["seed"] + 2)
    return ps, Q, blocks


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the harvest search kernel's source: the kernel and the distance and merge code it uses
BEAM_SOURCES = [os.path.join(ROOT, "paper_2609_30493_gb300", "csrc", f)
                for f in ("beam.cuh", "common.cuh", "beam_ang.cu")]


def kernel_source_sha256(files):
    """One hash over the kernel's source files, in the order given."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def ncu_traffic(kernel_files, profile="harvest_beam_paper_n1183514_d100.md"):
    """DRAM bytes per harvest launch from the committed ncu summary, if it was
    taken on the current kernel source (hash match), else None."""
    prof = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(prof):
        return None
    txt = open(prof).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256[^:\n]*:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    return float(m.group(1)) if h.group(1) == kernel_source_sha256(kernel_files) else None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, idx: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={idx}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def recall_at_10(X, Q, ids):
    """Recall of ids (nq x 10) against a float32 brute force on the device
    (measurement only)."""
    import torch
    Xt = torch.from_numpy(X).cuda()
    hits = 0
    for s in range(0, Q.shape[0], 1024):
        q = torch.from_numpy(Q[s:s + 1024]).cuda()
        dots = q @ Xt.T
        gt = torch.topk(dots, 10, dim=1).indices.cpu().numpy()
        got = ids[s:s + 1024]
        hits += sum(len(set(a.tolist()) & set(b.tolist())) for a, b in zip(gt, got))
    return hits / (Q.shape[0] * 10)


def job_rate(local_ms, steps, n_per_rank, world, dist_mod, device):
    """Whole-job rate of a replicated run: the slowest rank's time decides
    (max over ranks), every rank built n_per_rank points per step.  Returns
    (ms per step, points per second over all ranks)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if dist_mod is not None:
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    ms = float(t.item()) / steps
    return ms, world * n_per_rank / (ms / 1e3)


EF_LADDER = (10, 16, 24, 32, 48, 64, 96, 128)


def quality_report(fg, ix, ps, Q_d, spec, r_target=0.95):
    """Measurement only (outside the timed region): recall@10 and evaluations
    per query along the ef_s ladder, d@r (the evaluations per query of the
    first ef_s reaching recall r), with the queries' ground truth from a
    float32 PyTorch product; and local completeness (the fraction of a
    point's 10 nearest neighbours that sit in its final adjacency row) over
    every point, the neighbours from fgraft_knn_exact."""
    import torch
    X = torch.from_numpy(ps.X[:, :spec["d"]]).cuda()
    Q = Q_d[:, :spec["d"]]
    gtq = []
    for s in range(0, Q.shape[0], 1024):
        gtq.append(torch.topk(Q[s:s + 1024] @ X.T, 10, dim=1).indices)
    gtq = torch.cat(gtq)
    ladder = []
    d_at_r = None
    for ef in EF_LADDER:
        ids, _, ev = fg.fgraft_search(ix, Q_d, 10, ef)
        hit = (ids.long().unsqueeze(2) == gtq.unsqueeze(1)).any(dim=2).sum().item()
        rec = hit / (Q.shape[0] * 10)
        epq = float(ev.double().mean().item())
        ladder.append({"ef_s": ef, "recall_at_10": round(rec, 4), "evals_per_query": round(epq, 1)})
        if d_at_r is None and rec >= r_target:
            d_at_r = round(epq, 1)
    n = X.shape[0]
    off, fids = fg.fgraft_prune(ix)
    rows = torch.repeat_interleave(torch.arange(n, device=X.device), off[1:] - off[:-1])
    edge_keys = torch.sort(rows * n + fids.long()).values
    # the exact 10-NN of every point with the library's own kernel (BF16
    # tensor-core filter, canonical float32 rerank)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    kid, _, kst = fg.fgraft_knn_exact(ix.X, spec["d"], ps.metric, 10, stats=True)
    e1.record()
    torch.cuda.synchronize()
    keys = (torch.arange(n, device=X.device).unsqueeze(1) * n + kid.long()).reshape(-1)
    pos = torch.searchsorted(edge_keys, keys).clamp(max=edge_keys.numel() - 1)
    hits = int(((edge_keys[pos] == keys) & (kid.reshape(-1) >= 0)).sum().item())
    # cross-check of a sample against a float32 PyTorch product (equal up to
    # rounding ties of the two summation orders)
    pts = torch.from_numpy(np.random.default_rng(17).choice(n, size=min(n, 1000),
                                                             replace=False)).cuda()
    agree = 0
    for c0 in range(0, len(pts), 100):
        pc = pts[c0:c0 + 100]
        sc = X[pc] @ X.T if ps.metric == 1 else -(torch.cdist(X[pc], X) ** 2)
        sc[torch.arange(len(pc), device=X.device), pc] = -float("inf")
        tt = torch.topk(sc, 10, dim=1).indices
        agree += int((torch.sort(tt, dim=1).values == torch.sort(kid[pc].long(), dim=1).values)
                     .all(dim=1).sum().item())
        del sc
    same = agree / len(pts)
    out = {"recall_ladder": ladder, f"d_at_r{r_target}": d_at_r,
           "local_completeness_at_10": round(hits / (n * 10), 4),
           "exact_knn": {"points": n, "k": 10, "ms": round(e0.elapsed_time(e1), 2),
                         "filter_ms": round(kst["filter_ms"], 2),
                         "rerank_ms": round(kst["rerank_ms"], 2),
                         "rerank_evals_per_point": round(kst["rerank_evals"] / n, 1),
                         "full_scan_rows": int(kst["full_scan_rows"]),
                         "sample_rows_equal_to_torch_fp32": round(same, 4)}}
    return out


def _device_inputs(spec):
    import torch
    ps, Q, blocks = make_inputs(spec)
    return ps, Q, blocks, (torch.from_numpy(ps.X).cuda(), torch.from_numpy(Q).cuda(),
                           torch.from_numpy(blocks).cuda())


def _params(fg, spec):
    return fg.Params(T=spec["T"], R=spec["R"], ef_h=spec["ef_h"], B=spec["B"],
                     alpha=spec["alpha"], seed=spec["seed"], metric=fg.ANGULAR_F32)


def _step(fg, spec, params, X_t, Q_t, B_t, profile=False):
    """One pass of the whole hot path: scaffold, the B harvest blocks (one CUDA
    graph), final graph, query search, dense blocks (BF16 filter)."""
    ix = fg.fgraft_build_scaffold(X_t, spec["d"], params)
    if profile:
        fg.fgraft_index_profile(ix, True)
    fg.fgraft_harvest_all(ix, use_graph=True)
    ids, _, _ = fg.fgraft_search(ix, Q_t, spec["topk"], spec["ef_s"])
    di, _ = fg.fgraft_dense_block_dist(X_t, spec["d"], fg.ANGULAR_F32, B_t, spec["dense_k"],
                                       precision=1)
    return ix, ids, di


def _timed(fg, spec, params, dev_in, steps, warmup, flush, stream):
    """Warm-up steps, then `steps` timed steps (L2 flushed before each).  Returns
    (total ms, summed harvest-kernel ms, harvest launches, prune ms, summed
    counters, kernels launched, last step's outputs)."""
    import torch
    for _ in range(warmup):
        _step(fg, spec, params, *dev_in)
    torch.cuda.synchronize()
    launches0 = fg.fgraft_kernel_launches()
    total_ms, harvest_ms, harvest_launches, prune_ms = 0.0, 0.0, 0, 0.0
    ctr_sum, last = {}, None
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("timed")  # lets a profiler keep to the timed steps
        ix, ids, di = _step(fg, spec, params, *dev_in, profile=True)
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        hm, hl, pm = fg.fgraft_index_harvest_ms(ix, with_prune=True)
        harvest_ms += hm
        harvest_launches += hl
        prune_ms += pm
        for k_, v_ in fg.fgraft_index_counters(ix).items():
            ctr_sum[k_] = ctr_sum.get(k_, 0) + v_
        last = (ix, ids, di)
    launches = fg.fgraft_kernel_launches() - launches0
    return total_ms, harvest_ms, harvest_launches, prune_ms, ctr_sum, launches, last


def _alg_bytes(spec, ctr):
    """Algorithmic bytes of the harvest: one dependent vector gather at 32-byte
    sectors per evaluation plus 4 bytes per neighbour id scanned."""
    line = 32 * ((4 * spec["d"] + 31) // 32)
    return ctr.get("harvest_evals", 0) * line + ctr.get("ids_scanned", 0) * 4


def tune(fg, X_d, spec, params, sample, table=None):
    """The autotuner's harvest settings for this shape (kept in the process's
    table for every later build).  With a table file that exists, its
    settings are loaded instead; a table file that does not exist yet is
    written after tuning."""
    if table and os.path.exists(table):
        fg.fgraft_tuning_table_load(table)
        return {"loaded_from": os.path.basename(table)}
    ixt = fg.fgraft_build_scaffold(X_d, spec["d"], params)
    # calibrate on a middle block: later blocks scan longer neighbour lists
    for b in range(spec["B"] // 2):
        fg.fgraft_harvest_block(ixt, b)
    t = fg.fgraft_index_autotune(ixt, sample=sample)
    del ixt
    if table:
        fg.fgraft_tuning_table_save(table)
    return t


def incache_extra(fg, flush, stream, steps=3, warmup=2, tune_table=None):
    """The in-cache workload (40 MB of vectors, L2-resident): bound by the
    latency of the dependent gathers, not by HBM.  Reports the step rate, the
    harvest's evaluations per second, its algorithmic gather rate and the SM
    cycles per evaluation (the GB300's c_adapt, Section 5.3)."""
    import torch
    spec = INCACHE
    ps, Q, blocks, dev_in = _device_inputs(spec)
    params = _params(fg, spec)
    tuning = tune(fg, dev_in[0], spec, params, 4096, tune_table)
    clocks = Clocks(torch.cuda.current_device())
    tot, hms, hl, pms, ctr, _, _ = _timed(fg, spec, params, dev_in, steps, warmup, flush, stream)
    clk = clocks.stop()
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    evals = ctr.get("harvest_evals", 0)
    alg = _alg_bytes(spec, ctr)
    return {"workload": spec["workload"], "bound": "L2-resident; latency of the dependent gathers",
            "value": round(spec["n"] * steps / (tot / 1e3), 1), "unit": "pts/s",
            "ms_per_step": round(tot / steps, 3),
            "harvest_evals_per_s": round(evals / (hms / 1e3), 1) if hms else None,
            "harvest_alg_GBps": round(alg / (hms / 1e3) / 1e9, 1) if hms else None,
            "harvest_ms_per_block": round(hms / max(hl, 1), 4),
            "prune_ms_per_block": round(pms / max(hl, 1), 4),
            "sm_cycles_per_eval": round(hms / 1e3 * mhz * 1e6 * nsm / evals, 1) if evals else None,
            "sm_mhz": mhz,
            "autotune": {k_: (round(v_, 4) if isinstance(v_, float) else v_)
                         for k_, v_ in tuning.items()},
            "config": {k: spec[k] for k in ("n", "d", "k", "T", "B", "R", "ef_h", "alpha")}}


def paper_arms(fg, X_d, Q_d, ps, Q, spec, arms=((32, 1), (8, 1), (8, 2), (8, 4), (8, 8), (8, 16))):
    """The paper's Table 1 shape on the benchmark workload (untimed extra): the
    frozen T = 32 harvest and FGraft T = 8 at B = 1..16, R = 64, ef_h = 100;
    build time (scaffold, harvest, final graph; each arm autotuned first),
    harvest evaluations per second and recall@10 at ef_s = 64 and 128
    (float32 brute force)."""
    import torch
    d = spec["d"]
    gt = []
    for s0 in range(0, Q_d.shape[0], 1024):
        gt.append(torch.topk(Q_d[s0:s0 + 1024, :d] @ X_d[:, :d].T, 10, dim=1).indices)
    gt = torch.cat(gt)
    out = []
    for T, B in arms:
        p = fg.Params(T=T, R=spec["R"], ef_h=spec["ef_h"], B=B, alpha=spec["alpha"],
                      seed=spec["seed"], metric=fg.ANGULAR_F32)
        # each arm's own launch settings (the tuning table is keyed by T and B)
        tune(fg, X_d, dict(spec, T=T, B=B), p, 32768)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ix = fg.fgraft_build_scaffold(X_d, d, p)
        fg.fgraft_index_profile(ix, True)
        fg.fgraft_harvest_all(ix, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        hms, _ = fg.fgraft_index_harvest_ms(ix)
        c = fg.fgraft_index_counters(ix)
        rec = {}
        for ef in (64, 128):
            ids, _, ev = fg.fgraft_search(ix, Q_d, 10, ef)
            hit = (ids.long().unsqueeze(2) == gt.unsqueeze(1)).any(dim=2).sum().item()
            rec[f"recall_at_10_ef{ef}"] = round(hit / (Q_d.shape[0] * 10), 4)
            rec[f"evals_per_query_ef{ef}"] = round(float(ev.double().mean().item()), 1)
        ms = e0.elapsed_time(e1)
        out.append({"T": T, "B": B, "build_ms": round(ms, 1),
                    "pts_per_s": round(spec["n"] / (ms / 1e3), 1),
                    "harvest_evals": c["harvest_evals"],
                    "harvest_evals_per_s": round(c["harvest_evals"] / (hms / 1e3), 1), **rec})
        del ix
    return out


def dims_sweep(fg, dims=(32, 64, 128, 256, 512, 960), n=1_000_000):
    """Adaptive vs blocked cost per evaluation across d (Section 5.4, Table 5),
    untimed extra: Gaussian mixtures of 128 clusters (centres N(0, 25 I), unit
    noise, generated on the device), L2, T = 8, B = 8, R = 32, ef_h = 64; the
    harvest's evaluations per second and SM cycles per evaluation against the
    dense blocks' pairs per second (64 intra-cluster blocks of 1024, BF16
    filter with float32 rerank, and the raw Gram), and the fitted exponents."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    for d in dims:
        g = torch.Generator(device="cuda")
        g.manual_seed(d)
        lab = torch.randint(0, 128, (n,), generator=g, device="cuda")
        cent = 5.0 * torch.randn(128, d, generator=g, device="cuda")
        ld = (d + 3) // 4 * 4
        X = torch.zeros(n, ld, device="cuda")
        X[:, :d] = cent[lab] + torch.randn(n, d, generator=g, device="cuda")
        del cent
        p = fg.Params(T=8, R=32, ef_h=64, B=8, alpha=1.2, seed=0, metric=fg.L2_F32)
        ix = fg.fgraft_build_scaffold(X, d, p)
        fg.fgraft_index_profile(ix, True)
        fg.fgraft_harvest_all(ix, use_graph=False)
        hms, _ = fg.fgraft_index_harvest_ms(ix)
        c = fg.fgraft_index_counters(ix)
        del ix
        labn = lab.cpu().numpy()
        blocks = []
        rng = np.random.default_rng(d)
        for cl in rng.permutation(128):
            members = np.nonzero(labn == cl)[0]
            if len(members) >= 1024:
                blocks.append(np.sort(rng.choice(members, 1024, replace=False)))
            if len(blocks) == 64:
                break
        Bd = torch.from_numpy(np.stack(blocks).astype(np.int32)).cuda()
        pairs = len(blocks) * 1024 * 1023
        fg.fgraft_dense_block_dist(X, d, fg.L2_F32, Bd, 32, precision=1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fg.fgraft_dense_block_dist(X, d, fg.L2_F32, Bd, 32, precision=1)
        e1.record()
        torch.cuda.synchronize()
        dense = pairs / (e0.elapsed_time(e1) / 1e3)
        _, gms = fg.fgraft_dense_block_gram(X, d, fg.L2_F32, Bd, precision=1)
        gram = pairs / (gms / 1e3)
        rate = c["harvest_evals"] / (hms / 1e3)
        mhz = _sm_clock_mhz() or 2070.0
        rows.append({"d": d, "harvest_evals_per_s": round(rate, 1),
                     "sm_cycles_per_eval": round(hms / 1e3 * mhz * 1e6 * nsm / c["harvest_evals"], 1),
                     "harvest_alg_GBps": round(rate * 32 * ((4 * d + 31) // 32) / 1e9, 1),
                     "dense_pairs_per_s": round(dense, 1), "gram_pairs_per_s": round(gram, 1),
                     "gap_W": round(dense / rate, 2), "gap_W_gram": round(gram / rate, 2)})
        del X, Bd
        torch.cuda.empty_cache()
    ld = np.log([r["d"] for r in rows])
    fit = {"adaptive_cost_exponent": round(float(np.polyfit(ld, np.log([1 / r["harvest_evals_per_s"] for r in rows]), 1)[0]), 3),
           "dense_cost_exponent": round(float(np.polyfit(ld, np.log([1 / r["dense_pairs_per_s"] for r in rows]), 1)[0]), 3),
           "gram_cost_exponent": round(float(np.polyfit(ld, np.log([1 / r["gram_pairs_per_s"] for r in rows]), 1)[0]), 3)}
    fit["gap_exponent"] = round(fit["adaptive_cost_exponent"] - fit["dense_cost_exponent"], 3)
    return {"n": n, "rows": rows, "fit": fit,
            "data": "Gaussian mixture generated on the device (torch generator per d)"}


def _subtree_groups(par, max_size):
    """Maximal subtrees of at most max_size points of the tree with parent
    array par: (roots, labels, sizes), labels[v] = the root of v's maximal
    subtree (-1 for points in no such subtree), sizes[v] = |subtree(v)|."""
    par = np.asarray(par, np.int64)
    depth = (par >= 0).astype(np.int64)
    anc = par.copy()
    while True:  # pointer jumping: depth[v] = edges from v to anc[v]
        m = anc >= 0
        if not m.any():
            break
        a = anc[m]
        nd, na = depth.copy(), anc.copy()
        nd[m] = depth[m] + depth[a]
        na[m] = anc[a]
        depth, anc = nd, na
    size = np.ones(len(par), np.int64)
    levels = [np.flatnonzero(depth == dd) for dd in range(int(depth.max()) + 1)]
    for nodes in reversed(levels[1:]):
        np.add.at(size, par[nodes], size[nodes])
    top = (size <= max_size) & ((par < 0) | (size[np.maximum(par, 0)] > max_size))
    lab = np.full(len(par), -1, np.int64)
    for nodes in levels:
        t = top[nodes]
        lab[nodes[t]] = nodes[t]
        rest = nodes[~t]
        rest = rest[par[rest] >= 0]
        lab[rest] = lab[par[rest]]
    return np.flatnonzero(top), lab, size


def lockstep_gpu(fg, X_d, spec, ngroups=64, min_size=64, max_size=512, run_len=2432,
                 cap=32768, wblock=3):
    """Section 5.5 on the GPU harvest at the benchmark size (untimed extra).
    Lockstep density (Table 6): the visited sets V_i logged by the harvest
    searches themselves (fgraft_harvest_visited, each point on its own
    block's substrate S_b) for 64 coherent groups -- maximal tree-0 subtrees
    of at most 512 points, drawn among those of at least 64 -- and 64 random
    groups of the same sizes; density = sum |V_i| / (|group| |union V_i|),
    and the share of evaluations that go to vertices at least 8 members of
    the group evaluate.  Column-batched target loads: for windows of W
    consecutive searches of block 3's claim order (W = 4 is one CTA; 2432
    the searches in flight), the share of the window's evaluations that
    another search of the window repeats, 1 - |union| / sum |V_i|."""
    import torch
    params = _params(fg, spec)
    B = spec["B"]
    ix = fg.fgraft_build_scaffold(X_d, spec["d"], params)
    st = fg.fgraft_index_copy(ix)
    n = int(X_d.shape[0])
    tops, lab, size = _subtree_groups(st["parents"][0].cpu().numpy(), max_size)
    rng = np.random.default_rng(11)
    cand = tops[size[tops] >= min_size]
    pick = rng.choice(cand, size=min(ngroups, len(cand)), replace=False)
    order = np.argsort(lab, kind="stable")
    sl = lab[order]
    coherent = [order[np.searchsorted(sl, u):np.searchsorted(sl, u, side="right")] for u in pick]
    randoms = [rng.choice(n, size=len(g), replace=False) for g in coherent]
    sched = fg.fgraft_index_schedule(ix)
    q, r = n // B, n % B
    nb_w = q + (1 if wblock < r else 0)
    if sched is not None:
        start = wblock * q + min(wblock, r)
        qo = sched[1].cpu().numpy()[start:start + nb_w].astype(np.int64)
    else:
        qo = np.arange(nb_w, dtype=np.int64)
    off0 = nb_w // 2
    run = wblock + B * qo[off0:off0 + run_len]
    allp = np.unique(np.concatenate(coherent + randoms + [run]))
    pos = np.full(n, -1, np.int64)
    ids_all, cnt_all = [], []
    base = 0
    for b in range(B):
        pb = allp[allp % B == b].astype(np.int32)
        if len(pb):
            ids, cnt = fg.fgraft_harvest_visited(ix, torch.from_numpy(pb).cuda(), cap)
            ids_all.append(ids)
            cnt_all.append(cnt)
            pos[pb] = base + np.arange(len(pb))
            base += len(pb)
        fg.fgraft_harvest_block(ix, b)
    ids_all = torch.cat(ids_all)
    cnt_all = torch.cat(cnt_all)
    truncated = int((cnt_all > cap).sum().item())
    ar = torch.arange(cap, device=ids_all.device)

    def sets(pts):
        idx = torch.from_numpy(pos[np.asarray(pts)]).cuda()
        c = cnt_all[idx].clamp(max=cap)
        return ids_all[idx][ar[None, :] < c[:, None]], int(c.sum().item())

    def group_stats(groups):
        dens, share8, vs, us = [], [], [], []
        for g in groups:
            vals, tot = sets(g)
            uni, counts = torch.unique(vals, return_counts=True)
            dens.append(tot / (len(g) * uni.numel()))
            share8.append(float(counts[counts >= 8].sum().item()) / tot)
            vs.append(tot / len(g))
            us.append(uni.numel())
        return {"groups": len(groups), "median_size": int(np.median([len(g) for g in groups])),
                "mean_V": round(float(np.mean(vs)), 1), "mean_union": round(float(np.mean(us)), 1),
                "density_mean": round(float(np.mean(dens)), 4),
                "density_median": round(float(np.median(dens)), 4),
                "share_of_evals_to_targets_of_8_plus": round(float(np.mean(share8)), 4)}

    windows = []
    for W in (4, 16, 64, 256, run_len):
        sh = []
        for i in range(0, len(run) - W + 1, W):
            vals, tot = sets(run[i:i + W])
            sh.append(1.0 - torch.unique(vals).numel() / tot)
        windows.append({"W": W, "shared_share": round(float(np.mean(sh)), 4), "windows": len(sh)})
    vals, tot = sets(run)
    in_flight_union = int(torch.unique(vals).numel())
    row_bytes = 16 * ((spec["d"] * 4 + 15) // 16)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    del ix
    return {"coherent": group_stats(coherent), "random": group_stats(randoms),
            "windows_claim_order_block3": windows,
            "in_flight_union_vectors": in_flight_union,
            "l2_holds_vectors": int(l2 // row_bytes), "truncated_logs": truncated,
            "cap": cap, "data": "benchmark workload; V_i from the GPU harvest's own searches"}


def _extra(fn, *a, **kw):
    """An untimed extra measurement; a failure is recorded, not raised."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    fgbuild.build()
    fg.load()
    spec = dict(SPEC)
    if args.n:
        spec["n"] = args.n
    ps, Q, blocks, dev_in = _device_inputs(spec)
    X_d, Q_d, B_d = dev_in
    d = spec["d"]
    params = _params(fg, spec)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # ---- autotuner (outside the timed region): the harvest launch settings
    # for this shape, kept in the process's table for every later build ----
    tuning = tune(fg, X_d, spec, params, 32768, args.tune_table)

    # ---- timed region: inputs resident in HBM ----
    for _ in range(args.warmup):
        _step(fg, spec, params, *dev_in)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    total_ms, harvest_ms, harvest_launches, prune_ms, ctr_sum, launches, last = _timed(
        fg, spec, params, dev_in, args.steps, 0, flush, stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    n = spec["n"]
    ms_per_step, value = job_rate(total_ms, args.steps, n, world, dist if world > 1 else None,
                                  "cuda")

    # ---- breakdown (one untimed profiled pass) ----
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    flush.fill_(1.0)
    evs[0].record(stream)
    ix = fg.fgraft_build_scaffold(X_d, d, params)
    evs[1].record(stream)
    for b in range(spec["B"]):
        fg.fgraft_harvest_block(ix, b)
    evs[2].record(stream)
    fg.fgraft_prune(ix)
    evs[3].record(stream)
    ids, dist_, ev = fg.fgraft_search(ix, Q_d, spec["topk"], spec["ef_s"])
    evs[4].record(stream)
    di, dd, dst = fg.fgraft_dense_block_dist(X_d, d, fg.ANGULAR_F32, B_d, spec["dense_k"],
                                             precision=1, stats=True)
    evs[5].record(stream)
    torch.cuda.synchronize()
    names = ["scaffold", "harvest_blocks_no_graph", "final_prune", "search", "dense_blocks"]
    breakdown = {nm: round(evs[i].elapsed_time(evs[i + 1]), 3) for i, nm in enumerate(names)}
    search_evals = float(ev.double().sum().item())
    # the same blocks replayed as one CUDA graph (with the final graph), against
    # one launch sequence per block (with the final graph)
    ixg = fg.fgraft_build_scaffold(X_d, d, params)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1.0)
    g0.record(stream)
    fg.fgraft_harvest_all(ixg, use_graph=True)
    g1.record(stream)
    torch.cuda.synchronize()
    breakdown["harvest_graph_plus_final"] = round(g0.elapsed_time(g1), 3)
    breakdown["harvest_plain_plus_final"] = round(breakdown["harvest_blocks_no_graph"]
                                                  + breakdown["final_prune"], 3)
    # the graph-replayed and the plain build give the same final graph
    fa, fb = fg.fgraft_prune(ix), fg.fgraft_prune(ixg)
    graph_hash = hashlib.sha256(fa[0].cpu().numpy().tobytes() + fa[1].cpu().numpy().tobytes()
                                ).hexdigest()[:16]
    graph_same = bool(torch.equal(fa[0], fb[0]) and torch.equal(fa[1], fb[1]))
    del ixg

    # ---- dense blocks in the other precisions (untimed, same blocks) ----
    dense_other = {}
    for prec, name in ((1, "bf16"), (2, "fp8_e4m3")):
        # the filter's error against float64 on the reranked pairs (slow, separate call)
        _, _, est = fg.fgraft_dense_block_dist(X_d, d, fg.ANGULAR_F32, B_d, spec["dense_k"],
                                               precision=prec, stats=True, err64=True)
        dense_other[name + "_error_check"] = {"max_err_over_bound": round(est[4], 5),
                                              "max_canonical_err": est[5]}
    # the raw dense ceiling: the tensor-core Gram of every pair, no selection
    gram = {}
    for prec, name in ((1, "bf16"), (2, "fp8_e4m3")):
        fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, B_d, precision=prec)
        tms = []
        for _ in range(3):
            flush.fill_(1.0)
            _, gms = fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, B_d, precision=prec)
            tms.append(gms)
        gms = float(np.median(tms))
        dpad = ((d + 63) // 64) * 64 if prec == 1 else ((d + 127) // 128) * 128
        mma_flops = 2.0 * dpad * spec["dense_blocks"] * 1024 * 1024
        gram[name] = {"ms": round(gms, 4), "tflops_mma": round(mma_flops / (gms / 1e3) / 1e12, 1)}
    for prec, name in ((0, "fp32_cuda_cores"), (2, "fp8_e4m3")):
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        pi, pd, pst = fg.fgraft_dense_block_dist(X_d, d, fg.ANGULAR_F32, B_d, spec["dense_k"],
                                                 precision=prec, stats=True)
        q1.record(stream)
        torch.cuda.synchronize()
        same = bool(torch.equal(pi, di) and torch.equal(pd, dd))
        dense_other[name] = {"ms": round(q0.elapsed_time(q1), 3), "same_top_k_as_bf16": same}
        if prec == 2:
            dense_other[name]["rerank_fraction"] = round(pst[0], 5)
            dense_other[name]["filter_ms"] = round(pst[1], 4)
    quality = quality_report(fg, ix, ps, Q_d, spec)

    # ---- end to end through the public API, host buffers ----
    # inputs from pinned host memory; outputs into pinned host buffers made
    # once (sized for the largest final graph, n*R + 2(n-1) ids)
    Xh = torch.from_numpy(ps.X).pin_memory()
    Qh = torch.from_numpy(Q).pin_memory()
    Bh = torch.from_numpy(blocks).pin_memory()
    h2d = Xh.numel() * 4 + Qh.numel() * 4 + Bh.numel() * 4
    nb_d = blocks.shape[0] * blocks.shape[1]
    h_off = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
    h_ids = torch.empty(n * spec["R"] + 2 * (n - 1), dtype=torch.int32, pin_memory=True)
    h_qi = torch.empty((Q.shape[0], spec["topk"]), dtype=torch.int32, pin_memory=True)
    h_qd = torch.empty((Q.shape[0], spec["topk"]), dtype=torch.float32, pin_memory=True)
    h_di = torch.empty((nb_d, spec["dense_k"]), dtype=torch.int32, pin_memory=True)
    h_dd = torch.empty((nb_d, spec["dense_k"]), dtype=torch.float32, pin_memory=True)
    del ix
    e2e_ms, d2h = 0.0, 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Xd2 = Xh.to("cuda", non_blocking=True)
        Qd2 = Qh.to("cuda", non_blocking=True)
        Bd2 = Bh.to("cuda", non_blocking=True)
        ix2 = fg.fgraft_build_scaffold(Xd2, d, params)
        fg.fgraft_harvest_all(ix2, use_graph=True)
        off2, gids2 = fg.fgraft_prune(ix2)  # copies out the graph harvest_all made
        ids2, dist2, ev2 = fg.fgraft_search(ix2, Qd2, spec["topk"], spec["ef_s"])
        di2, dd2 = fg.fgraft_dense_block_dist(Xd2, d, fg.ANGULAR_F32, Bd2, spec["dense_k"],
                                              precision=1)
        nnz = gids2.numel()
        h_off.copy_(off2, non_blocking=True)
        h_ids[:nnz].copy_(gids2, non_blocking=True)
        h_qi.copy_(ids2, non_blocking=True)
        h_qd.copy_(dist2, non_blocking=True)
        h_di.copy_(di2.reshape(nb_d, -1), non_blocking=True)
        h_dd.copy_(dd2.reshape(nb_d, -1), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        d2h = (h_off.numel() * 8 + nnz * 4 + h_qi.numel() * 4 + h_qd.numel() * 4 +
               h_di.numel() * 4 + h_dd.numel() * 4)
        del ix2, Xd2, Qd2, Bd2, off2, gids2, ids2, dist2, ev2, di2, dd2
    _, e2e_value = job_rate(e2e_ms, args.steps, n, world, dist if world > 1 else None, "cuda")
    extras = not args.n and not args.no_extras
    arms = _extra(paper_arms, fg, X_d, Q_d, ps, Q, spec) if extras else None
    dims = _extra(dims_sweep, fg) if extras and not args.no_dims else None
    lockstep = _extra(lockstep_gpu, fg, X_d, spec) if extras else None
    extra = incache_extra(fg, flush, stream,
                          tune_table=args.tune_table + ".incache" if args.tune_table else None) \
        if extras else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    rec = recall_at_10(ps.X[:, :d], Q[:, :d], last[1].cpu().numpy())
    hbm, peak_kind = peaks()
    evals = ctr_sum.get("harvest_evals", 0)
    alg_bytes = _alg_bytes(spec, ctr_sum)
    achieved = alg_bytes / (harvest_ms / 1e3) / 1e9 if harvest_ms > 0 else 0.0
    traffic = ncu_traffic(BEAM_SOURCES)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    nvalid = (blocks >= 0).sum(axis=1).astype(np.int64)
    dense_pairs = int((nvalid * (nvalid - 1)).sum())
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "pts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": spec["workload"], "n": n, "d": d, "metric_kind": "angular",
                   "clusters": spec["k"], "cluster_sizes": "zipf(1.1)", "T": spec["T"],
                   "B": spec["B"], "R": spec["R"], "ef_h": spec["ef_h"], "alpha": spec["alpha"],
                   "nq": spec["nq"], "ef_s": spec["ef_s"], "dense_blocks": spec["dense_blocks"],
                   "block_size": spec["block_size"], "dense_k": spec["dense_k"],
                   "parallelism": f"replicas{world}", "schedule": args.schedule,
                   "l2": "flushed before each timed step (256 MiB write); the vectors "
                         f"({ps.X.nbytes / 1e6:.0f} MB) exceed L2"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": traffic, "kernel": "beam_kernel (harvest search)",
                     "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes / max(harvest_launches, 1),
                     "launch_ms": harvest_ms / max(harvest_launches, 1)},
        "harvest_evals_per_s": round(evals / (harvest_ms / 1e3), 1) if harvest_ms else None,
        "harvest_sm_cycles_per_eval": round(harvest_ms / 1e3 * mhz * 1e6 * nsm / evals, 1)
        if evals else None,
        "harvest_prune_ms_per_block": round(prune_ms / max(harvest_launches, 1), 4),
        "prune_evals_per_s": round(ctr_sum.get("prune_evals", 0) / (prune_ms / 1e3), 1)
        if prune_ms else None,
        "build_evals_per_s": round((ctr_sum.get("harvest_evals", 0) + ctr_sum.get("prune_evals", 0)
                                    + ctr_sum.get("sat_evals", 0)
                                    + ctr_sum.get("final_prune_evals", 0))
                                   / (ms_per_step * args.steps / 1e3), 1),
        "counters_per_build": {k_: v_ // args.steps for k_, v_ in ctr_sum.items()},
        "recall_at_10": round(rec, 4),
        "search_evals_per_query": round(search_evals / spec["nq"], 1),
        "dense_pairs": dense_pairs,
        "dense_pairs_per_s": round(dense_pairs / (breakdown["dense_blocks"] / 1e3), 1),
        "dense_filter_ms": round(dst[1], 4), "dense_rerank_ms": round(dst[2], 4),
        "dense_prep_ms": round(dst[3], 4),
        "dense_gram_pairs_per_s": round(dense_pairs / (gram["bf16"]["ms"] / 1e3), 1),
        "dense_gram": gram,
        "dense_rerank_fraction": round(dst[0], 5),
        "adaptive_dense_gap": round((dense_pairs / (breakdown["dense_blocks"] / 1e3))
                                    / (evals / (harvest_ms / 1e3)), 2) if harvest_ms else None,
        "dense_other_precisions": dense_other,
        "autotune": {k_: (round(v_, 4) if isinstance(v_, float) else v_)
                     for k_, v_ in tuning.items()},
        "graph_replay_same_graph": graph_same,
        "final_graph_sha256_16": graph_hash,
        "quality": quality,
        "breakdown_ms": breakdown,
        "incache": extra,
        "paper_arms": arms,
        "dims_sweep": dims,
        "lockstep_gpu": lockstep,
        "e2e": {"value": round(e2e_value, 1), "unit": "pts/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        work = sum(ctr_sum.get(k_, 0) for k_ in ("sat_evals", "harvest_evals", "prune_evals",
                                                  "final_prune_evals"))
        out["cpu_baseline"] = cpu_baselines(ps, spec, work / args.steps / n)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(ps, spec, sample_n=CPU_SAMPLE_N, seed=7, nthreads=None):
    """The oracle, as it stands, on a random subset of the workload's points."""
    import oracle
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(ps.n, size=min(sample_n, ps.n), replace=False))
    Xs = np.ascontiguousarray(ps.X[sel])
    D = oracle.Data(Xs, spec["d"], 1)
    cores = nthreads or os.cpu_count() or 1
    t0 = time.perf_counter()
    g = oracle.build_graph(D, spec["T"], spec["R"], spec["ef_h"], spec["B"], spec["alpha"],
                           spec["seed"], nthreads=cores)
    dt = time.perf_counter() - t0
    c = g["counters"]
    work = sum(c[k] for k in ("sat_evals", "harvest_evals", "prune_evals", "final_prune_evals"))
    return {"value": round(len(sel) / dt, 1), "unit": "pts/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle FGraft build (SAT forest, scaffold, {spec['B']} blocks, final graph) "
                      f"of a seeded {len(sel)}-point subset of the workload, same T/R/ef_h/B/alpha",
            "seconds": round(dt, 2), "evals_per_point": round(work / len(sel), 1)}


def cpu_baselines(ps, spec, gpu_evals_per_point=None):
    """The oracle on all host cores (the reported baseline) and on one core (a
    smaller subset, so that the bench stays within minutes).  A subset has
    shorter searches than the whole workload, so the oracle's rate is also
    given scaled by distance evaluations per point (the work the paper counts,
    Section 2): subset rate x subset evaluations per point / the whole
    workload's evaluations per point (the GPU build's counters, which equal
    the oracle's by definition)."""
    out = cpu_baseline(ps, spec)
    one = cpu_baseline(ps, spec, sample_n=CPU_SAMPLE_N // 4, seed=8, nthreads=1)
    out["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample", "seconds",
                                                "evals_per_point")}
    if gpu_evals_per_point:
        out["scaled_to_workload"] = {
            "value": round(out["value"] * out["evals_per_point"] / gpu_evals_per_point, 1),
            "unit": "pts/s", "workload_evals_per_point": round(gpu_evals_per_point, 1),
            "how": "subset rate x subset evaluations per point / workload evaluations per point"}
    return out


def run_reference(args):
    rank, world, local = env_rank()
    if rank != 0:
        return
    spec = dict(SPEC)
    if args.n:
        spec["n"] = args.n
    ps, Q, blocks = make_inputs(spec)
    import oracle
    oracle.build()
    sample_n = 10_000
    for _ in range(args.warmup):
        cpu_baseline(ps, spec, sample_n=2_000)
    secs = 0.0
    for i in range(args.steps):
        r = cpu_baseline(ps, spec, sample_n=sample_n, seed=11 + i)
        secs += r["seconds"]
    value = args.steps * sample_n / secs
    cores = os.cpu_count() or 1
    sample = (f"oracle FGraft build of a seeded {sample_n}-point subset of the workload per step "
              f"(SAT forest, scaffold, {spec['B']} blocks, final graph), same T/R/ef_h/B/alpha")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "pts/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(secs / args.steps * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": spec["n"], "d": spec["d"], "T": spec["T"],
                      "B": spec["B"], "R": spec["R"], "ef_h": spec["ef_h"],
                      "alpha": spec["alpha"], "parallelism": "cpu-oracle"},
           "cpu_baseline": {"value": round(value, 1), "unit": "pts/s", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 1), "unit": "pts/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _sm_clock_mhz():
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout.split()
        return float(out[0])
    except Exception:
        return None


def run_dims(args):
    """Cost per distance evaluation of the adaptive harvest and of the dense block,
    across d (Section 5.4, Table 5): Gaussian mixture, 128 clusters, L2, T = 8, B = 8,
    R = 32, ef_h = 64, plus byte vectors at d = 128."""
    import torch
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    from paper_2609_30493_gb300 import synth
    fgbuild.build()
    fg.load()
    n = args.n or 1_000_000
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    dims = [(int(t[:-2]), "u8") if t.endswith("u8") else (int(t), "f32")
            for t in args.dims.split(",")]
    for d, kind in dims:
        ps = synth.uint8_mixture(n, d, 128, 0) if kind == "u8" else synth.gaussian_mixture(n, d, 128, 0)
        X = torch.from_numpy(ps.X).cuda()
        p = fg.Params(T=8, R=32, ef_h=64, B=8, alpha=1.2, seed=0, metric=ps.metric)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = fg.fgraft_build_scaffold(X, d, p)
        torch.cuda.synchronize()
        t_sc = time.perf_counter() - t0
        fg.fgraft_index_profile(ix, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for b in range(8):
            fg.fgraft_harvest_block(ix, b)
        e1.record()
        torch.cuda.synchronize()
        hms, hl = fg.fgraft_index_harvest_ms(ix)
        c = fg.fgraft_index_counters(ix)
        clk = _sm_clock_mhz() or 2070.0
        evals = c["harvest_evals"]
        rate = evals / (hms / 1e3)
        dense = dense_simt = gram = rerank = None
        if kind == "f32":
            blocks = synth.intra_cluster_blocks(ps.labels, 64, 1024, 2)
            Bd = torch.from_numpy(blocks).cuda()
            pairs = 64 * 1024 * 1023
            for prec in (0, 1):
                fg.fgraft_dense_block_dist(X, d, 0, Bd, 32, precision=prec)
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record()
                for _ in range(3):
                    _, _, st = fg.fgraft_dense_block_dist(X, d, 0, Bd, 32, precision=prec,
                                                          stats=True)
                f1.record()
                torch.cuda.synchronize()
                rate = pairs / (f0.elapsed_time(f1) / 3 / 1e3)
                if prec == 0:
                    dense_simt = rate
                else:
                    dense, gram, rerank = rate, pairs / (st[1] / 1e3), st[0]
            rate = evals / (hms / 1e3)
        row = {"mode": "dims", "d": d, "kind": kind, "n": n, "scaffold_s": round(t_sc, 3),
               "harvest_ms": round(hms, 2), "harvest_evals": evals,
               "harvest_evals_per_s": round(rate, 1),
               "sm_cycles_per_eval": round(hms / 1e3 * clk * 1e6 * nsm / evals, 1),
               "harvest_bytes_per_eval": 32 * ((ps.X.itemsize * d + 31) // 32),
               "harvest_GBps": round(rate * 32 * ((ps.X.itemsize * d + 31) // 32) / 1e9, 1),
               "dense_pairs_per_s": round(dense, 1) if dense else None,
               "dense_gram_pairs_per_s": round(gram, 1) if gram else None,
               "dense_rerank_fraction": round(rerank, 5) if rerank is not None else None,
               "dense_simt_pairs_per_s": round(dense_simt, 1) if dense_simt else None,
               "gap_W": round(dense / rate, 2) if dense else None,
               "gap_W_gram": round(gram / rate, 2) if gram else None,
               "reruns": c["reruns"]}
        rows.append(row)
        print(json.dumps(row), flush=True)
        del ix, X
        torch.cuda.empty_cache()
    f = [r for r in rows if r["kind"] == "f32"]
    if len(f) < 2:
        return
    ld = np.log([r["d"] for r in f])
    ka = np.polyfit(ld, np.log([1.0 / r["harvest_evals_per_s"] for r in f]), 1)[0]
    kd = np.polyfit(ld, np.log([1.0 / r["dense_pairs_per_s"] for r in f]), 1)[0]
    kg = np.polyfit(ld, np.log([1.0 / r["dense_gram_pairs_per_s"] for r in f]), 1)[0]
    print(json.dumps({"mode": "dims-fit", "adaptive_cost_exponent": round(float(ka), 3),
                      "dense_cost_exponent": round(float(kd), 3),
                      "gap_exponent": round(float(ka - kd), 3),
                      "gram_cost_exponent": round(float(kg), 3),
                      "gram_gap_exponent": round(float(ka - kg), 3)}), flush=True)


def run_paper(args):
    """Paper-scale angular arms (Section 4, Table 1 shape): n = 1,183,514, d = 100,
    256 clusters with Zipf(1.1) sizes; frozen T = 32 and FGraft T = 8 at
    B = 1, 2, 4, 8, 16; R = 64, ef_h = 100; recall@10 and evaluations per query
    over a beam-width ladder, d@0.95 interpolated (Section 2)."""
    import torch
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    from paper_2609_30493_gb300 import synth
    fgbuild.build()
    fg.load()
    n = args.n or 1_183_514
    ps = synth.vmf_like(n, 100, 256, 0, 20.0, sizes="zipf")
    Q = synth.queries(ps, 10_000, 1)
    X = torch.from_numpy(ps.X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    Xt = X[:, :100]
    gts = []
    for s0 in range(0, len(Q), 1024):
        gts.append(torch.topk(Qd[s0:s0 + 1024, :100] @ Xt.T, 10, dim=1).indices.cpu().numpy())
    gt = np.concatenate(gts)
    arms = [tuple(int(v) for v in a.split("x")) for a in args.arms.split(",")]
    tunes = [tuple(int(v) for v in t.split("x")) for t in args.tunes.split(",")]
    for (T, B), (hl2, wpc) in [(a, t) for a in arms for t in tunes]:
        p = fg.Params(T=T, R=64, ef_h=100, B=B, alpha=1.2, seed=0, metric=fg.ANGULAR_F32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = fg.fgraft_build_scaffold(X, 100, p)
        if hl2 or wpc:
            fg.fgraft_index_tune(ix, hash_log2=hl2, warps_per_cta=wpc)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fg.fgraft_index_profile(ix, True)
        fg.fgraft_harvest_all(ix, use_graph=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        hms, hl = fg.fgraft_index_harvest_ms(ix)
        c = fg.fgraft_index_counters(ix)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        fg.fgraft_prune(ix)  # the final graph again, timed alone
        f1.record()
        torch.cuda.synchronize()
        final_s = f0.elapsed_time(f1) / 1e3
        ladder = []
        for ef in [] if args.no_ladder else [10, 16, 24, 32, 48, 64, 96, 128]:
            ids, dist, ev = fg.fgraft_search(ix, Qd, 10, ef)
            ids = ids.cpu().numpy()
            rec = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / 10 for a, b in zip(ids, gt)]))
            ladder.append((ef, rec, float(ev.double().mean().item())))
        d95 = None
        for (e0, r0, v0), (e1_, r1, v1) in zip(ladder, ladder[1:]):
            if r0 < 0.95 <= r1:
                d95 = v0 + (0.95 - r0) * (v1 - v0) / (r1 - r0)
        row = {"mode": "paper", "schedule": args.schedule, "hash_log2": hl2, "wpc": wpc,
               "n": n, "T": T, "B": B, "R": 64, "ef_h": 100,
               "scaffold_s": round(t1 - t0, 3), "harvest_and_final_s": round(t2 - t1, 3),
               "final_s": round(final_s, 3),
               "build_s": round(t2 - t0, 3), "pts_per_s": round(n / (t2 - t0), 1),
               "harvest_kernel_ms": round(hms, 1),
               "harvest_evals_per_s": round(c["harvest_evals"] / (hms / 1e3), 1),
               "counters": c, "recall_ladder": ladder,
               "dist_per_query_at_0.95": round(d95, 1) if d95 else None}
        print(json.dumps(row), flush=True)
        del ix
        torch.cuda.empty_cache()


def batched_inputs(i, n, d, device):
    """Build i of the batched configuration, generated on the device with a
    torch generator seeded by i: d = 64 or 960, unit vectors from 64
    vMF-like clusters (kappa = 20, equal sizes); d = 128, uint8 from a mixture
    of 128 Gaussian clusters (centres N(0, 25 I), unit noise) mapped by
    clip(round(60 + 30 z / sqrt(26)), 0, 255).  Rows padded to 16 bytes."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(1000 + i)
    if d == 128:
        cent = 5.0 * torch.randn(128, d, generator=g, device=device)
        lab = torch.randint(0, 128, (n,), generator=g, device=device)
        z = cent[lab] + torch.randn(n, d, generator=g, device=device)
        return torch.clamp(torch.round(60.0 + 30.0 * z / 26.0 ** 0.5), 0, 255).to(torch.uint8)
    mu = torch.nn.functional.normalize(torch.randn(64, d, generator=g, device=device), dim=1)
    lab = torch.randperm(n, generator=g, device=device) % 64
    x = mu[lab] + torch.randn(n, d, generator=g, device=device) / 20.0 ** 0.5
    return torch.nn.functional.normalize(x, dim=1).contiguous()


def run_batched(args):
    """Many independent builds at once (64 by default): n log-uniform in
    [10^4, 5 * 10^5], d from {64, 128, 960}; T = 8, B = 8, R = 32, ef_h = 64.
    Timed: every scaffold, then block by block all indices together through
    fgraft_harvest_block_multi, then every final graph.  Untimed comparison:
    the same builds one after another."""
    import torch
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    fgbuild.build()
    fg.load()
    nbuild = args.batch
    rng = np.random.default_rng(5)
    ns = np.floor(np.exp(rng.uniform(np.log(1e4), np.log(5e5), nbuild))).astype(np.int64)
    ds = rng.choice([64, 128, 960], nbuild)
    data = [batched_inputs(i, int(ns[i]), int(ds[i]), "cuda") for i in range(nbuild)]
    torch.cuda.synchronize()

    def params(d):
        return fg.Params(T=8, R=32, ef_h=64, B=8, alpha=1.2, seed=0,
                         metric=fg.L2_U8 if d == 128 else fg.ANGULAR_F32)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def batched(phases=None):
        e0 = ev()
        ixs = [fg.fgraft_build_scaffold(data[i], int(ds[i]), params(int(ds[i])))
               for i in range(nbuild)]
        e1 = ev()
        for b in range(8):
            fg.fgraft_harvest_block_multi(ixs, b)
        e2 = ev()
        for ix in ixs:
            fg.fgraft_prune(ix)
        e3 = ev()
        if phases is not None:
            phases.append((e0, e1, e2, e3))
        return ixs

    def one_by_one(phases):
        # the same calls build after build: scaffold, blocks, final graph
        out = []
        for i in range(nbuild):
            e0 = ev()
            ix = fg.fgraft_build_scaffold(data[i], int(ds[i]), params(int(ds[i])))
            e1 = ev()
            for b in range(8):
                fg.fgraft_harvest_block(ix, b)
            e2 = ev()
            fg.fgraft_prune(ix)
            e3 = ev()
            phases.append((int(ds[i]), e0, e1, e2, e3))
            out.append(ix)
        return out

    for _ in range(max(args.warmup, 1)):
        del_ = batched()
        del del_
    torch.cuda.synchronize()
    clocks = Clocks(0)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    times = []
    bph = []
    for _ in range(args.steps):
        t0.record()
        ixs = batched(bph)
        t1.record()
        torch.cuda.synchronize()
        times.append(t0.elapsed_time(t1))
        del ixs
    clk = clocks.stop()
    sph = []
    t0.record()
    seq = one_by_one(sph)
    t1.record()
    torch.cuda.synchronize()
    seq_ms = t0.elapsed_time(t1)
    same = True
    ixs = batched()
    for a_, b_ in zip(ixs, seq):
        oa, ob = fg.fgraft_prune(a_), fg.fgraft_prune(b_)
        same &= bool(torch.equal(oa[0], ob[0]) and torch.equal(oa[1], ob[1]))
    # where the time goes: phase sums of both ways, and the one-by-one
    # harvest by dimension
    nst = max(len(bph), 1)
    b_ms = {k: round(sum(p[i].elapsed_time(p[i + 1]) for p in bph) / nst, 3)
            for i, k in enumerate(("scaffold", "harvest", "final"))}
    s_ms = {k: round(sum(p[i + 1].elapsed_time(p[i + 2]) for p in sph), 3)
            for i, k in enumerate(("scaffold", "harvest", "final"))}
    by_d = {}
    for p in sph:
        t = by_d.setdefault(str(p[0]), {"builds": 0, "n": 0, "harvest_ms": 0.0})
        t["builds"] += 1
        t["harvest_ms"] = round(t["harvest_ms"] + p[2].elapsed_time(p[3]), 3)
    for i in range(nbuild):
        by_d[str(int(ds[i]))]["n"] += int(ns[i])
    ms = float(np.mean(times))
    total_n = int(ns.sum())
    print(json.dumps({
        "metric": "batched FGraft builds pts/s, 1 GB300", "mode": "batched",
        "value": round(total_n / (ms / 1e3), 1), "unit": "pts/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "dtype": "f32 and u8", "data": "synthetic (device generator)",
        "config": {"workload": f"batched-{nbuild}-builds", "builds": nbuild, "sum_n": total_n,
                   "n_min": int(ns.min()), "n_max": int(ns.max()),
                   "builds_by_d": {str(k): int((ds == k).sum()) for k in (64, 128, 960)},
                   "T": 8, "B": 8, "R": 32, "ef_h": 64},
        "one_by_one_ms": round(seq_ms, 3),
        "batched_vs_one_by_one": round(seq_ms / ms, 3),
        "phases_ms": {"batched": b_ms, "one_by_one": s_ms},
        "one_by_one_harvest_by_d": by_d,
        "same_graphs_as_one_by_one": same,
        "clocks": clk}), flush=True)


def run_cap(args):
    """Section 6's negative result on the in-cache workload: the scaffold's
    rows capped at K nearest (K = 0 is no cap); build time, work (distance
    evaluations) and quality (recall ladder, local completeness) per K."""
    import torch
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    fgbuild.build()
    fg.load()
    spec = dict(INCACHE)
    ps, Q, blocks = make_inputs(spec)
    d = spec["d"]
    X_d = torch.from_numpy(ps.X).cuda()
    Q_d = torch.from_numpy(Q).cuda()
    params = fg.Params(T=spec["T"], R=spec["R"], ef_h=spec["ef_h"], B=spec["B"],
                       alpha=spec["alpha"], seed=spec["seed"], metric=fg.ANGULAR_F32)
    for cap in (0, 64, 32, 16, 8):
        fg.fgraft_tune_scaffold_cap(cap)
        ts = []
        for r in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ix = fg.fgraft_build_scaffold(X_d, d, params)
            fg.fgraft_harvest_all(ix, use_graph=False)
            torch.cuda.synchronize()
            if r >= args.warmup:
                ts.append(time.perf_counter() - t0)
        c = fg.fgraft_index_counters(ix)
        sizes = ix.sizes()
        q = quality_report(fg, ix, ps, Q_d, spec)
        work = c["harvest_evals"] + c["prune_evals"] + c["final_prune_evals"] + c["sat_evals"]
        print(json.dumps({"mode": "cap", "cap": cap, "n": spec["n"], "build_ms": round(1e3 * float(np.median(ts)), 3),
                          "scaffold_nnz": sizes["scaffold_nnz"], "counters": c, "work": work,
                          "recall_at_10_ef64": next(x["recall_at_10"] for x in q["recall_ladder"] if x["ef_s"] == 64),
                          "recall_at_10_ef128": next(x["recall_at_10"] for x in q["recall_ladder"] if x["ef_s"] == 128),
                          "evals_per_query_ef128": next(x["evals_per_query"] for x in q["recall_ladder"] if x["ef_s"] == 128),
                          "local_completeness_at_10": q["local_completeness_at_10"]}), flush=True)
        del ix
    fg.fgraft_tune_scaffold_cap(0)


def run_tc(args):
    """The tensor-core Gram kernels alone, for profiling: the Gram-only dense
    blocks on the benchmark's 64 blocks repeated 16 times (1,024 blocks),
    twice, then the exact 10-NN of the first 16,384 points among all n."""
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    fgbuild.build()
    fg.load()
    spec = dict(SPEC)
    if args.n:
        spec["n"] = args.n
    _, _, _, (X_d, _, B_d) = _device_inputs(spec)
    Bn = B_d.repeat(16, 1).contiguous()
    d = spec["d"]
    out = {"mode": "tc", "n": spec["n"], "gram_ms": []}
    for _ in range(2):
        _, gms = fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, Bn, precision=1)
        out["gram_ms"].append(round(gms, 4))
    _, _, st = fg.fgraft_knn_exact(X_d, d, fg.ANGULAR_F32, 10, 0, min(16384, spec["n"]),
                                   stats=True)
    out["knn"] = st
    print(json.dumps(out), flush=True)


def run_lockstep(args):
    """The lockstep-density and column-batching measurement alone."""
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    fgbuild.build()
    fg.load()
    spec = dict(SPEC)
    if args.n:
        spec["n"] = args.n
    _, _, _, (X_d, _, _) = _device_inputs(spec)
    print(json.dumps({"mode": "lockstep", "n": spec["n"], **lockstep_gpu(fg, X_d, spec)}),
          flush=True)


def run_dense(args):
    """The dense-block ceiling alone (Section 5.3) on the benchmark workload's 64
    intra-cluster blocks of 1024 points (top-64 per row): the canonical float32
    kernel on CUDA cores, the BF16 and FP8 tensor-core filters with float32
    rerank (all three top-k identical), and the raw tensor-core Gram without
    selection.  L2 is flushed before every timed call."""
    import torch
    from paper_2609_30493_gb300 import build as fgbuild
    from paper_2609_30493_gb300 import fgraft as fg
    fgbuild.build()
    fg.load()
    spec = dict(SPEC)
    if args.n:
        spec["n"] = args.n
    ps, Q, blocks, (X_d, Q_d, B_d) = _device_inputs(spec)
    d, k = spec["d"], spec["dense_k"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    nvalid = (blocks >= 0).sum(axis=1).astype(np.int64)
    pairs = int((nvalid * (nvalid - 1)).sum())
    ref = None
    for prec, name in ((0, "fp32_cuda_cores"), (1, "bf16"), (2, "fp8_e4m3")):
        for _ in range(max(args.warmup, 1)):
            fg.fgraft_dense_block_dist(X_d, d, fg.ANGULAR_F32, B_d, k, precision=prec)
        ts, st = [], None
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gi, gd, st = fg.fgraft_dense_block_dist(X_d, d, fg.ANGULAR_F32, B_d, k,
                                                    precision=prec, stats=True)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        same = None if ref is None else bool(torch.equal(gi, ref[0]) and torch.equal(gd, ref[1]))
        ref = ref or (gi, gd)
        print(json.dumps({"mode": "dense", "precision": name, "blocks": int(len(blocks)),
                          "pairs": pairs, "k": k, "ms": round(ms, 4),
                          "pairs_per_s": round(pairs / (ms / 1e3), 1),
                          "filter_ms": round(st[1], 4), "rerank_ms": round(st[2], 4),
                          "prep_ms": round(st[3], 4), "rerank_fraction": round(st[0], 5),
                          "same_top_k_as_fp32": same}), flush=True)
    for prec, name in ((1, "bf16"), (2, "fp8_e4m3")):
        fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, B_d, precision=prec)
        tms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            _, gms = fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, B_d, precision=prec)
            tms.append(gms)
        gms = float(np.median(tms))
        dpad = ((d + 63) // 64) * 64 if prec == 1 else ((d + 127) // 128) * 128
        flops = 2.0 * dpad * len(blocks) * 1024 * 1024
        print(json.dumps({"mode": "dense-gram", "precision": name, "ms": round(gms, 4),
                          "pairs_per_s": round(pairs / (gms / 1e3), 1),
                          "tflops_mma": round(flops / (gms / 1e3) / 1e12, 1)}), flush=True)
    # the same Gram over more blocks (the 64 blocks repeated): 64 blocks are
    # 3.4 tiles of 128 rows per SM, too few to fill the MMA pipeline
    for prec, name in ((1, "bf16"), (2, "fp8_e4m3")):
        dpad = ((d + 63) // 64) * 64 if prec == 1 else ((d + 127) // 128) * 128
        for reps in (4, 16, 64):
            Bn = B_d.repeat(reps, 1).contiguous()
            fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, Bn, precision=prec)
            tms = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                _, gms = fg.fgraft_dense_block_gram(X_d, d, fg.ANGULAR_F32, Bn, precision=prec)
                tms.append(gms)
            gms = float(np.median(tms))
            nbn = int(Bn.shape[0])
            flops = 2.0 * dpad * nbn * 1024 * 1024
            print(json.dumps({"mode": "dense-gram-scale", "precision": name, "blocks": nbn,
                              "ms": round(gms, 4),
                              "pairs_per_s": round(pairs * reps / (gms / 1e3), 1),
                              "tflops_mma": round(flops / (gms / 1e3) / 1e12, 1)}), flush=True)
            del Bn


def main():
    args = parse()
    if args.impl != "reference" and args.schedule != "auto":
        from paper_2609_30493_gb300 import build as fgbuild, fgraft as fg
        fgbuild.build()
        fg.load()
        fg.fgraft_tune_schedule({"id": 0, "coherent": 1}[args.schedule])
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "dims":
        run_dims(args)
    elif args.mode == "paper":
        run_paper(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "cap":
        run_cap(args)
    elif args.mode == "dense":
        run_dense(args)
    elif args.mode == "lockstep":
        run_lockstep(args)
    elif args.mode == "tc":
        run_tc(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
