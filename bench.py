#!/usr/bin/env python3
"""Decoded Mbit/s of batched syndrome-based sum-product BP on one GB300.

Workload (defaults): the rate-0.1 synthetic MET-LDPC ensemble at n = 10^6,
64 codewords per batch, 100 fixed flooding iterations, sigma from
beta = 0.90 (BIAWGN capacity), half-precision message storage with float
arithmetic.  One step = one mld_decode_y call over the whole batch: interleave,
100 x (check update + variable update), final hard decision and syndrome
check, de-interleave.  The message state (578 MB at f16) and the inputs
(256 MB) exceed the 129 MB L2, so no flush is needed between steps.

Reported: ``value`` (device-resident inputs), ``e2e`` (host pinned inputs and
outputs through the same public call, copies inside the timed region), the
roofline of the dominant kernel (check update) from per-launch CUDA events,
clocks sampled during the timed region, and the FP64 oracle timed on the
host cores (``cpu_baseline``).  ``--impl reference`` times the oracle alone.

Under torchrun (N > 1) every rank decodes its own batch on its own GPU with
no collective on the data path (replicas); the timing uses a barrier and the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "decoded Mbit/s at n=1e6, 64 codewords, fixed iters"
UNIT = "Mbit/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rate", type=float, default=0.1)
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--msg", default="f16", choices=["f16", "f32"])
    ap.add_argument("--slab", type=int, default=0)
    ap.add_argument("--beta", type=float, default=0.90)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--train-steps", type=int, default=80)
    ap.add_argument("--workload", default="fixed", choices=["fixed", "uneven", "wbp"],
                    help="fixed: one code, fixed iterations (the headline); uneven: 96 codewords over "
                         "rates 0.1/0.05/0.02 and n in {2^16, 2^18, 10^6}, caps 100/150/200, early "
                         "termination, one captured plan")
    ap.add_argument("--tune-cache", default=None)
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the sub-records (FP32 storage; rates 0.05 and 0.02)")
    ap.add_argument("--sub-steps", type=int, default=8)
    ap.add_argument("--vn-update", default="gather", choices=["gather", "accumulate"],
                    help="variable update of the headline decoder: CSC gather (deterministic) or "
                         "accumulation of the new messages inside the check update (atomic adds)")
    ap.add_argument("--staging", default="direct", choices=["direct", "bulk", "bulk_lsu"],
                    help="check-update operands of the headline decoder: read directly, or staged in "
                         "shared memory by bulk copies one group of checks ahead")
    return ap.parse_args()


DEFAULT_ITERS = {0.1: 100, 0.05: 150, 0.02: 200}

# The library times the kernels of every TIMING_EVERY-th iteration (events on
# the launching stream); sampling keeps the event records out of the step time.
TIMING_EVERY = 10

# DRAM bytes (read + write) of one check-update pass per (codeword x bit),
# from ncu's dram__bytes_read.sum + dram__bytes_write.sum of the three
# check-class launches of one iteration (rate 0.1, n = 3e5, 64 codewords,
# half messages: 396.83 MB); traffic grows with n, so it is scaled by the
# units a full pass processes.  Valid for the kernel of this commit only
# (see profiles/).
CHECK_PASS_TRAFFIC_PER_CW_BIT = {(0.1, "f16"): 396.83e6 / (64 * 3e5)}


def algorithmic_bytes(st: dict, msg: str, schedule: str = "flooding") -> tuple[float, float]:
    """Minimum bytes per codeword of one check-update pass and of one whole
    iteration, at message width b (2 for half storage, 4 for float):
      check pass: r read and written on every core edge (2 b e_core), the
        degree-1 channel terms read once (b m2), core posteriors read once
        (4 n_core), syndrome bits (m / 8);
      iteration: r read and written once (2 b e_core), degree-1 terms
        (b m2), core VNs: channel term read, posterior written and read
        (n_core (b + 8)), syndrome bits (m / 8).
    Layered schedule (the pass is the whole iteration): r read and written
    once (2 b e_core); a core VN's posterior is read and written in every
    layer that holds one of its checks, once per core edge (8 e_core: the
    posteriors, 4 B per codeword and VN, exceed L2 at full size); degree-1
    terms (b m2); syndrome bits (m / 8)."""
    b = 2 if msg == "f16" else 4
    e, m2, nc, m = st["e_core"], st["n_deg1"], st["n_core"], st["n_cn"]
    if schedule == "layered":
        it = 2 * b * e + 8 * e + b * m2 + m / 8
        return it, it
    check = 2 * b * e + b * m2 + 4 * nc + m / 8
    iteration = 2 * b * e + b * m2 + nc * (b + 8) + m / 8
    return check, iteration


def workload_config(a) -> dict:
    return {
        "workload": (f"synthetic MET-LDPC rate {a.rate}, n={a.n}, {a.batch} codewords, "
                     f"{a.iters} fixed BP iterations, beta={a.beta}"),
        "rate": a.rate, "n": a.n, "codewords": a.batch, "iters": a.iters,
        "beta": a.beta, "msg_storage": a.msg, "vn_update": a.vn_update, "staging": a.staging,
        "l2": "inputs and message state larger than L2 (no flush needed)",
        "parallelism": "replicas",
    }


def rank_data_seed(rank: int) -> int:
    """Replicas decode different codewords: rank r draws data seed 1000 + 64 r."""
    return 1000 + 64 * rank


def reduce_over_ranks(dist, ms: float, launches: int, device) -> tuple[float, int]:
    """Max of the timed region over ranks (the slowest replica sets the job
    time) and the sum of kernel launches; identity without a process group."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([launches], dtype=torch.int64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def job_throughput(world: int, batch: int, n: int, steps: int, ms_max: float) -> float:
    """Whole-job decoded Mbit/s: all ranks' bits over the slowest rank's time."""
    return world * batch * n * steps / (ms_max * 1e-3) / 1e6


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(wl, codewords: int, iters: int, threads: int) -> float:
    """Wall time of the FP64 oracle on the first `codewords` of the batch."""
    import oracle
    t = time.perf_counter()
    oracle.decode_y(wl.graph, wl.y[:codewords], wl.sigma[:codewords], wl.s[:codewords],
                    iters=iters, threads=threads)
    return time.perf_counter() - t


def cpu_baseline(wl, a) -> dict:
    """Oracle throughput extrapolated to the full iteration count.

    Runs the oracle on `cores` codewords for 1 and for 3 iterations; the
    difference gives the per-iteration cost, the rest the fixed cost.
    """
    cores = host_cores()
    c = max(1, min(cores, a.batch))
    t1 = oracle_sample(wl, c, 1, c)
    t3 = oracle_sample(wl, c, 3, c)
    per_it = max((t3 - t1) / 2.0, 1e-9)
    fixed = max(t1 - per_it, 0.0)
    t_full = fixed + a.iters * per_it
    return {"value": c * a.n / t_full / 1e6, "unit": UNIT, "cores": c, "kind": "oracle",
            "sample": (f"{c} codewords x n={a.n}, 1 and 3 iterations timed "
                       f"({t1:.2f} s, {t3:.2f} s), extrapolated to {a.iters} iterations")}


def run_reference(a, wl):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    cores = host_cores()
    c = max(1, min(cores, a.batch))
    k = 3
    for _ in range(a.warmup):
        oracle_sample(wl, c, k, c)
    times = [oracle_sample(wl, c, k, c) for _ in range(a.steps)]
    t = sum(times)
    # each step decodes c codewords for k of the a.iters iterations
    value = a.steps * c * a.n * k / a.iters / t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded MET ensemble, BIAWGN samples)", "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": c, "kind": "oracle",
                         "sample": f"each step: {c} codewords x n={a.n} x {k} iterations "
                                   f"(value scaled to {a.iters} iterations)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = (uuid or "").lower().replace("gpu-", "")
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="mld_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            if self.uuid and p[1].lower().replace("gpu-", "") != self.uuid:
                continue
            rows.append(p)
        if not rows:
            return None
        try:
            sm = [float(r[2]) for r in rows]
            smax = max(float(r[3]) for r in rows)
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def measured_peak_hbm() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def uneven_record(total: int, beta: float, msg: str, steps: int, warmup: int, rank: int, dev,
                  tune_cache=None) -> dict:
    """Uneven batch: every codeword draws its (rate, length); one plan (one
    CUDA-graph launch) decodes all groups with per-codeword early termination
    and each rate's iteration cap; slab widths chosen by the autotuner."""
    import torch
    import paper_1711_01783_gb300 as mld
    from paper_1711_01783_gb300.tune import SlabWidthTuner
    from synthetic import make_uneven_workload

    groups = make_uneven_workload(total, seed=3 + rank, beta=beta)
    tuner = SlabWidthTuner(tune_cache)
    jobs, widths = [], {}
    for rate, n, wl in groups:
        g = mld.Graph.from_edges(wl.graph)
        B = wl.y.shape[0]
        W = tuner.choose(g, B, msg)
        widths[f"{rate}/{n}"] = (B, W)
        jobs.append(dict(decoder=mld.Decoder(g, B, msg_dtype=msg, slab_width=W), y=torch.from_numpy(wl.y).to(dev),
                         sigma=torch.from_numpy(wl.sigma).to(dev), syndrome=torch.from_numpy(wl.s).to(dev),
                         max_iters=DEFAULT_ITERS[rate]))
    plan = mld.Plan(jobs, early_term=True)
    for _ in range(warmup):
        plan.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        outs = plan.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    bits = sum(wl.y.shape[0] * wl.y.shape[1] for _, _, wl in groups)
    rec = {"value": bits / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "workload": f"{total} codewords, (rate, n) uniform over {{0.1,0.05,0.02}} x {{2^16,2^18,10^6}}, "
                       f"caps 100/150/200, early termination, beta={beta}, {msg} messages",
           "groups (batch, slab width)": widths, "gpu_launches": plan.launches * steps,
           "frames_converged": sum(int(o["converged"].sum().item()) for o in outs),
           "mean_iters": [round(float(o["iters_used"].float().mean().item()), 2) for o in outs]}
    plan.close()
    return rec


def run_uneven(a, world, rank, local):
    """The uneven batch as the workload of the line (--workload uneven)."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    rec = uneven_record(a.batch, a.beta, a.msg, a.steps, a.warmup, rank, dev, a.tune_cache)
    clk = clocks.stop()
    line = {
        "metric": "decoded Mbit/s, uneven batch (mixed rates and lengths, early termination)",
        "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded MET ensembles, BIAWGN samples)",
        "config": {"workload": rec["workload"], "msg_storage": a.msg,
                   "groups (batch, slab width)": rec["groups (batch, slab width)"],
                   "l2": "n=10^6 groups exceed L2"},
        "gpu_launches": rec["gpu_launches"], "frames_converged": rec["frames_converged"],
        "mean_iters": rec["mean_iters"], "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_wbp(a, world, rank, local):
    """Weighted BP: for T = 10, 15 and 20 unrolled iterations, train the
    per-(iteration, edge type) weights on decoder-generated samples (rate 0.1,
    n = 10^5, 16 codewords, checkpoint every 5, Adam on the mean BCE), then
    compare the frame error rate of the trained weights with unit weights
    (plain BP) after the same T iterations at n = 10^6: an iterations-to-FER
    curve.  value = training throughput at T = 20 (codeword bits through
    forward + adjoint per second)."""
    import torch
    import paper_1711_01783_gb300 as mld
    from synthetic import make_workload, preset_graph

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_tr, B_tr, k = 100_000, 16, 5
    beta = a.beta
    g_tr = preset_graph(0.1, n_tr, 10)
    G_tr = mld.Graph.from_edges(g_tr)
    dec = mld.Decoder(G_tr, B_tr, msg_dtype="f32", slab_width=16)

    def batch(seed):
        wl = make_workload(0.1, n_tr, B_tr, 10, seed, beta=beta, graph=g_tr)
        llr = torch.from_numpy(2.0 * wl.y / (wl.sigma[:, None] ** 2)).to(dev)
        y = 1.0 - 2.0 * torch.from_numpy(wl.x.astype(np.float32)).to(dev)
        return llr, torch.from_numpy(wl.s).to(dev), y

    data = [batch(20_000 + i) for i in range(16)]
    val = batch(40_000)
    # held-out evaluation set at n = 10^6
    n_ev, B_ev = 1_000_000, 64
    wl_ev = make_workload(0.1, n_ev, B_ev, 11, 30_000, beta=beta)
    dec_ev = mld.Decoder(mld.Graph.from_edges(wl_ev.graph), B_ev, msg_dtype="f32")
    llr_ev = torch.from_numpy(2.0 * wl_ev.y / (wl_ev.sigma[:, None] ** 2)).to(dev)
    s_ev = torch.from_numpy(wl_ev.s).to(dev)
    x_ev = torch.from_numpy(wl_ev.x).to(dev)

    curve = {}
    ms = None
    for T in (10, 15, 20):
        wt = torch.ones((T, 3), device=dev, requires_grad=True)
        opt = torch.optim.Adam([wt], lr=0.003)

        def val_loss():
            with torch.no_grad():
                soft, _ = dec.wbp_forward(val[0], val[1], wt.detach(), keep_tape=False)
                return float(torch.nn.functional.softplus(-val[2] * soft).mean())

        def step(i):
            llr, s, y = data[i % len(data)]
            opt.zero_grad()
            soft = mld.weighted_bp(dec, llr, s, wt, ckpt_k=k)
            loss = torch.nn.functional.softplus(-y * soft).mean()
            loss.backward()
            opt.step()
            return loss

        before = val_loss()
        for i in range(a.warmup):
            step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(a.train_steps):
            step(a.warmup + i)
        e1.record()
        torch.cuda.synchronize()
        if T == 20:
            ms = e0.elapsed_time(e1) / a.train_steps
        after = val_loss()
        rec = {"val_loss_unit_weights": before, "val_loss_trained": after,
               "weights_mean_per_type": wt.detach().mean(dim=0).tolist()}
        for name, wv in (("plain", torch.ones((T, 3), device=dev)), ("weighted", wt.detach())):
            soft, _ = dec_ev.wbp_forward(llr_ev, s_ev, wv, keep_tape=False)
            bits = (soft < 0).to(torch.uint8)
            rec[f"fer_{name}"] = float((bits != x_ev).any(dim=1).float().mean())
            rec[f"ber_{name}"] = float((bits != x_ev).float().mean())
        curve[f"T{T}"] = rec
    line = {
        "metric": "weighted-BP training throughput (forward + adjoint), codeword bits per second",
        "value": B_tr * n_tr / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": world, "steps": a.train_steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded MET ensemble, BIAWGN samples)",
        "config": {"workload": f"rate 0.1, n={n_tr}, {B_tr} codewords, T=10/15/20, checkpoint every {k}, "
                               f"Tx3 weights, Adam lr 0.003, beta={beta}; evaluated at n={n_ev}, {B_ev} codewords"},
        "iterations_to_fer": curve,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def time_steps(step, steps: int, warmup: int, stream, barrier) -> float:
    """Device time (ms) of `steps` calls after `warmup` untimed ones, bracketed
    by a barrier and a synchronize on both sides."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1)


def kernel_summary(kt: dict, st: dict, msg: str, batch: int, iters: int, steps: int, ms_step: float,
                   peak: float, schedule: str = "flooding") -> dict:
    """Check-pass and whole-decode roofline fractions from the library's
    per-iteration CUDA events (one timed region = one pass; with the layered
    schedule the pass is the iteration's layers)."""
    check_b, iter_b = algorithmic_bytes(st, msg, schedule)
    check_ms = kt["check_ms"] / max(1, kt["check_timed"])
    var_ms = kt["var_ms"] / max(1, kt["var_timed"])
    achieved = check_b * batch / (check_ms * 1e-3) / 1e9
    decode_gbs = iter_b * batch * iters / (ms_step * 1e-3) / 1e9
    return {"achieved": achieved, "frac": achieved / peak, "pass_ms": check_ms, "var_update_ms": var_ms,
            "algorithmic_bytes_per_pass": check_b * batch,
            "algorithmic_bytes_per_iteration": iter_b * batch,
            "decode_gbs": decode_gbs, "frac_decode": decode_gbs / peak,
            "check_launches_per_pass": kt["check_launches"] / max(1, iters * steps),
            "timed_passes": kt["check_timed"],
            "share_check": check_ms * iters / max(1e-9, ms_step)}


def sub_record(rate: float, msg: str, a, rank: int, dev, dist, barrier, peak: float,
               vn_update: str = "gather", schedule: str = "flooding", check_rule: str = "sum_product",
               structured: bool = False) -> dict:
    """One more fixed-iteration workload measured like the headline (device-
    resident inputs, CUDA events, max over ranks), with fewer steps.
    structured: the layer-structured ensemble, decoded with its own layers."""
    import torch
    import paper_1711_01783_gb300 as mld
    from synthetic import make_workload, preset_graph_layered
    iters = DEFAULT_ITERS[rate]
    graph = preset_graph_layered(rate, a.n, 2) if structured else None
    wl = make_workload(rate, a.n, a.batch, 2, rank_data_seed(rank), beta=a.beta, graph=graph)
    g = mld.Graph.from_edges(wl.graph)
    if schedule == "layered":
        g.set_layers(wl.graph.meta["layer_of_check"] if structured else None)
    dec = mld.Decoder(g, a.batch, msg_dtype=msg, vn_update=vn_update, schedule=schedule, check_rule=check_rule)
    y = torch.from_numpy(wl.y).to(dev)
    sig = torch.from_numpy(wl.sigma).to(dev)
    syn = torch.from_numpy(wl.s).to(dev)
    out = dict(bits=torch.empty((a.batch, a.n), dtype=torch.uint8, device=dev), post=None,
               converged=torch.empty(a.batch, dtype=torch.uint8, device=dev),
               iters_used=torch.empty(a.batch, dtype=torch.int32, device=dev))
    stream = torch.cuda.current_stream()
    step = lambda: dec.decode_y(y, sig, syn, iters, out=out)  # noqa: E731
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    dec.timing(TIMING_EVERY)
    dec.read_timing()
    ms = time_steps(step, a.sub_steps, 0, stream, barrier)
    dec.timing(0)
    kt = dec.read_timing()
    ms_max, launches = reduce_over_ranks(dist, ms, kt["check_launches"] + kt["var_launches"]
                                         + kt["syndrome_launches"] + kt["layout_launches"], dev)
    world = dist.get_world_size() if dist is not None else 1
    ks = kernel_summary(kt, g.stats, msg, a.batch, iters, a.sub_steps, ms_max / a.sub_steps, peak, schedule)
    conv = int(out["converged"].sum().item())
    rec = {"value": job_throughput(world, a.batch, a.n, a.sub_steps, ms_max), "unit": UNIT,
           "ms_per_step": ms_max / a.sub_steps, "steps": a.sub_steps, "warmup": 3,
           "rate": rate, "iters": iters, "msg_storage": msg, "vn_update": vn_update, "schedule": schedule,
           "check_rule": check_rule, "ensemble": "layer-structured" if structured else "plain",
           "n_layers": g.layers()[1] if schedule == "layered" else None,
           "gpu_launches": launches,
           "frames_converged": conv, "fer": 1.0 - conv / a.batch}
    rec.update({k: ks[k] for k in ("frac", "frac_decode", "pass_ms", "var_update_ms", "share_check")})
    dec.close()
    g.close()
    return rec


def md_frontend(a, dev, peak: float, steps: int = 10) -> dict:
    """Multidimensional-reconciliation kernels on the benchmark's shape
    (64 x 10^6 samples): bytes each must move (Bob: y, bits in; alpha, |y|
    out = 9.5 B per sample; Alice: x, alpha, |y| in, LLR out = 12.5 B per
    sample) over their CUDA-event time."""
    import torch
    import paper_1711_01783_gb300 as mld
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    x = torch.randn((a.batch, a.n), device=dev, generator=g)
    y = x + 0.8 * torch.randn((a.batch, a.n), device=dev, generator=g)
    bits = torch.randint(0, 2, (a.batch, a.n), device=dev, dtype=torch.uint8, generator=g)
    nv = torch.full((a.batch,), 0.64, device=dev)
    out = {}
    for name, fn, per in (("bob", lambda: mld.md_bob(y, bits), 9.5),
                          ("alice", lambda: mld.md_alice(x, al, yn, nv), 12.5)):
        if name == "alice":
            al, yn = mld.md_bob(y, bits)
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gbs = per * a.batch * a.n / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "GB/s": gbs, "frac": gbs / peak, "bytes_per_sample": per,
                     "Msamples/s": a.batch * a.n / (ms * 1e-3) / 1e6}
    return out


def peg_record(dev, n: int = 4096, frames: int = 256, beta: float = 0.42, cap: int = 80) -> dict:
    """PEG construction of the rate-0.1 family on the host (mld_peg_edges)
    and what it buys: frame error rate of the PEG code and of the socket-
    permutation code of the same degrees on the same kind of channel, decoded
    on the GPU (float messages, early termination)."""
    import torch
    import paper_1711_01783_gb300 as mld
    from synthetic import biawgn_observe, bob_syndrome, preset_graph, random_bits, sigma_for_beta
    from types import SimpleNamespace
    rate, core, d2 = 0.1, 0.2, 20
    n_c = int(round(core * n))
    deg = np.zeros((3, n), np.int64)
    deg[0, :n_c] = 3
    deg[0, :int(round(0.4 * n_c))] = 2
    deg[1, :n_c] = d2
    deg[2, n_c:] = 1
    m1, m2 = n_c - int(round(rate * n)), n - n_c
    mask = np.concatenate([np.full(m1, 1), np.full(m2, 6)])
    t0 = time.perf_counter()
    ev, ec, et = mld.peg_edges(deg, mask, np.random.default_rng(1).permutation(m1 + m2))
    t_peg = time.perf_counter() - t0
    graphs = {"peg": SimpleNamespace(n_vn=n, n_cn=m1 + m2, edge_vn=ev, edge_cn=ec, edge_type=et),
              "socket": preset_graph(rate, n, 1)}
    sig = sigma_for_beta(rate, beta)
    res = {"n": n, "edges": int(ev.shape[0]), "construction_s": t_peg,
           "construction_kedges_per_s": ev.shape[0] / t_peg / 1e3,
           "fer_workload": f"{frames} frames, beta={beta}, cap {cap}, early termination, f32"}
    for name, g in graphs.items():
        x = random_bits(frames, n, 77)
        s = bob_syndrome(g, x)
        y = biawgn_observe(x, sig, 77)
        G = mld.Graph.from_edges(g)
        out = mld.Decoder(G, frames, msg_dtype="f32").decode_y(
            torch.from_numpy(y).to(dev), torch.full((frames,), sig, device=dev), torch.from_numpy(s).to(dev),
            cap, early_term=True)
        res[f"fer_{name}"] = 1.0 - float(out["converged"].float().mean())
    return res


def rule_comparison(a, dev, barrier, beta: float = 0.30, cap: int = 100, steps: int = 5) -> dict:
    """Sum-product against offset min-sum where both decode: rate 0.1,
    n = 10^6, 64 codewords, early termination (cap 100), flooding schedule."""
    import torch
    import paper_1711_01783_gb300 as mld
    from synthetic import make_workload
    wl = make_workload(0.1, a.n, a.batch, 2, 8600, beta=beta)
    g = mld.Graph.from_edges(wl.graph)
    y = torch.from_numpy(wl.y).to(dev)
    sig = torch.from_numpy(wl.sigma).to(dev)
    syn = torch.from_numpy(wl.s).to(dev)
    x = torch.from_numpy(wl.x).to(dev)
    stream = torch.cuda.current_stream()
    res = {"workload": f"rate 0.1, n={a.n}, {a.batch} codewords, beta={beta}, early termination, cap {cap}, "
                       f"{a.msg} messages, flooding; min-sum offset {mld.DEFAULT_MS_OFFSET} nats"}
    for rule in ("sum_product", "min_sum"):
        dec = mld.Decoder(g, a.batch, msg_dtype=a.msg, check_rule=rule)
        holder = {}

        def step():
            holder["o"] = dec.decode_y(y, sig, syn, cap, early_term=True, want_post=True)
        for _ in range(2):
            step()
        ms = time_steps(step, steps, 0, stream, barrier) / steps
        o = holder["o"]
        frame_err = (o["bits"] != x).any(dim=1) | (o["converged"] == 0)
        res[rule] = {"ms_per_decode": ms, "value": a.batch * a.n / (ms * 1e-3) / 1e6, "unit": UNIT,
                     "mean_iters": float(o["iters_used"].float().mean()), "max_iters": int(o["iters_used"].max()),
                     "fer": float(frame_err.float().mean()), "frames": a.batch}
        dec.close()
    g.close()
    return res


def schedule_comparison(a, dev, barrier, betas=(0.40, 0.42), cap: int = 100, steps: int = 5,
                        structured: bool = False) -> dict:
    """Flooding against the layered schedule where frames converge: rate 0.1,
    n = 10^6, 64 codewords, early termination with a cap of 100 iterations.
    Per (beta, schedule): decode time, decoded Mbit/s, mean iterations, FER.
    structured: the layer-structured ensemble, layered with its own groups."""
    import torch
    import paper_1711_01783_gb300 as mld
    from synthetic import make_workload, preset_graph, preset_graph_layered
    graph = preset_graph_layered(0.1, a.n, 2) if structured else preset_graph(0.1, a.n, 2)
    g = mld.Graph.from_edges(graph)
    g.set_layers(graph.meta["layer_of_check"] if structured else None)
    n_layers = g.layers()[1]
    stream = torch.cuda.current_stream()
    how = "the ensemble's own check groups" if structured else "the library's default layering"
    res = {"workload": f"rate 0.1, n={a.n}, {a.batch} codewords, early termination, cap {cap}, "
                       f"{a.msg} messages, {'layer-structured' if structured else 'plain'} ensemble; "
                       f"layered: {how} ({n_layers} layers)"}
    for beta in betas:
        wl = make_workload(0.1, a.n, a.batch, 2, 7000, beta=beta, graph=graph)
        y = torch.from_numpy(wl.y).to(dev)
        sig = torch.from_numpy(wl.sigma).to(dev)
        syn = torch.from_numpy(wl.s).to(dev)
        x = torch.from_numpy(wl.x).to(dev)
        # flooding without soft output checks the syndrome inside the next
        # check pass (host-driven loop); with soft output, and layered, the
        # iterations run in the device loop
        for sched, post in (("flooding", False), ("flooding", True), ("layered", False)):
            dec = mld.Decoder(g, a.batch, msg_dtype=a.msg, schedule=sched)
            holder = {}

            def step():
                holder["o"] = dec.decode_y(y, sig, syn, cap, early_term=True, want_post=post)
            for _ in range(2):
                step()
            ms = time_steps(step, steps, 0, stream, barrier) / steps
            o = holder["o"]
            frame_err = (o["bits"] != x).any(dim=1) | (o["converged"] == 0)
            res[f"beta{beta}_{sched}{'_soft' if post else ''}"] = {
                "ms_per_decode": ms, "value": a.batch * a.n / (ms * 1e-3) / 1e6, "unit": UNIT,
                "mean_iters": float(o["iters_used"].float().mean()),
                "max_iters": int(o["iters_used"].max()),
                "fer": float(frame_err.float().mean()), "frames": a.batch}
            dec.close()
    g.close()
    return res


def main():
    a = parse()
    if a.workload == "wbp":
        if a.beta == 0.90:
            a.beta = 0.40
        run_wbp(a, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                int(os.environ.get("LOCAL_RANK", "0")))
        return
    if a.workload == "uneven":
        if a.batch == 64:
            a.batch = 96
        if a.iters is None:
            a.iters = 0
        run_uneven(a, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                   int(os.environ.get("LOCAL_RANK", "0")))
        return
    if a.iters is None:
        a.iters = DEFAULT_ITERS.get(a.rate, 100)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from synthetic import make_workload
    seed_graph = 2  # 1 + index of the n = 10^6 workload

    if a.impl == "reference":
        if rank != 0:
            return
        wl = make_workload(a.rate, a.n, min(a.batch, host_cores()), seed_graph, 1000, beta=a.beta)
        run_reference(a, wl)
        return

    import torch
    import paper_1711_01783_gb300 as mld

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    wl = make_workload(a.rate, a.n, a.batch, seed_graph, rank_data_seed(rank), beta=a.beta)
    g = mld.Graph.from_edges(wl.graph)
    dec = mld.Decoder(g, a.batch, msg_dtype=a.msg, slab_width=a.slab, vn_update=a.vn_update, staging=a.staging)
    st = g.stats
    y = torch.from_numpy(wl.y).to(dev)
    sig = torch.from_numpy(wl.sigma).to(dev)
    syn = torch.from_numpy(wl.s).to(dev)
    out = dict(bits=torch.empty((a.batch, a.n), dtype=torch.uint8, device=dev), post=None,
               converged=torch.empty(a.batch, dtype=torch.uint8, device=dev),
               iters_used=torch.empty(a.batch, dtype=torch.int32, device=dev))
    stream = torch.cuda.current_stream()

    def step():
        dec.decode_y(y, sig, syn, a.iters, out=out)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs -----------------------------
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    dec.timing(TIMING_EVERY)
    dec.read_timing()
    clocks.start()
    ms = time_steps(step, a.steps, 0, stream, barrier)
    clk = clocks.stop()
    dec.timing(0)
    kt = dec.read_timing()
    ms_max, launches = reduce_over_ranks(dist, ms, kt["check_launches"] + kt["var_launches"]
                                         + kt["syndrome_launches"] + kt["layout_launches"], dev)
    value = job_throughput(world, a.batch, a.n, a.steps, ms_max)
    frames_converged = int(out["converged"].sum().item())

    # ---- end to end through the host-pointer path ---------------------------
    e2e = None
    if not a.no_e2e:
        y_h = torch.from_numpy(wl.y).pin_memory()
        sig_h = torch.from_numpy(wl.sigma).pin_memory()
        s_h = torch.from_numpy(wl.s).pin_memory()
        out_h = dict(bits=torch.empty((a.batch, a.n), dtype=torch.uint8).pin_memory(), post=None,
                     converged=torch.empty(a.batch, dtype=torch.uint8).pin_memory(),
                     iters_used=torch.empty(a.batch, dtype=torch.int32).pin_memory())
        dec.decode_y(y_h, sig_h, s_h, a.iters, out=out_h)  # warm the path
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(a.e2e_steps):
            dec.decode_y(y_h, sig_h, s_h, a.iters, out=out_h)  # waits for the stream
        h1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        te = torch.tensor([max(h0.elapsed_time(h1), wall * 1e3)], dtype=torch.float64, device=dev)
        if dist is not None:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        h2d = a.batch * a.n * 4 + a.batch * 4 + a.batch * st["n_cn"]
        d2h = a.batch * a.n + a.batch + 4 * a.batch
        e2e = {"value": world * a.batch * a.n * a.e2e_steps / (float(te.item()) * 1e-3) / 1e6,
               "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- roofline of the check update ---------------------------------------
    # One check-update pass per iteration (one launch per check class); its
    # time is the sum of those launches, measured by the library's CUDA events
    # on the launching stream during the timed region.
    peak, peak_kind = measured_peak_hbm()
    ks = kernel_summary(kt, st, a.msg, a.batch, a.iters, a.steps, ms_max / a.steps, peak)
    # the counters were taken on the gather variant's check kernel
    tpb = CHECK_PASS_TRAFFIC_PER_CW_BIT.get((a.rate, a.msg)) if a.vn_update == "gather" else None
    roofline = {"bound": "hbm", "achieved": ks["achieved"], "peak": peak, "unit": "GB/s",
                "frac": ks["frac"], "traffic": tpb * a.batch * a.n if tpb else None,
                "kernel": "k_check_update (one pass = all check classes of one iteration)",
                "peak_kind": peak_kind}
    roofline.update({k: v for k, v in ks.items() if k not in ("achieved", "frac")})
    dec.close()
    g.close()

    # ---- sub-records: the same measurement on the other storage type and
    # the other rates (fewer steps each) --------------------------------------
    sub = {}
    if not a.no_sub and a.n == 1_000_000 and a.batch == 64:
        other = "f32" if a.msg == "f16" else "f16"
        sub[f"rate{a.rate}_{other}"] = sub_record(a.rate, other, a, rank, dev, dist, barrier, peak, a.vn_update)
        for r in (0.1, 0.05, 0.02):
            if r != a.rate:
                sub[f"rate{r}_{a.msg}"] = sub_record(r, a.msg, a, rank, dev, dist, barrier, peak, a.vn_update)
        vo = "accumulate" if a.vn_update == "gather" else "gather"
        for m in (a.msg, other):
            sub[f"rate{a.rate}_{m}_{vo}"] = sub_record(a.rate, m, a, rank, dev, dist, barrier, peak, vo)
        sub[f"rate{a.rate}_{a.msg}_layered"] = sub_record(a.rate, a.msg, a, rank, dev, dist, barrier, peak,
                                                          "gather", "layered")
        sub["schedules_converging"] = schedule_comparison(a, dev, barrier)
        sub[f"rate{a.rate}_{a.msg}_layered_structured"] = sub_record(a.rate, a.msg, a, rank, dev, dist, barrier,
                                                                     peak, "gather", "layered", structured=True)
        sub["schedules_converging_structured"] = schedule_comparison(a, dev, barrier, betas=(0.40, 0.42),
                                                                     structured=True)
        sub[f"rate{a.rate}_{a.msg}_minsum"] = sub_record(a.rate, a.msg, a, rank, dev, dist, barrier, peak,
                                                         check_rule="min_sum")
        sub["rules_converging"] = rule_comparison(a, dev, barrier)
        sub["md_frontend"] = md_frontend(a, dev, peak)
        sub["peg"] = peg_record(dev)
        sub["uneven"] = uneven_record(96, a.beta, a.msg, 3, 1, rank, dev)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(wl, a)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded MET ensemble, BIAWGN samples)", "config": workload_config(a),
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu, "clocks": clk,
            "frames_converged": frames_converged, "fer": 1.0 - frames_converged / a.batch,
            "sub": sub,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
