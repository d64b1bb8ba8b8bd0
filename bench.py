#!/usr/bin/env python
"""Benchmark: space-time vertices+edges per second of the continuous-time
loop-cluster update of the S=1/2 antiferromagnetic Heisenberg chain.

One step = one loop update (insertion, linking, union-find, flip, rewrite,
measurement) of a single chain with L = 2^16 sites at beta = 2^12 (about
1.9e8 graph vertices, 3.7e8 world-line fragments per update).  V+E counts the
paper's graph: fragments + 2 x vertices (Sec. 4.4).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own chain (seed 1 + rank): independent Markov
chains, weak scaling, no collective on the data path.  `--impl reference`
times the CPU oracle (the plain restatement of the method under oracle/) on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (L, beta, thermalization updates before warm-up)
    "L65536_beta4096": (1 << 16, float(1 << 12), 6),
    "L1048576_beta1024": (1 << 20, float(1 << 10), 4),
    "L64_beta16": (64, 16.0, 1000),
    "L16384_beta4096": (1 << 14, float(1 << 12), 6),
}
DEFAULT_WORKLOAD = "L65536_beta4096"
# Oracle sample of the same workload: same beta, fewer sites.
ORACLE_SAMPLE_L = 1024
KERNELS_PER_UPDATE = 11
RECORD_BYTES = 104


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def phase_bytes(rec, ncell, L):
    """Algorithmic bytes per phase of one update from its counts."""
    n = float(rec["n"])
    no, nn = float(rec["n_off_old"]), float(rec["n_off_new"])
    return {
        # read old operator times, write vertex time/flag/parent, cell offsets,
        # clear three bitmaps
        "insert": 8 * no + 13 * n + 8 * ncell + 3 * n / 8,
        "cut": 16.0 * L,
        # vertex times once, predecessor links out, flag RMW, two parent reads per edge
        "link_union": 26 * n + 4 * ncell,
        # parent read + root write + three bitmaps
        "loop_ids": 8.375 * n,
        # links, flags, two roots, three times per vertex, new flag
        "loop_props": 42 * n + 4 * ncell,
        "op_offsets": 16 * (ncell / 128.0),
        # flags, new operator times read + written, cell offsets
        "op_rewrite": n + 16 * nn + 8 * ncell,
        "spin_rewrite": 2.0 * L + 64.0,
    }


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample(beta, steps, warmup, L=ORACLE_SAMPLE_L):
    """Times the keyed CPU oracle on L sites at the workload's beta."""
    from oracle import orc
    p = orc.params(L, beta, seed=1)
    st = orc.neel(p)
    orc.keyed_run(p, 0, warmup, st)
    t0 = time.perf_counter()
    recs = orc.keyed_run(p, warmup, steps, st)
    dt = time.perf_counter() - t0
    ve = float((recs["n_seg"] + 2 * recs["n"]).sum())
    return ve / dt, dt, recs


def run_reference(args, world, rank):
    L, beta, _ = WORKLOADS[args.workload]
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    value, dt, recs = oracle_sample(beta, steps, warm)
    line = {
        "impl": "reference", "metric": "space-time vertices+edges/s per loop update", "value": value,
        "unit": "V+E/s", "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"S=1/2 AFM Heisenberg chain, J=1, L={L}, beta={beta:g}, single chain; "
                               f"CPU oracle sample L={ORACLE_SAMPLE_L} at the same beta",
                   "L": L, "beta": beta, "sample_L": ORACLE_SAMPLE_L},
        "cpu_baseline": {"value": value, "unit": "V+E/s", "cores": 1, "kind": "oracle",
                         "sample": f"keyed oracle, L={ORACLE_SAMPLE_L}, beta={beta:g}, {steps} updates after {warm}"},
        "e2e": {"value": value, "unit": "V+E/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_1810_07485_gb300 import lcqmc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    L, beta, therm = WORKLOADS[args.workload]
    stream = torch.cuda.Stream()
    ch = lcqmc.Chain(L, beta, seed=1 + rank, stream=stream.cuda_stream)
    geo = ch.geometry()
    # thermalization from the Neel state, then W warm-up updates (untimed)
    ch.update(therm + args.warmup)
    ch.sync()
    ch.records()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # -- device-timed region: K updates on the chain's stream -----------------
    clk = Clocks(local)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ch.update(args.steps)
    e1.record(stream)
    ch.sync()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    recs = ch.records()
    ve_local = float((recs["n_seg"] + 2 * recs["n"]).sum())
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    v = torch.tensor([ve_local], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    ve_tot = float(v.item())
    value = ve_tot / (ms_max * 1e-3)

    # -- end to end through the public API: update + record readback per step --
    barrier()
    t0 = time.perf_counter()
    ve_e2e = 0.0
    for _ in range(args.steps):
        ch.update(1)
        r = ch.records()
        ve_e2e += float((r["n_seg"] + 2 * r["n"]).sum())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    ve2 = torch.tensor([ve_e2e], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
        dist.all_reduce(ve2, op=dist.ReduceOp.SUM)
    e2e_value = float(ve2.item()) / float(te.item())

    # -- per-phase device times (CUDA events between phases, same stream) -------
    nph = min(10, max(3, args.steps))
    ch.set_phase_timing(True)
    ch.update(nph)
    ch.sync()
    ph = ch.phase_times()
    pr = ch.records()
    ch.set_phase_timing(False)
    nb = {k: 0.0 for k in ph}
    for r in pr:
        for k, b in phase_bytes(r, geo.ncell, L).items():
            nb[k] += b
    dom = max(ph, key=lambda k: ph[k])
    peak, peak_kind = load_peaks()
    achieved = nb[dom] / (ph[dom] * 1e-3) / 1e9 if ph[dom] > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom, "peak_kind": peak_kind,
                "phase_ms_per_update": {k: ph[k] / nph for k in ph},
                "phase_frac_of_hbm": {k: (nb[k] / (ph[k] * 1e-3) / 1e9) / peak if ph[k] > 0 else None for k in ph}}

    cpu = None
    if rank == 0:
        val, dt, _ = oracle_sample(beta, 4, 2)
        cpu = {"value": val, "unit": "V+E/s", "cores": 1, "kind": "oracle",
               "sample": f"keyed oracle, L={ORACLE_SAMPLE_L}, beta={beta:g}, 4 updates after 2 ({dt:.1f} s)"}
    mean_n = float(recs["n"].mean())
    line = {
        "metric": "space-time vertices+edges/s per loop update", "value": value, "unit": "V+E/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"S=1/2 AFM Heisenberg chain, J=1, L={L}, beta={beta:g}, one chain per GPU "
                               f"(seed 1+rank), Neel start, {therm}+{args.warmup} untimed updates",
                   "L": L, "beta": beta, "vertices_per_update": mean_n,
                   "l2": "inputs larger than L2 (state and per-update graph are several GB)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "V+E/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": RECORD_BYTES},
        "gpu_launches": KERNELS_PER_UPDATE * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    ch.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    args = ap.parse_args()
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
