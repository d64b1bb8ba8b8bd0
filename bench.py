#!/usr/bin/env python
"""Benchmark: space-time vertices+edges per second of the continuous-time
loop-cluster update of the S=1/2 antiferromagnetic Heisenberg chain.

One step = one loop update (insertion, linking, union-find, flip, rewrite,
measurement) of a single chain with L = 2^20 sites at beta = 2^10 (about
7.4e8 graph vertices, 1.5e9 world-line fragments per update), the largest
single-chain configuration of the benchmark list.  V+E counts the paper's
graph: fragments + 2 x vertices (Sec. 4.4).  The same line carries the
batched form beside it: 4096 uneven chains, 100 updates each, packed per
phase and replayed from a CUDA graph, against the same chains launched one
at a time (per-chain completion p50/p99, results identical); and the served
form: Poisson request streams at 20 and 50 requests/s (latency p50/p99 per
block of 50 updates, V+E/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-batched]
  python bench.py --mode batched [--chains C --updates U]   (the batched form alone)
  python bench.py --mode served [--requests R --rate Hz]    (request stream)

Under torchrun each rank runs its own chain (seed 1 + rank): independent Markov
chains, weak scaling, no collective on the data path.  `--impl reference`
times the CPU oracle (the plain restatement of the method under oracle/) on a
bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (L, beta, thermalization updates before warm-up)
    "L65536_beta4096": (1 << 16, float(1 << 12), 6),
    "L1048576_beta1024": (1 << 20, float(1 << 10), 4),
    "L64_beta16": (64, 16.0, 1000),
    "L16384_beta4096": (1 << 14, float(1 << 12), 6),
}
DEFAULT_WORKLOAD = "L1048576_beta1024"
# Oracle sample of the same workload: the same beta, fewer sites, started from
# a thermalized state (its resident set, about 1 GB, is far beyond the caches).
ORACLE_SAMPLE_L = 8192
# The batched form beside the single chain (the benchmark list's batched
# configuration): chains, updates per chain, device budget of one wave.
BATCH_CHAINS, BATCH_UPDATES, BATCH_BUDGET_GB = 4096, 100, 150.0
# The served form beside them: request streams at a light and at a saturating
# rate (latency per update block, p50 / p99, and V+E/s).
SERVED_RATES, SERVED_SECONDS, SERVED_LMAX = (20.0, 50.0), 10.0, 4096
KERNELS_PER_UPDATE = 12
# DRAM bytes per vertex of each phase's kernels (DRAM bytes of one ncu
# capture at L=16384, beta=4096 -- dram__bytes.sum.per_second x
# gpu__time_duration.sum -- divided by that update's vertex count;
# profiles/topkernels_L16384_beta4096.md), valid for the kernel source with
# this sha1 only.  The same tile shapes and per-vertex work hold at
# L=2^20, beta=2^10, so the full launch's traffic is this figure times its
# vertex count.  With the temporal moment on, the loop-properties and
# operator-rewrite kernels differ and have no entry.  The compression kernel
# was captured from the first source listed; the other kernels from an
# earlier one that differs from it only in S >= 1 staging.  The second
# source flattens the linking kernel's shared-memory forest by root walks
# instead of pointer jumping (the same global loads and stores); the third
# also stages the loop-properties kernel's ticks before its first barrier
# (the same loads).
TRAFFIC_PER_VERTEX = {"insert": 13.5, "link_union": 26.7, "loop_ids": 6.6, "loop_props": 25.0,
                      "op_rewrite": 14.8}
TRAFFIC_PER_VERTEX_TEMPORAL = {k: v for k, v in TRAFFIC_PER_VERTEX.items() if k not in ("loop_props", "op_rewrite")}
TRAFFIC_KERNELS_SHA1 = ("2bcd43154d5dbe04227fe45c685d4a3e85f64f03", "7f31eb08d2f1539aba0a26c771a385c99bf920e5",
                        "fa8691b2a774215fa52e6afef9cb78fd57fd7843")


# DRAM bytes per launch of each Swendsen-Wang phase at L = 8192, K = K_c (one
# ncu capture; profiles/sw_L8192_Kc.md), valid for sw.cu with this sha1 only.
SW_TRAFFIC = {"tile_bonds_uf": 294.5e6, "boundary_merge": 173.2e6, "roots_flip": 444.6e6,
              "open_sizes_record": 24.4e6}
# the profiled source, and the current one, whose kernels are the same (it
# only adds an NVTX range around the host's update loop)
SW_TRAFFIC_SHA1 = ("dadb5c42ae8fdb32d88e4c88ee578722234bd1c4", "e7d41349163f593cc5c0ea1dba9a5d2e5e8bd8bb")


def kernels_sha1(name="kernels.cu"):
    import hashlib
    with open(os.path.join(ROOT, "paper_1810_07485_gb300", "csrc", name), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def host_cpu():
    """The host's CPU model and logical core count (for the CPU baseline)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def phase_bytes(rec, ncell, L):
    """Algorithmic bytes per phase of one update from its counts: every datum
    the phase must read or write, counted once (re-reads served by caches are
    not counted)."""
    n = float(rec["n"])
    no, nn = float(rec["n_off_old"]), float(rec["n_off_new"])
    return {
        # old operator times and offsets in; vertex time/flag/cell and cell
        # offsets out; four per-vertex bitmaps cleared
        "insert": 8 * no + 10 * n + 8 * ncell + n / 2,
        "cut": 16.0 * L,
        # vertex time and cell in, predecessor links and parent forest out,
        # flag read-modify-write, cell offsets
        "link_union": 23 * n + 4 * ncell,
        # parent read, root written, open-mark / open-root / flip bitmaps
        "loop_ids": 8.375 * n,
        # cell, links, flag read+write, parent, time, flip bits; new-operator
        # counts per cell
        "loop_props": 23.125 * n + 4 * ncell,
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


def chain_seed(rank):
    """Each rank runs its own independent chain: the seed keys every random
    number of the update, so distinct seeds give distinct Markov chains."""
    return 1 + rank


def over_ranks(world, elapsed, units, device):
    """Whole-job figures: the slowest rank's elapsed time (max) and the units
    processed by all ranks (sum).  With one rank, the inputs unchanged."""
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    v = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), float(v.item())


def oracle_sample(beta, steps, warmup, L=ORACLE_SAMPLE_L, state=None):
    """Times the keyed CPU oracle on L sites at the workload's beta: `steps`
    updates after `warmup` untimed ones, from the Neel state or from
    state = (s0, op_ptr, op_tau, sweep)."""
    from oracle import orc
    p = orc.params(L, beta, seed=1)
    if state is None:
        st, sweep0 = orc.neel(p), 0
    else:  # a copy: the oracle updates its state in place
        st, sweep0 = orc.State(state[0], state[1], state[2]).copy(), int(state[3])
    orc.keyed_run(p, sweep0, warmup, st)
    t0 = time.perf_counter()
    recs = orc.keyed_run(p, sweep0 + warmup, steps, st)
    dt = time.perf_counter() - t0
    ve = float((recs["n_seg"] + 2 * recs["n"]).sum())
    return ve / dt, dt, recs


def oracle_sample_all_cores(beta, steps, warmup, L=ORACLE_SAMPLE_L, procs=None, state=None):
    """The oracle on every host core at once, one independent chain per core
    (the paper's independent-chain strategy)."""
    from oracle import timing
    return timing.all_cores_sample(L, beta, steps, warmup, procs, state=state)


def gpu_thermalized_sample(beta, L=ORACLE_SAMPLE_L, updates=20, seed=1):
    """A thermalized state of the oracle's sample chain (L sites at the
    workload's beta), made by the GPU update: (s0, op_ptr, op_tau, sweep)."""
    from paper_1810_07485_gb300 import lcqmc
    ch = lcqmc.Chain(L, beta, seed=seed)
    try:
        ch.update(updates)
        s0, ptr, tau = ch.export_config()
        return s0, ptr.astype(np.int64), tau, int(ch.geometry().sweep)
    finally:
        ch.close()


def workload_name(L, beta):
    return f"S=1/2 AFM Heisenberg chain, J=1, L={L}, beta={beta:g}, single chain, FP64 tau, int32 vertex ids"


def run_reference(args, world, rank):
    """The CPU oracle on the host cores, rank 0 only: W untimed updates from
    the Neel state (thermalization), then K timed ones, on the sample chain."""
    L, beta, _ = WORKLOADS[args.workload]
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    sL = min(L, ORACLE_SAMPLE_L)
    value, dt, recs = oracle_sample(beta, steps, warm, L=sL)
    sample = (f"keyed oracle on one core, L={sL} at beta={beta:g} (a bounded sample of the workload), "
              f"{steps} timed updates after {warm} from the Neel state")
    line = {
        "impl": "reference", "metric": "space-time vertices+edges/s per loop update", "value": value,
        "unit": "V+E/s", "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(L, beta) + f"; CPU oracle sample L={sL} at the same beta",
                   "L": L, "beta": beta, "sample_L": sL},
        "cpu_baseline": {"value": value, "unit": "V+E/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": sample},
        "e2e": {"value": value, "unit": "V+E/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_sw_reference(args, world, rank):
    """Reference arm of the Swendsen-Wang mode: the CPU oracle on rank 0."""
    if rank != 0:
        return
    value, dt = sw_oracle_sample(args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": "Swendsen-Wang site updates/s (2D Ising, union-find benchmark)",
        "value": value, "unit": "site updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps * (SW_L / SW_ORACLE_L) ** 2,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"Swendsen-Wang, L={SW_L}, K=K_c; CPU oracle sample L={SW_ORACLE_L}",
                   "L": SW_L, "K": SW_K, "sample_L": SW_ORACLE_L},
        "cpu_baseline": {"value": value, "unit": "site updates/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": f"Swendsen-Wang oracle, L={SW_ORACLE_L}, {args.steps} updates after "
                                   f"{args.warmup}"},
        "e2e": {"value": value, "unit": "site updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_1810_07485_gb300 import lcqmc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    L, beta, therm = WORKLOADS[args.workload]
    stream = torch.cuda.Stream()
    ch = lcqmc.Chain(L, beta, seed=chain_seed(rank), stream=stream.cuda_stream)
    if args.temporal:
        ch.set_temporal(True)
    geo = ch.geometry()
    # thermalization from the Neel state, the block sizes of the union-find
    # phases tuned (8 trials of 2 updates), then W warm-up updates (untimed)
    ch.update(therm)
    tuning = ch.autotune(2)
    ch.update(args.warmup)
    ch.sync()
    ch.records()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # -- device-timed region: K updates on the chain's stream -----------------
    # An update that outgrows its buffers stops, and lcqmc_sync grows them and
    # runs it again after the end event: the window would miss that work.  The
    # window is timed again (with the grown buffers) if that happened.
    clk = Clocks(local)
    retimed = 0
    for attempt in range(3):
        r0 = ch.geometry().replays
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ch.update(args.steps)
        e1.record(stream)
        ch.sync()
        barrier()
        recs = ch.records()[-args.steps:]
        if ch.geometry().replays == r0:
            break
        retimed += 1
        log(f"bench: {ch.geometry().replays - r0} update(s) re-run after buffer growth inside the timed "
            f"window; timing again")
    else:
        raise SystemExit("bench: buffer growth inside every timed window")
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    ve_local = float((recs["n_seg"] + 2 * recs["n"]).sum())
    ms_max, ve_tot = over_ranks(world, ms, ve_local, "cuda")
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
    e2e_max, ve2_tot = over_ranks(world, e2e_s, ve_e2e, "cuda")
    e2e_value = ve2_tot / e2e_max

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
    traffic = None  # bytes per launch, only while the kernels are the profiled ones
    tpv = TRAFFIC_PER_VERTEX_TEMPORAL if args.temporal else TRAFFIC_PER_VERTEX
    if kernels_sha1() in TRAFFIC_KERNELS_SHA1 and dom in tpv:
        traffic = tpv[dom] * float(pr["n"].mean())
    upd_ms = sum(ph.values())
    upd_achieved = sum(nb.values()) / (upd_ms * 1e-3) / 1e9 if upd_ms > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "algorithmic_bytes": nb[dom] / nph, "kernel": dom, "peak_kind": peak_kind,
                "scope": "frac is the dominant phase's; whole_update covers every phase of the update",
                "whole_update": {"achieved": upd_achieved, "frac": upd_achieved / peak,
                                 "algorithmic_bytes": sum(nb.values()) / nph, "ms": upd_ms / nph},
                "phase_ms_per_update": {k: ph[k] / nph for k in ph},
                "phase_frac_of_hbm": {k: (nb[k] / (ph[k] * 1e-3) / 1e9) / peak if ph[k] > 0 else None for k in ph}}
    mean_n = float(recs["n"].mean())
    ch.close()

    cpu = None
    if rank == 0:
        sL = min(L, ORACLE_SAMPLE_L)
        state = gpu_thermalized_sample(beta, L=sL)
        val, dt, _ = oracle_sample(beta, 4, 0, L=sL, state=state)
        cpu = {"value": val, "unit": "V+E/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"keyed oracle on one core, L={sL} at beta={beta:g} (the workload's beta and "
                         f"vertex density), 4 updates from a state thermalized by 20 GPU updates "
                         f"({dt:.1f} s)"}
        try:
            allv, procs = oracle_sample_all_cores(beta, 4, 0, L=sL, state=state)
            cpu["all_cores"] = {"value": allv, "cores": procs,
                                "sample": f"{procs} independent keyed-oracle chains at once (seeds 1..{procs}), "
                                          f"one per core, each the same sample"}
        except Exception as e:  # the one-core figure stands alone
            cpu["all_cores"] = {"value": None, "error": repr(e)[:200]}
    batched = served = None
    if world == 1 and not args.no_batched and args.workload == DEFAULT_WORKLOAD:
        batched = batched_record(BATCH_CHAINS, BATCH_UPDATES, BATCH_BUDGET_GB)
        served = {"workload": f"Poisson arrivals for {SERVED_SECONDS:g} s at each rate, S in {{1/2,1}}, L log-uniform "
                              f"[64,{SERVED_LMAX}], beta=L*U, U log-uniform [1/4,4], 50 updates + readout each; "
                              f"{BATCH_BUDGET_GB:g} GB budget, 512 slots",
                  "rates": [served_record(int(rate * SERVED_SECONDS), rate, SERVED_LMAX, 50, BATCH_BUDGET_GB, 512,
                                          SERVED_SECONDS + 20.0) for rate in SERVED_RATES]}
    line = {
        "metric": "space-time vertices+edges/s per loop update", "value": value, "unit": "V+E/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(L, beta) + f", one chain per GPU (seed 1+rank), Neel start, "
                               f"{therm}+16+{args.warmup} untimed updates (16: autotuning trials)",
                   "L": L, "beta": beta, "vertices_per_update": mean_n,
                   "temporal_moment": bool(args.temporal), "tuning": tuning, "retimed_windows": retimed,
                   "l2": "inputs larger than L2 (state and per-update graph are tens of GB)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "V+E/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": lcqmc.RECORD_DTYPE.itemsize,
                "note": "each step is lcqmc_update(h, 1) plus the readback of its record; the chain's "
                        "world-line state lives on the device by design (the paper's nodes keep their "
                        "world lines), so no input is copied in per step"},
        "gpu_launches": KERNELS_PER_UPDATE * args.steps,
        "clocks": clocks,
    }
    if batched is not None:
        line["batched"] = batched
    if served is not None:
        line["served"] = served
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def log(msg):
    print(msg, file=sys.stderr, flush=True)


def _pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def batched_record(n_chains, updates, budget_gb):
    """Many independent uneven chains (L log-uniform in [32, 4096], beta = L U,
    U log-uniform in [1/4, 4], seeds 0..n-1): batched launches (chains packed
    per phase, CUDA-graph replay, memory-bounded waves in footprint order) vs
    the same kernels launched chain by chain.  Per-chain results must be
    identical.  Completion times count from the start of each leg."""
    import torch
    from paper_1810_07485_gb300 import lcqmc, workloads
    specs = workloads.batch_specs(n_chains, seed=0)
    foot = [lcqmc.footprint(s["L"], s["beta"]) for s in specs]
    order = sorted(range(len(specs)), key=lambda i: foot[i])
    budget = budget_gb * 1e9
    waves, cur, used = [], [], 0.0
    for i in order:
        if cur and used + foot[i] > budget:
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(i)
        used += foot[i]
    if cur:
        waves.append(cur)
    lcqmc.Chain(8, 1.0).close()  # context warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_b, obs_b = {}, {}
    for wave in waves:
        bt = lcqmc.Batch([specs[i] for i in wave])
        bt.update(updates)
        bt.sync()
        tw = time.perf_counter() - t0
        for j, i in enumerate(wave):
            obs_b[i] = bt.measure(j)
            done_b[i] = tw
        bt.close()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    done_1, obs_1 = {}, {}
    for i in order:
        s = specs[i]
        ch = lcqmc.Chain(s["L"], s["beta"], seed=s["seed"])
        ch.update(updates)
        obs_1[i] = ch.measure()
        done_1[i] = time.perf_counter() - t0
        ch.close()
    t1 = time.perf_counter() - t0
    same = sum(1 for i in obs_b if list(obs_b[i].sum) == list(obs_1[i].sum) and
               list(obs_b[i].sumsq) == list(obs_1[i].sumsq))
    ve = float(sum(o.sum[7] for o in obs_b.values()))
    return {
        "workload": f"{n_chains} S=1/2 chains, L log-uniform [32,4096], beta=L*U, U log-uniform [1/4,4], "
                    f"seeds 0..{n_chains - 1}, {updates} updates each",
        "waves": len(waves), "budget_gb": budget_gb, "vertices_edges": ve,
        "batched": {"seconds": tb, "ve_per_s": ve / tb, "p50_s": _pct(list(done_b.values()), 50),
                    "p99_s": _pct(list(done_b.values()), 99)},
        "one_by_one": {"seconds": t1, "ve_per_s": ve / t1, "p50_s": _pct(list(done_1.values()), 50),
                       "p99_s": _pct(list(done_1.values()), 99)},
        "speedup": t1 / tb, "identical_results": f"{same}/{len(specs)}",
    }


def run_batched(args):
    """The batched form alone (see batched_record)."""
    import torch
    torch.cuda.set_device(0)
    rec = batched_record(args.chains, args.updates, args.budget_gb)
    line = {"metric": "batched chains: V+E/s and per-chain completion p50/p99 vs one-by-one", "mode": "batched",
            "value": rec["batched"]["ve_per_s"], "unit": "V+E/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic", "config": {"workload": rec["workload"], "waves": rec["waves"],
                                            "budget_gb": rec["budget_gb"]}}
    line.update({k: rec[k] for k in ("batched", "one_by_one", "speedup", "identical_results")})
    print(json.dumps(line), flush=True)


def served_record(n_requests, rate, req_lmax, req_updates, budget_gb, slots, time_limit):
    """Poisson stream of requests (S in {1/2, 1}, L log-uniform in [64, L_max],
    beta = L U, U log-uniform in [1/4, 4], req_updates updates + readout
    each) into the continuous-batching server; polling bounded by
    time_limit.  Latency = submit to result, per request (one update block)."""
    from paper_1810_07485_gb300 import lcqmc, workloads
    stream = workloads.request_stream(n_requests, rate, L_max=req_lmax, n_updates=req_updates, seed=0)
    srv = lcqmc.Server(int(budget_gb * 1e9), slots)
    rejected = {}
    tickets = {}
    t0 = time.perf_counter()
    for k, (ta, s) in enumerate(stream):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        try:
            tickets[k] = srv.submit(s["L"], s["beta"], s["n_updates"], S=s["S"], seed=s["seed"])
        except lcqmc.LcqmcError as e:
            rejected[k] = e.code
    log(f"served {rate}/s: {len(tickets)} submitted, {len(rejected)} rejected at submission")
    res = {}
    t_log = time.perf_counter()
    while time.perf_counter() - t0 < time_limit and len(res) < len(tickets):
        for k, t in tickets.items():
            if k not in res:
                r = srv.poll(t)
                if r is not None:
                    res[k] = (r.status, r.t_done - r.t_submit, r.t_admit - r.t_submit, r.vertices_edges, r.t_done)
        if time.perf_counter() - t_log > 5.0:
            t_log = time.perf_counter()
            log(f"served {rate}/s: t={t_log - t0:.1f}s finished {len(res)}/{len(tickets)}")
        time.sleep(0.01)
    wall = time.perf_counter() - t0
    srv.close()
    done = {k: v for k, v in res.items() if v[0] == 0}
    lat = [v[1] for v in done.values()]
    ve = float(sum(v[3] for v in done.values()))
    last = max((v[4] for v in done.values()), default=wall)
    rej_s = {0.5: 0, 1.0: 0}
    for k in rejected:
        rej_s[stream[k][1]["S"]] += 1
    return {
        "rate_per_s": rate, "submitted": len(stream), "rejected_at_admission": len(rejected),
        "rejected_fraction": {"S=1/2": rej_s[0.5] / max(1, sum(1 for _, s in stream if s["S"] == 0.5)),
                              "S=1": rej_s[1.0] / max(1, sum(1 for _, s in stream if s["S"] == 1.0))},
        "completed": len(done), "failed": len(res) - len(done), "unfinished_at_limit": len(tickets) - len(res),
        "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99),
        "queue_wait_p50_s": _pct([v[2] for v in done.values()], 50), "ve_per_s": ve / last if last > 0 else None,
        "wall_s": wall,
    }


def run_served(args):
    """The served form at one rate, or at each rate of --sweep (one JSON line)."""
    import torch
    torch.cuda.set_device(0)
    rates = [float(x) for x in args.sweep.split(",")] if args.sweep else [args.rate]
    out = []
    for rate in rates:
        n_req = args.requests if not args.sweep else int(round(rate * args.sweep_seconds))
        out.append(served_record(n_req, rate, args.req_lmax, args.req_updates, args.budget_gb, args.slots,
                                 args.time_limit))
    line = {
        "metric": "served requests: latency p50/p99 per update block and V+E/s", "mode": "served",
        "value": out[-1]["ve_per_s"], "unit": "V+E/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": f"Poisson arrivals, S in {{1/2,1}}, L log-uniform [64,{args.req_lmax}], beta=L*U, "
                               f"U log-uniform [1/4,4], {args.req_updates} updates + readout each",
                   "hbm_budget_gb": args.budget_gb, "slots": args.slots, "time_limit_s": args.time_limit,
                   "arrival_seconds_per_rate": args.sweep_seconds if args.sweep else None},
        "rates": out,
    }
    print(json.dumps(line), flush=True)


# Swendsen-Wang 2D Ising benchmark of the paper's union-find (Sec. 4.1):
# L = 8192 at K_c = ln(1 + sqrt 2)/2, 128 burn-in steps from the ordered state.
SW_L = 8192
SW_K = math.log(1.0 + math.sqrt(2.0)) / 2.0
SW_BURN_IN = 128
SW_ORACLE_L = 1024
SW_KERNELS_PER_UPDATE = 5
SW_TILE = (64, 32)


def sw_phase_bytes(L):
    """Algorithmic bytes of each phase of one update (every datum read or
    written once): spins and the local-root word per site, the tile bitmaps,
    edge masks and partial sums per tile, the open-root bitmap per 32 sites."""
    N = L * L
    nt = -(-L // SW_TILE[0]) * -(-L // SW_TILE[1])
    tile_bits = 2 * 64 * 4  # local-root and open-component bitmaps
    return {"tile_bonds_uf": N * (1 + 4) + nt * (tile_bits + 4 + 8 + 16),
            "boundary_merge": nt * (4 + 8),
            "roots_flip": N * (4 + 1 + 1) + nt * (tile_bits + 24),
            "open_sizes_record": (N // 32 + 1) * 4 + nt * 48}


def sw_oracle_sample(steps=5, warmup=2, L=SW_ORACLE_L):
    from oracle import orc
    s = np.zeros(L * L, np.uint8)
    orc.sw_run(L, SW_K, 1, 0, warmup, s)
    t0 = time.perf_counter()
    orc.sw_run(L, SW_K, 1, warmup, steps, s)
    dt = time.perf_counter() - t0
    return L * L * steps / dt, dt


def run_sw(args, world, rank, local):
    import torch

    from paper_1810_07485_gb300 import lcqmc

    torch.cuda.set_device(local)
    L, N = SW_L, SW_L * SW_L
    stream = torch.cuda.Stream()
    h = lcqmc.SWIsing(L, SW_K, seed=chain_seed(rank), stream=stream.cuda_stream)
    h.update(SW_BURN_IN + args.warmup)
    h.sync()
    h.records()
    torch.cuda.synchronize()
    clk = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.update(args.steps)
    e1.record(stream)
    h.sync()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    recs = h.records()
    ms_max, units = over_ranks(world, ms, float(N * args.steps), "cuda")
    value = units / (ms_max * 1e-3)
    # end to end through the public API: one update and its record per step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.update(1)
        h.records()
    e2e_s = time.perf_counter() - t0
    e2e_max, units2 = over_ranks(world, e2e_s, float(N * args.steps), "cuda")
    # per-phase device times
    nph = min(10, max(3, args.steps))
    h.set_phase_timing(True)
    h.update(nph)
    ph = h.phase_times()
    h.set_phase_timing(False)
    nb = sw_phase_bytes(L)
    peak, peak_kind = load_peaks()
    dom = max(ph, key=lambda k: ph[k])
    achieved = nb[dom] * nph / (ph[dom] * 1e-3) / 1e9
    traffic = SW_TRAFFIC.get(dom) if kernels_sha1("sw.cu") in SW_TRAFFIC_SHA1 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes": nb[dom], "kernel": dom, "peak_kind": peak_kind,
                "phase_ms_per_update": {k: ph[k] / nph for k in ph},
                "phase_frac_of_hbm": {k: (nb[k] * nph / (ph[k] * 1e-3) / 1e9) / peak if ph[k] > 0 else None
                                      for k in ph}}
    cpu = None
    if rank == 0:
        val, dt = sw_oracle_sample()
        cpu = {"value": val, "unit": "site updates/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"Swendsen-Wang oracle, L={SW_ORACLE_L}, K=K_c, 5 updates after 2 ({dt:.1f} s)"}
    uf_ms = (ph["tile_bonds_uf"] + ph["boundary_merge"]) / nph
    line = {
        "metric": "Swendsen-Wang site updates/s (2D Ising, union-find benchmark)", "value": value,
        "unit": "site updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"Swendsen-Wang, L={L}, K=K_c=ln(1+sqrt2)/2, ordered start, "
                               f"{SW_BURN_IN}+{args.warmup} untimed steps, seed 1+rank",
                   "L": L, "K": SW_K, "mean_clusters": float(recs["n_clusters"].mean()),
                   "mean_largest_cluster": float(recs["max_cluster"].mean()),
                   "union_find_ms_per_step": uf_ms,
                   "paper_union_find_s_per_step_1_thread": 0.097,
                   "l2": "inputs larger than L2 (spins, forest and size arrays: 0.6 GB)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": units2 / e2e_max, "unit": "site updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": lcqmc.SW_RECORD_DTYPE.itemsize},
        "gpu_launches": SW_KERNELS_PER_UPDATE * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="single", choices=["single", "batched", "served", "sw"])
    ap.add_argument("--chains", type=int, default=BATCH_CHAINS)
    ap.add_argument("--updates", type=int, default=BATCH_UPDATES)
    ap.add_argument("--no-batched", action="store_true",
                    help="leave the batched and served records out of the single-chain line")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=10.0)
    ap.add_argument("--req-lmax", type=int, default=4096)
    ap.add_argument("--req-updates", type=int, default=50)
    ap.add_argument("--slots", type=int, default=512)
    ap.add_argument("--time-limit", type=float, default=60.0)
    ap.add_argument("--sweep", default="", help="served mode: comma-separated arrival rates (req/s)")
    ap.add_argument("--sweep-seconds", type=float, default=10.0,
                    help="served sweep: seconds of arrivals at each rate")
    ap.add_argument("--temporal", action="store_true",
                    help="also measure the temporal moment chi(pi, 2 pi/beta) (single mode)")
    args = ap.parse_args()
    world, rank, local = dist_setup(args.gpus)
    if args.mode == "batched":
        run_batched(args)
        return
    if args.mode == "served":
        run_served(args)
        return
    if args.mode == "sw":
        if args.impl == "reference":
            run_sw_reference(args, world, rank)
        else:
            run_sw(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
