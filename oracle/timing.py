"""Timing of the CPU oracle on every host core (test infrastructure: used by
the benchmark's CPU-baseline leg only).

One independent keyed-oracle chain per core, as the paper runs independent
chains side by side: the rate is the V+E of all chains over the slowest
chain's time.  Workers start by spawn (the caller may already hold a GPU
context, which a forked child must not inherit).
"""
import multiprocessing as mp
import os
import time


def chain_sample(job):
    """One chain: (L, beta, seed, warmup, steps[, state]) -> (V+E of the timed
    updates, seconds).  state = (s0, op_ptr, op_tau, sweep) starts the chain
    from that configuration instead of the Neel state."""
    L, beta, seed, warmup, steps = job[:5]
    state = job[5] if len(job) > 5 else None
    from oracle import orc
    p = orc.params(L, beta, seed=seed)
    if state is None:
        st, sweep0 = orc.neel(p), 0
    else:
        st, sweep0 = orc.State(state[0], state[1], state[2]).copy(), int(state[3])
    orc.keyed_run(p, sweep0, warmup, st)
    t0 = time.perf_counter()
    recs = orc.keyed_run(p, sweep0 + warmup, steps, st)
    return float((recs["n_seg"] + 2 * recs["n"]).sum()), time.perf_counter() - t0


def _memory_cap(bytes_per_chain=3e9):
    """Chains that fit the host's available memory (a chain of the default
    sample, L = 8192 at beta = 1024, peaks near 1.5 GB)."""
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        return max(1, int(avail // bytes_per_chain))
    except (ValueError, OSError):
        return 1


MAX_PROCS = 32  # bounds the sample's start-up time on large hosts


def all_cores_sample(L, beta, steps, warmup, procs=None, state=None):
    """(V+E/s over procs chains run at once, procs); every chain starts from
    state (or the Neel state) with its own seed."""
    procs = procs or min(os.cpu_count() or 1, _memory_cap(), MAX_PROCS)
    with mp.get_context("spawn").Pool(procs) as pool:
        out = pool.map(chain_sample, [(L, beta, 1 + k, warmup, steps, state) for k in range(procs)])
    return sum(v for v, _ in out) / max(t for _, t in out), procs
