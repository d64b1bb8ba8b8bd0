"""Multi-rank benchmark logic on CPU: two gloo ranks, no GPU.

Under torchrun each rank advances its own independent chain (seed 1 + rank)
and no collective touches the data path; the only exchange is the final
reduction of the timed figures (max of elapsed time, sum of units).  These
tests run that reduction and the per-rank chains (on the oracle) as two real
processes, and check that the reference arm does its work on rank 0 only.
"""
import argparse
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                          WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        import torch.distributed as dist

        import bench
        from oracle import orc
        w, r, loc = bench.dist_setup(world)
        assert (w, r, loc) == (world, rank, rank)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        # each rank's own chain: a small keyed update sequence on the oracle
        p = orc.params(16, 4.0, seed=bench.chain_seed(rank))
        st = orc.neel(p)
        recs = orc.keyed_run(p, 0, 6, st)
        ve = float((recs["n_seg"] + 2 * recs["n"]).sum())
        elapsed = 1.0 + 0.5 * rank
        t_max, ve_tot = bench.over_ranks(world, elapsed, ve, "cpu")
        got = [None] * world
        dist.all_gather_object(got, (ve, recs["n"].tolist(), st.s0.tolist()))
        dist.destroy_process_group()
        q.put((rank, t_max, ve_tot, ve, got))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, "error", repr(e), None, None))


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_and_shard(orc):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = {}
    for _ in range(world):
        rank, *rest = q.get(timeout=240)
        out[rank] = rest
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank in range(world):
        assert out[rank][0] != "error", out[rank][1]
    # the reduction: slowest rank's time, all ranks' units, identical on every rank
    ve = [out[r][2] for r in range(world)]
    for r in range(world):
        t_max, ve_tot = out[r][0], out[r][1]
        assert t_max == 1.0 + 0.5 * (world - 1)
        assert ve_tot == sum(ve)
    # the ranks ran distinct chains (different seeds give different graphs)
    got = out[0][3]
    assert got[0][1] != got[1][1] or got[0][2] != got[1][2]
    # and each rank's chain is the one a single process gets with that seed
    import bench
    for r in range(world):
        p = orc.params(16, 4.0, seed=bench.chain_seed(r))
        st = orc.neel(p)
        recs = orc.keyed_run(p, 0, 6, st)
        assert recs["n"].tolist() == got[r][1]
        assert st.s0.tolist() == got[r][2]


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.over_ranks(1, 2.5, 7.0, "cpu") == (2.5, 7.0)


def test_reference_arm_only_on_rank0(capsys, monkeypatch):
    import bench
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(a) or (1.0, 1.0, None))
    args = argparse.Namespace(workload=bench.DEFAULT_WORKLOAD, steps=3, warmup=3, gpus=2)
    bench.run_reference(args, 2, 1)
    assert capsys.readouterr().out == "" and not called
    bench.run_reference(args, 2, 0)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1 and len(called) == 1
    import json
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_rank_seeds_distinct():
    import bench
    seeds = [bench.chain_seed(r) for r in range(8)]
    assert len(set(seeds)) == 8


@pytest.mark.timeout(300)
def test_oracle_all_cores_sample(orc):
    # The all-core oracle baseline: independent chains in spawned processes,
    # each the same as the chain run alone with its seed.
    import bench
    val, procs = bench.oracle_sample_all_cores(4.0, 2, 1, L=16, procs=2)
    assert procs == 2 and val > 0
    from oracle import timing
    ve, dt = timing.chain_sample((16, 4.0, 2, 1, 2))
    p = orc.params(16, 4.0, seed=2)
    st = orc.neel(p)
    orc.keyed_run(p, 0, 1, st)
    r = orc.keyed_run(p, 1, 2, st)
    assert ve == float((r["n_seg"] + 2 * r["n"]).sum())


def test_sw_reference_arm_line(capsys):
    # bench.py --impl reference --mode sw: the oracle on rank 0 only, with the
    # contract's keys; the other ranks print nothing.
    import json

    import bench
    args = argparse.Namespace(steps=3, warmup=3, gpus=2)
    bench.run_sw_reference(args, 2, 1)
    assert capsys.readouterr().out == ""
    bench.run_sw_reference(args, 2, 0)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["unit"] == "site updates/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["L"] == bench.SW_L
