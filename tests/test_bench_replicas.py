"""The replica path of bench.py (one graph, or one batch, per GPU; no
data-path collective): the slowest rank sets the job's time and the job's
throughput counts every rank's work.  Two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [40.0, 55.0][rank]
    slowest = bench.max_over_ranks(ms, world, device="cpu")
    out[rank] = (slowest, bench.job_throughput(7, slowest, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_all_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        slowest, value = out[r]
        assert slowest == 55.0
        assert value == pytest.approx(2 * 7 / 0.055)


def test_single_rank_passes_values_through():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(3, 500.0, 1) == pytest.approx(6.0)


def test_oracle_comparison_of_a_bench_line():
    """The bench line's vs_oracle block: relative eigenvalue error (the null
    eigenvalue left out), residual ratio and relative cut error against the
    stored oracle run, or None where no oracle run is stored."""
    import json

    import bench
    w = bench.WORKLOADS["c2"]
    gold = json.load(open(os.path.join(bench.ROOT, "tests", "golden", w["golden"])))
    ev = list(gold["eigenvalues"])
    ev[2] *= 1.0 + 3e-4                               # one perturbed eigenvalue
    st = {"eigenvalues": ev, "resnorm": [0.0] + [0.5 * w["tol"] * abs(t) for t in ev[1:]]}
    v = bench.vs_oracle(w, st, gold["cut"] * 1.01, "mixed_bf16")
    assert v["eigenvalue_max_rel_err"] == pytest.approx(3e-4, rel=1e-9)
    assert v["eigenvalue_rel_tol"] == 1e-3 and v["cut_rel_tol"] == 0.02
    assert v["cut_rel_err"] == pytest.approx(0.01, rel=1e-9)
    assert v["max_resnorm_over_tol_theta"] == pytest.approx(0.5, rel=1e-12)
    assert bench.vs_oracle(w, st, gold["cut"], "fp64")["eigenvalue_rel_tol"] == 1e-6
    assert bench.vs_oracle(bench.WORKLOADS["c5"], st, 1.0, "mixed_bf16") is None
