"""The benchmark's multi-rank logic on CPU: two gloo ranks, each timing its
own replica, report the slowest rank's time, and the whole-job throughput
counts every rank's cells (weak scaling, no collective on the data path)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms, torch.device("cpu"))
        out[rank] = (ms, bench.whole_job_gpts(512 ** 3, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_whole_job_value():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 512 ** 3 / 0.150 / 1e9)


def test_single_rank_helpers_without_a_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_gpts(1000, 1, 1.0) == pytest.approx(1e-3)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    monkeypatch.setattr(bench, "workload", lambda args: pytest.fail("rank 1 must not build the workload"))
    assert bench.main() == 0


def test_reference_arm_json_line(monkeypatch, capsys):
    """The reference arm (the oracle timed on the host) prints one JSON line
    with the contract's keys; a small grid keeps it to a second."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--n", "16", "--bubbles", "1",
                                      "--steps", "1", "--warmup", "3"])
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["warmup"] >= 3 and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and 1 <= cb["cores"] <= (os.cpu_count() or 1)
    assert "16x16x16" in cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_algorithmic_bytes_per_cell_at_512():
    """The roofline's numerators: algorithmic bytes per cell of each pass
    kernel of the 512^3 benchmark (residual 21.1 averaged over the 40-pass
    exact/update cycle, y transforms 8.0, z solve 20.1 for the hybrid and
    21.1 for the FP64-recurrence plan, inverse x 16.2)."""
    sys.path.insert(0, ROOT)
    import types
    import bench
    w = types.SimpleNamespace(nx=512, ny=512, nz=512)
    npts = 512 ** 3
    per_cell = {k: bench.algorithmic(k, w, "mixed")["bytes"] / npts
                for k in ("resid_fftx", "ffty_fwd", "tridiag_z", "fftx_inv_update")}
    assert per_cell["resid_fftx"] == pytest.approx(21.1, abs=0.05)
    assert per_cell["ffty_fwd"] == pytest.approx(8.03, abs=0.05)
    assert per_cell["tridiag_z"] == pytest.approx(20.1, abs=0.05)
    assert per_cell["fftx_inv_update"] == pytest.approx(16.2, abs=0.05)
    z64 = bench.algorithmic("tridiag_z", w, "mixed_z64")
    assert z64["bytes"] / npts == pytest.approx(21.1, abs=0.05)
    assert z64["fp64_flops"] == 8 * 257 * 512 * 512
    # the residual's DRAM traffic per launch: 39 update passes to 1 exact
    assert bench.DRAM_B_PER_CELL["resid_fftx"] * npts == pytest.approx(2.670e9, rel=2e-3)
