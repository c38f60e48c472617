"""bench.py's multi-rank plumbing on CPU with gloo, world size 2.

The benchmark runs independent replicas (no data-path collective); ranks
meet only at barriers and the max/sum reductions of the timing and solve
counts, which these tests exercise without a GPU.  The reference arm's JSON
line is checked on the small workload.
"""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w = bench.dist_init("gloo")
    bench.barrier()
    t = bench.reduce_scalar(1.0 + rank, "max")
    n = bench.reduce_scalar(10.0 * (rank + 1), "sum")
    bench.barrier()
    q.put((r, w, t, n))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 2.0, 30.0), (1, 2, 2.0, 30.0)]


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_scalar(3.5, "max") == 3.5
    assert bench.dist_env()[1] >= 1


def test_reference_arm_line(monkeypatch, capsys):
    import bench
    import synthetic
    from oracle import response
    from oracle.basis import Basis
    from oracle.hamiltonian import dense_hamiltonian, ks_states

    def tiny_setup():
        s = synthetic.make_system("tiny")
        b = Basis(s.grid, s.cell)
        ks = ks_states(b, s.v_r, s.n_occ)
        h = dense_hamiltonian(b, s.v_r)
        dv = synthetic.random_grid_potentials(5, 1, s.grid, s.cell)[0]
        return s, b, ks, h, dv, response.occupied_grid(b, ks)

    monkeypatch.setattr(bench, "_oracle_setup", tiny_setup)
    for k in ("RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
