"""The multi-rank harness of bench.py on CPU ranks (gloo, world size 2).

With N > 1 each rank runs an independent replica (weak scaling): the only
communication is the barrier around the timed region and the MAX over ranks
of the elapsed time.  These tests run that logic in two spawned processes
over 127.0.0.1, and check that the reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class A:
        gpus = world
        impl = "reference"       # gloo backend, no GPU
    r, w, local = bench.dist_init(A())
    bench.barrier(w)
    m = bench.max_over_ranks(1.5 + r, w)
    q.put((r, w, local, m))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 0, 2.5), (1, 2, 1, 2.5)]


def test_reference_arm_prints_on_rank_zero_only():
    """Two CPU ranks of the reference arm (the FP64 oracle on host cores):
    one JSON line, from rank 0; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "cfg1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and '"impl": "reference"' in lines[0], r.stdout
    import json
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_loads_only_the_oracle():
    """The reference arm is the FP64 oracle alone: after a run, the process
    has mapped the oracle's library and not the product's (the history depth
    it pre-fills comes from the oracle's own geometry, not from a plan of the
    product library)."""
    code = ("import runpy, sys\n"
            f"sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '0', '--workload', 'cfg1']\n"
            f"runpy.run_path({os.path.join(ROOT, 'bench.py')!r}, run_name='__main__')\n"
            "maps = open('/proc/self/maps').read()\n"
            "assert 'librp_oracle.so' in maps, 'oracle not loaded'\n"
            "assert '/librp.so' not in maps, 'product library loaded by the reference arm'\n"
            "print('MAPS_OK')\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "MAPS_OK" in r.stdout
