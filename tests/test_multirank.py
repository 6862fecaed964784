"""The bench's N > 1 path on the CPU (world size 2, gloo, 127.0.0.1): every rank is an
independent replica of the step (RR sets are independent units: no data-path
collective), so the only exchange is the end-of-run reduction -- the maximum of the
ranks' timed seconds and the sum of their RR sets -- and the reference arm runs on
rank 0 alone while the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code: str, world: int = 2, timeout: float = 120.0):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=timeout)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_step_results_take_max_time_and_sum_sets():
    code = (
        "import json, bench\n"
        "rank, world, _ = bench.dist_env()\n"
        "dist = bench.init_dist(world, 'gloo')\n"
        "sec, sets = bench.reduce_step_results(dist, 'cpu', 1.5 + rank, 1000.0 * (rank + 1))\n"
        "dist.barrier()\n"
        "print(json.dumps({'rank': rank, 'sec': sec, 'sets': sets}))\n"
        "dist.destroy_process_group()\n")
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _run_ranks(code)]
    for o in outs:
        assert o["sec"] == 2.5 and o["sets"] == 3000.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.reduce_step_results(None, "cpu", 1.25, 7.0) == (1.25, 7.0)


def test_reference_arm_prints_once_from_rank_zero():
    # the oracle reference arm at N = 2: rank 0 prints one JSON line, rank 1 exits at once
    code = (
        "import bench\n"
        "bench.main(['--impl', 'reference', '--workload', 'c2', '--gpus', '2', '--steps', '1',"
        " '--warmup', '1', '--scale', '12'])\n")
    outs = _run_ranks(code, timeout=300.0)
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    rec = json.loads(lines0[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0
