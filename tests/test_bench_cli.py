"""CPU checks of bench.py's host logic: the reference arm (the oracle timed on
the host) prints one contract line, and under torchrun with two gloo ranks only
rank 0 prints while both exit 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c0", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "MTM applies/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_two_gloo_ranks():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "c0", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def test_rank_reductions_with_gloo():
    """max/sum over ranks as bench.py computes them, on two gloo ranks."""
    code = r'''
import os, sys, torch.distributed as dist
sys.path.insert(0, os.environ["ROOT"])
import bench
dist.init_process_group("gloo")
r = dist.get_rank()
mx = bench.max_over_ranks(2, float(r + 1))
sm = bench.sum_over_ranks(2, float(r + 1))
assert mx == 2.0 and sm == 3.0, (mx, sm)
dist.destroy_process_group()
'''
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", ROOT=ROOT)
    script = os.path.join(os.environ.get("TMPDIR", "/tmp"), "hh_rank_reduce_%d.py" % os.getpid())
    with open(script, "w") as f:
        f.write(code)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), script]
    try:
        r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    finally:
        os.remove(script)
    assert r.returncode == 0, r.stderr[-2000:]


def test_cpu_baseline_reports_one_thread_and_all_cores():
    """The oracle baseline: one thread, and one spawned copy per host core."""
    import bench
    import workloads
    r = bench.cpu_baseline(workloads.C0, seconds=0.3)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
    a = r["all_cores"]
    assert a["cores"] >= 1 and a["value"] > 0 and a["kind"] == "oracle"


def test_algorithmic_bytes_per_site():
    """11 words per CG step (r, p, L in and p, q out for the direction and
    Q p; x, p, r, q in and x, r out for the updates), a true-residual step
    reads x, L, b and writes r (plus x32 in and out and r32 out when mixed)."""
    import bench
    assert bench.bytes_per_site("cg", "fp64") == 88
    assert bench.bytes_per_site("cg", "mixed") == 44
    assert bench.bytes_per_site("cg", "mixed-fix16link") == 42
    assert bench.bytes_per_site("ru", "fp64") == 32
    assert bench.bytes_per_site("ru", "mixed-bf16link") == bench.bytes_per_site("ru", "mixed") == 44


def test_us_per_engine_iteration():
    import bench
    cnt = {"cg_steps": 2000, "ru_steps": 4, "engine_launches": 1, "engine_ms": 30.09}
    assert abs(bench.us_per_engine_iteration(cnt) - 30090.0 / 1003.0) < 1e-9
    assert bench.us_per_engine_iteration({"cg_steps": 0, "ru_steps": 0, "engine_launches": 0,
                                          "engine_ms": 0.0}) is None
