"""Host-side logic of bench.py on the CPU: the reference arm's JSON line, rank handling, and
the max-over-ranks aggregation of the multi-process path (gloo, world size 2)."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(10.0 + 5.0 * rank)
    out[rank] = v
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 15.0


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_nonzero_rank_does_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "rows/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD


def test_kernel_source_hash_ignores_comments_only(tmp_path):
    """The DRAM-traffic record is keyed by the kernel source without comments: a comment edit
    keeps it, a code edit invalidates it."""
    a = tmp_path / "a.cu"
    a.write_text("// one\n__global__ void k(int* x) {\n    x[0] = 1;  // set\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("/* two */\n__global__ void k(int* x) {\n\n    x[0] = 1;\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("__global__ void k(int* x) {\n    x[0] = 2;\n}\n")
    assert bench.kernel_source_hash(str(a)) == bench.kernel_source_hash(str(b))
    assert bench.kernel_source_hash(str(a)) != bench.kernel_source_hash(str(c))



def test_roofline_counts_follow_the_cost_model():
    """flops_executed = (1/3) K^3 per LDL^T factorization + 2 K^2 per solved column; the
    survey count uses (2/3) K^3 (§4.3 cost model); frac = achieved / peak."""
    K, q = 65, 7
    st = {"sum_k3": 10 * K ** 3, "sum_k2_cols": 10 * K * K * q, "flops_refine": 0.0}
    r = bench.roofline_entry([st, st], 2.0, "k")
    ex = 2 * (10 * K ** 3 / 3.0 + 2.0 * 10 * K * K * q)
    sv = 2 * (10 * 2.0 * K ** 3 / 3.0 + 2.0 * 10 * K * K * q)
    assert abs(r["flops_executed"] - ex) <= 1e-9 * ex and abs(r["flops_survey"] - sv) <= 1e-9 * sv
    assert abs(r["achieved"] - ex / 2e-3 / 1e12) <= 1e-12
    assert abs(r["frac"] - r["achieved"] / bench.FP64_PEAK_TFLOPS) <= 1e-12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"


def test_host_cpu_reports_cores_and_a_model():
    cores, model = bench.host_cpu()
    assert cores >= 1 and isinstance(model, str) and model
