"""CPU checks of bench.py's host logic: the multi-rank max reduction over gloo
(world size 2), the algorithmic flop count, the traffic lookup, and the
reference arm's JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.reduce_max(float(rank + 1) * 1.5, world)
    bench.barrier(world)
    out[rank] = v
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 3.0, 1: 3.0}


def test_single_rank_reduce_is_identity():
    assert bench.reduce_max(2.5, 1) == 2.5


def test_step_flops():
    D = 32
    assert bench.step_flops(D, D, D) == 2 * D ** 7 + 16 * D ** 6


def test_captured_traffic_only_for_profiled_workload():
    v = bench.captured_traffic("ising_044_d32", "tf32")
    assert v is None or v > 4 * 32 ** 5              # at least the read of P (part of Q stays in L2)
    assert bench.captured_traffic("potts3_d64", "bf16x3") is None


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "ising_bc_d8", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "RG-steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.parametrize("workload,unit", [("heisenberg_b4_d8", "update steps/s"),
                                           ("itebd_heisenberg_d16", "update steps/s")])
def test_reference_arm_quantum_workloads(workload, unit):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", workload, "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == unit
    assert d["config"]["workload"] == workload
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["d2h_bytes_per_step"] == 0


def test_transient_steps_schedule():
    import bench
    # each step squares the fused dimension (capped at D_cut): 2 -> 4 -> 16 -> D_cut
    assert bench.transient_steps(2, 16) == 4
    assert bench.transient_steps(2, 24) == 6
    assert bench.transient_steps(2, 40) == 6
    assert bench.transient_steps(2, 4) == 2
    assert bench.transient_steps(3, 9) == 2


def test_clock_sampler_names_the_visible_gpu(monkeypatch):
    """nvidia-smi numbers GPUs physically: without a device UUID from torch the
    sampler must use the local-th entry of CUDA_VISIBLE_DEVICES, not the rank."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a visible GPU names itself by UUID")
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,GPU-1234")
    assert bench.gpu_selector(0) == "5"
    assert bench.gpu_selector(1) == "GPU-1234"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_selector(0) == "0"


def test_clock_summary_reports_cycles_per_step():
    s = bench.ClockSampler(0)
    s.lines = ["2070, 2070, 900, Not Active, Not Active, Not Active, Active",
               "2060, 2070, 910, Not Active, Not Active, Not Active, Not Active"]
    out = s.summary(ms_per_step=2.0)
    assert out["sm_mhz"] == 2065.0 and out["reasons"] == ["sw_power_cap"]
    assert out["mcycles_per_step"] == round(2.0 * 2065.0 / 1e3, 4)


def test_sweep_partition_is_a_balanced_cover():
    from workloads import sweep256
    models = sweep256()
    for world in (1, 2, 3, 4, 8):
        parts = bench.partition_instances(models, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(models)))
        loads = [sum(2.0 * models[i].D_cut ** 7 for i in p) for p in parts]
        # longest-processing-time first: no rank carries more than the mean plus one instance
        assert max(loads) - sum(loads) / world <= 2.0 * 40 ** 7 + 1e-6


def _sweep_rank(rank, world, port, out):
    import torch.distributed as dist
    from workloads import sweep256
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    models = sweep256()
    mine = bench.partition_instances(models, world)[rank]
    got = bench.gather_floats([float(i) for i in mine], world)
    out[rank] = got
    dist.destroy_process_group()


def test_sweep_shards_gather_over_two_gloo_ranks():
    """Each rank derives its own share of the sweep with no communication; the
    only exchange is the host gather after the timed region, which must hand
    every rank every instance exactly once."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_sweep_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert sorted(int(v) for v in out[r]) == list(range(256))


def test_eig_block_work_figures():
    """The eigensolver block: block size 5k/4 rounded up to 8, the FP64-grade
    G X work of both environments per step, and the dense FP64 bound."""
    class Info:
        def __init__(self, iters):
            self.eig_path, self.eig_iters, self.eig_rr = 2, iters, 1
            self.eig_sweeps32, self.eig_sweeps = 3, 0
    D, ms = 32, 2.0
    blk = bench.eig_block({"ms": {"eig": ms}}, 1, D, {"fp64_tflops": 1.0}, [Info(8), Info(10)])
    n, m = D * D, 48
    assert blk["block_m"] == m
    assert blk["gx_fp64_grade_flops_per_step"] == 9 * 2 * (2.0 * n * n * m)
    assert abs(blk["gx_fp64_grade_tflops_over_eig_time"] - 9 * 4.0 * n * n * m / 2e-3 / 1e12) < 1e-3
    dense = 2 * (4.0 / 3.0) * n ** 3
    assert abs(blk["dense_bound_over_eig_time"] - dense / 1e12 * 1e3 / ms) < 1e-3
    assert blk["subspace_iterations_per_step"] == 9
