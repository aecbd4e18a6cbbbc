"""Host-side logic of bench.py that needs no GPU: the oracle arm (--impl reference) prints
the contract's JSON line, ranks other than 0 exit without work (also under a two-rank
torchrun launch, which prints exactly one line), and the L2 policy picks flushing exactly
for the workloads whose working set fits in L2."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    p = _run({}, "--impl", "reference", "--workload", "chain64_N8_B10000", "--steps", "2", "--warmup", "0",
             "--ref-samples", "64")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "FFS samples/s" and d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "chain64_N8_B10000" and d["config"]["B_per_step"] == 64
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "samples/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--workload",
             "chain64_N8_B10000", "--steps", "1", "--warmup", "0", "--ref-samples", "16")
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_l2_policy():
    flushed = {k for k, s in bench.WORKLOADS.items()
               if bench.working_set_bytes(s["L"], s["N"], s["B"], s["cplx"], "df64") < 2 * bench.L2_BYTES}
    assert flushed == {"chain64_N8_B10000"}
    # the 64x64 lattice: 4096 samples x 32 slabs x 32 (s + 1) rows x 32 complex double-floats
    s = bench.WORKLOADS["lattice64x64_N1024_B4096"]
    assert bench.working_set_bytes(s["L"], s["N"], s["B"], s["cplx"], "df64") > 4096 * 512 * 32 * 33 * 16


def test_reference_arm_under_torchrun_prints_one_line():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--workload", "chain64_N8_B10000", "--steps", "1",
                        "--warmup", "0", "--ref-samples", "16"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_oracle_plan_large_workload_uses_all_cores_in_one_process():
    """A workload whose oracle sample is tens of seconds on one core is timed as whole
    samples in one process with BLAS on every core (cores = the threads used)."""
    import numpy as np

    from paper_2109_07358_gb300 import workloads as w

    U = w.haar(2048, 512, seed=1)  # L N^2 x 4 = 2.1e9 multiply-adds: the large-workload plan
    n, threads = bench.oracle_plan(U, 8, target_s=0.5)
    assert threads == (os.cpu_count() or 1) and 1 <= n <= 8
    rate, wall, cores = bench.oracle_baseline(U, 1, threads=threads)
    assert rate > 0 and wall > 0 and cores == threads
    small = w.chain_L64_N8()
    n, threads = bench.oracle_plan(small, 100, target_s=0.2)
    assert threads == 1 and n >= 2


def test_kernel_launch_count_matches_the_launch_structure():
    # Anderson chain N = 2048, one wave, K = 3 steps: per step 2048 residual and per-step
    # launches, one permutation kernel, and at the 63 panel ends panel_s, the new-row
    # kernel (+ C's slices when k0 > 0) and the old-row pass (two slice kernels and the
    # product when k0 > 0, the operand kernel always): 4534, the count of the ncu list
    K, ends = 3, 63
    n = bench.kernel_launches(2048 * K, 2048 * K, ends * K, ends * K, ends * K, K, 2048)
    assert n // K == 2048 + 2048 + 1 + ends + (ends + ends - 1) + (ends + 3 * (ends - 1))
    assert n // K == 4534
    # two waves double every count, including the panel ends without old rows
    n2 = bench.kernel_launches(2 * 2048 * K, 2 * 2048 * K, 2 * ends * K, 2 * ends * K, 2 * ends * K, 2 * K, 2048)
    assert n2 == 2 * n
    # without the tensor-core trailing update each region is one kernel
    assert bench.kernel_launches(10, 10, 2, 2, 0, 1, 2048) == 25


def test_blocked_bytes_model():
    L, N, e = 4096, 96, 8
    full = bench.blocked_bytes_per_sample(L, N, e)
    gs = bench.blocked_bytes_per_sample(L, N, e, gsum=32)
    # the draw reads L / 32 sums and one group of 32 weights instead of all L weights
    assert full["step"] - gs["step"] == N * 4 * (L - (L // 32 + 32))
    assert full["new"] == gs["new"] and full["top"] == gs["top"]
    # panel ends: k0 = 0 (T = 64) and k0 = 32 (T = 32); k0 = 64 ends the chain
    assert full["new"] == e * ((0 * 64 + 2 * 32 * 64) + (32 * 32 + 2 * 32 * 32))
    assert full["top"] == e * ((2 * 0 * 64 + 0) + (2 * 32 * 32 + 32 * 32))
