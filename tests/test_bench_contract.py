"""The benchmark's reference arm (the FP64 oracle on the host) keeps the JSON-line
contract, and under several ranks only rank 0 works and prints. CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_line_has_the_contract_keys():
    r = _run({"RANK": "0"}, "--workload", "rect256", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "clips/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["config"]["workload"] == "rect256" and d["config"]["n"] == 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "clips/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--workload", "rect256", "--steps", "1", "--gpus", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_flop_and_byte_accounting():
    """The benchmark's accounting: the truncated-DFT method's real flops per iteration,
    16 K k n^2 + 8 k n^2 + 16 K n k^2 + 16 n k^2 (0.142 GFLOP at 256^2, K = 8, k = 15;
    58.5 GFLOP at 2048^2, K = 24, k = 35), and the per-pixel algorithmic bytes of the
    streaming kernels."""
    sys.path.insert(0, ROOT)
    import bench
    assert abs(bench.algorithmic_flops_per_iter(256, 8, 15) / 1e9 - 0.142) < 0.0005
    assert abs(bench.algorithmic_flops_per_iter(2048, 24, 35) / 1e9 - 58.5) < 0.05
    px = 2048 * 2048
    assert bench.kernel_bytes("resist", 2048, 24, 35, True) == 9 * px
    # the level-set step's method bytes (phi, V in; phi, mask out) on either path
    assert bench.kernel_bytes("levelset_step", 2048, 24, 35, False) == 13 * px
    assert bench.kernel_bytes("levelset_step", 2048, 24, 35, True) == 13 * px
    # the EDT row pass in the solve: column distances and mask in, phi out (no d^2 kept)
    assert bench.kernel_bytes("edt_rows", 2048, 24, 35, True) == 9 * px
    # the difference window removes the K dependence of the n^2-sized work
    assert bench.window_flops_per_iter(2048, 24, 35) < bench.algorithmic_flops_per_iter(2048, 24, 35) / 10
