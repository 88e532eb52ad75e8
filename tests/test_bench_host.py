"""The benchmark's control flow and JSON line on the CPU, with the device and the library faked.

Every call the benchmark makes into CUDA or the library is replaced by a stand-in that records
its arguments (no device work happens); the test checks that the default transform benchmark
times blocks of nvec and of 1 vector on both sides and prints one JSON line with the keys the
measurement contract needs.
"""
import json
import os
import runpy
import subprocess
import sys

import torch

from paper_2301_13264_gb300 import binding as B
import paper_2301_13264_gb300.synth as synth


class _Event:
    def __init__(self, **kw):
        self.t = 0.0

    def record(self, *a):
        import time
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return max((other.t - self.t) * 1e3, 1e-3)


class _Stream:
    cuda_stream = 0


def test_transform_benchmark_json(monkeypatch, capsys):
    calls = []

    def transform(h, side, nv, X, Y):
        assert X.is_contiguous() and Y.is_contiguous() and X.shape[0] >= nv and Y.shape[0] >= nv
        calls.append((side, nv))

    as_tensor = torch.as_tensor
    monkeypatch.setattr(torch, "as_tensor", lambda x, *a, **k: as_tensor(x, *a, **{q: w for q, w in k.items()
                                                                                   if q != "device"}))
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: _Stream())
    monkeypatch.setattr(B, "ccsd_create", lambda *a, **k: object())
    monkeypatch.setattr(B, "ccsd_solve_ground", lambda h: (-1.0, 3))
    monkeypatch.setattr(B, "ccsd_jacobian_transform", transform)
    monkeypatch.setattr(B, "ccsd_profile_start", lambda h: None)
    monkeypatch.setattr(B, "ccsd_profile_stop", lambda h: {k: 1.0 for k, _ in B.ProfileData._fields_})
    monkeypatch.setattr(B, "ccsd_destroy", lambda h: None)
    monkeypatch.setattr(B, "eom_solve_right", lambda h, n: ([0.3, 0.4], 5))
    monkeypatch.setattr(B, "eom_solve_left", lambda h, n: ([0.3, 0.4], 6))
    monkeypatch.setattr(B, "ccsd_derivative_coupling", lambda h, k, l, nd, dh, dB: [0.01 * (k + 2 * l)])
    monkeypatch.setattr(B, "ccsd_stats", lambda h: {"flops_fp64": 1.0, "flops_tc": 2.0, "gemms": 3, "tc_gemms": 4})
    monkeypatch.setattr(synth, "workload", lambda name: synth.make_hamiltonian(2, 4, 6, seed=0))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--no-e2e", "--no-cpu-baseline", "--steps", "2", "--warmup", "3",
                                      "--nvec", "3"])
    runpy.run_path(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"),
                   run_name="__main__")
    line = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(line) == 1
    out = json.loads(line[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks",
                "right_transforms_per_s", "left_transforms_per_s", "block1_transforms_per_s"):
        assert key in out, key
    assert out["steps"] == 2 and out["warmup"] == 3 and out["n_gpus"] == 1
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic", "frac_of_fp64_peak"):
        assert key in out["roofline"], key
    # the time-to-coupling comparison measured in the same run
    for key in ("workload", "mixed_s", "reference_s", "reference_form", "speedup", "energy_diff",
                "omega_diff_per_root", "coupling_rel_diff_per_pair"):
        assert key in out["ttc"], key
    # warm-up and timed steps (3 + 2 steps of right + left at nvec), the two separate 8-vector runs per
    # side, then one untimed and two timed single-vector transforms per side
    assert calls[:10] == [(0, 3), (1, 3)] * 5
    assert calls.count((0, 1)) == 3 and calls.count((1, 1)) == 3


def test_time_to_coupling_json(monkeypatch, capsys):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    created = []

    def create(eps, h, Bm, o, v, naux, opt):
        created.append(opt.precision)
        return object()

    monkeypatch.setattr(B, "ccsd_create", create)
    monkeypatch.setattr(B, "ccsd_solve_ground", lambda h: (-1.0, 3))
    monkeypatch.setattr(B, "eom_solve_right", lambda h, n: ([0.3, 0.4], 5))
    monkeypatch.setattr(B, "eom_solve_left", lambda h, n: ([0.3, 0.4], 6))
    monkeypatch.setattr(B, "ccsd_derivative_coupling", lambda h, k, l, nd, dh, dB: [0.01 * (k + 2 * l)])
    monkeypatch.setattr(B, "ccsd_stats", lambda h: {"flops_fp64": 1.0, "flops_tc": 2.0, "gemms": 3, "tc_gemms": 4})
    monkeypatch.setattr(B, "ccsd_destroy", lambda h: None)
    monkeypatch.setattr(synth, "workload", lambda name: synth.make_hamiltonian(2, 4, 6, seed=0))
    monkeypatch.setattr(B, "ccsd_profile_start", lambda h: None)
    monkeypatch.setattr(B, "ccsd_profile_stop", lambda h: {})
    monkeypatch.setattr(B, "ccsd_profile_records", lambda h: [
        {"engine": 1, "ms": 2.0, "flops": 4e12}, {"engine": 2, "ms": 1.0, "flops": 1e12},
        {"engine": 1, "ms": 3.0, "flops": 1e12}])
    monkeypatch.setattr(sys, "argv", ["bench.py", "--ttc", "mixed,fp64tc,fp64", "--workload", "thymine_dz",
                                      "--ttc-profile"])
    runpy.run_path(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"),
                   run_name="__main__")
    out = json.loads([l for l in capsys.readouterr().out.splitlines() if l.startswith("{")][0])
    assert created == [B.PREC_MIXED, B.PREC_FP64_TC, B.PREC_FP64]
    assert out["forms"]["mixed"]["gemm_time"]["split-bf16 TC"] == {"launches": 2, "ms": 5.0, "alg_tflop": 5.0}
    assert set(out["forms"]) == {"mixed", "fp64tc", "fp64"}
    for form in ("mixed", "fp64tc"):
        cmp = out["forms"][form]["vs_fp64"]
        assert cmp["energy_diff"] == 0.0 and cmp["coupling_rel_diff"] == 0.0 and cmp["speedup"] > 0


def test_transform_flops_count_the_ladder_packed():
    """The ladder enters at its pair-packed size, o^2 v^4 / 4 multiply-adds per vector;
    at o=33, v=228, naux=900 one transform is about 10.2 TFLOP of algorithmic work."""
    bench = runpy.run_path(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    for (o, v, naux) in [(2, 5, 7), (33, 228, 900)]:
        total, ladder = bench["transform_flops"](o, v, naux)
        assert ladder == 2.0 * o * o * v ** 4 / 4.0
        assert total > ladder
    total, _ = bench["transform_flops"](33, 228, 900)
    assert 9.5e12 < total < 11e12


def test_reference_arm_loads_nothing_of_the_library(tmp_path):
    """The reference arm runs the oracle alone: neither the binding module nor the CUDA
    library may be loaded in its process."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    probe = tmp_path / "probe.py"
    probe.write_text(
        "import json, runpy, sys\n"
        f"sys.path.insert(0, {root!r})\n"
        "sys.argv = ['bench.py', '--impl', 'reference', '--workload', 'small', '--steps', '5', '--warmup', '1']\n"
        f"runpy.run_path({os.path.join(root, 'bench.py')!r}, run_name='__main__')\n"
        "maps = open('/proc/self/maps').read()\n"
        "assert 'libccsd_gb300' not in maps, 'CUDA library loaded'\n"
        "assert 'paper_2301_13264_gb300.binding' not in sys.modules, 'binding imported'\n"
        "print('CLEAN')\n")
    r = subprocess.run([sys.executable, str(probe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = [l for l in r.stdout.splitlines() if l.startswith("{")][0]
    out = json.loads(line)
    assert out["impl"] == "reference" and out["steps"] == 2 and out["steps_requested"] == 5
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert "CLEAN" in r.stdout


def test_contraction_table_sums_launches_per_step():
    ns = runpy.run_path(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    rec = lambda label, ms, eng=1, lad=0: {"label": label, "engine": eng, "ladder": lad, "batch": 1, "m": 256,
                                           "n": 128, "k": 64, "ms": ms, "flops": 2.0 * 256 * 128 * 64,
                                           "issued_flops": 12.0 * 256 * 128 * 64}
    # two steps of three launches: the ladder twice per step, a DFMA contraction once
    recs = [rec("Y[ijab] += W[abcd] * X[ijcd] (pp-ladder, + pairs)", 4.0, lad=1),
            rec("Y[ijab] += W[abcd] * X[ijcd] (pp-ladder, + pairs)", 4.0, lad=1),
            rec("Z[ij] += F[ik] * X[kj]", 2.0, eng=0)] * 2
    table = ns["contraction_table"](recs, 2, "test")
    rows = [l for l in table.splitlines() if l.startswith("| `")]
    assert len(rows) == 2
    assert "pp-ladder" in rows[0] and "(ladder)" in rows[0]      # slowest first
    cells = [c.strip() for c in rows[0].split("|")]
    assert cells[4] == "2" and cells[5] == "8.00" and cells[6] == "80.0%"
    # 2 M N K flops over 4 ms per launch
    assert abs(float(cells[7]) - 2.0 * 256 * 128 * 64 / 4e-3 / 1e12) < 0.06
    assert "FP64 DFMA" in rows[1] and "10.0 ms per step" in table
    assert cells[9] == "0" and rows[1].rstrip().endswith("| — |")
