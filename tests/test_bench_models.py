"""CPU checks of the algorithmic work models that bench.py divides by measured times (the roofline
numerators): warp steps of the wavefront schedule, tape bytes per adjoint launch, and FLOPs per
cell of the forward and adjoint maps, against counts made independently here."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_models", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _steps_by_simulation(points):
    """Warp steps counted by walking the schedule: lane r works on local step t at column
    (t - r) mod P of strip (t - r) // P; the sweep ends after the last lane's last cell."""
    rows = cols = points - 1
    P = max(cols, 32)
    last = 0
    for r in range(32):
        for s in range((rows + 31) // 32):
            if s * 32 + r < rows:
                last = max(last, s * P + r + cols - 1)
    return last + 1


@pytest.mark.parametrize("points", [2, 20, 33, 34, 129, 257])
def test_tape_steps_match_the_schedule(bench, points):
    assert bench.tape_steps(points) == _steps_by_simulation(points)


def test_tape_bytes_of_the_bench_launch(bench):
    # 128 x 128 pairs of 257-point paths, N = 6: per lane and warp step a row of 14 floats (the 12
    # derivatives d a'_n/dM, d b'_n/dM, the exponent and M: 56 B) written by the forward, read by
    # the adjoint, which writes one dk/dM float
    assert bench.tape_steps(257) == 2079
    assert bench.tape_forward_bytes(128 * 128, 257) == 16384 * 2079 * 32 * 56
    assert bench.tape_adjoint_bytes(128 * 128, 257) == 16384 * 2079 * 32 * (56 + 4)
    assert bench.tape_adjoint_bytes(128 * 128, 257, esize=8) == 16384 * 2079 * 32 * (112 + 8)


def test_flops_per_cell(bench):
    N, d = 6, 8
    # per edge and output n: N multiply-adds for the corner term plus Hankel coupling; for n >= 1
    # the Toeplitz terms 1 <= k < n (the k = n term is a_n e_0 = a_n) and the e_n scaling
    corner_hankel = 2 * (N + 1) * N
    toeplitz = 2 * sum(n - 1 for n in range(1, N + 1))
    scale = 2 * N
    assert bench.flops_per_cell(N, d) == 2 * (corner_hankel + toeplitz + scale + N + d) == 280
    assert bench.tape_forward_flops_per_cell(N, d) == 280 + 2 * 2 * (N - 1)
    # adjoint: Hankel weights (n >= 1), Toeplitz transposes (each from its e_0 term) and Hankel
    # couplings of both edges, dk/dM from the 2N recorded derivatives, and e_m rebuilt from M
    transposes = 2 * sum(N - k for k in range(N + 1))
    assert bench.tape_adjoint_flops_per_cell(N) == 2 * (2 * N + transposes + corner_hankel + 2 * N + N) == 312


def test_clock_samples_are_summarised_and_the_temporary_file_removed(bench, monkeypatch):
    monkeypatch.delenv("SK_CLOCKS_CSV", raising=False)
    c = bench.ClockSampler(0)
    c.proc = object()  # as if nvidia-smi had run: summarise what it wrote
    with open(c.path, "w") as f:
        f.write("0, 1965, 2070, 900.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                "0, 1980, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                "0, [N/A], 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s == {"sm_mhz": 1972.5, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert not os.path.exists(c.path)


def test_reference_arm_line_keeps_the_contract(bench, monkeypatch, capsys):
    """bench.py --impl reference prints one JSON line on the GPU arm's metric, unit and direction
    (so a ratio of the two arms is defined), its ms_per_step is the time of the steps it ran, and
    it carries the cpu_baseline and e2e objects with no host-device bytes.  The oracle's timing is
    stubbed here; the line is built as in a real run."""
    import argparse
    import inspect
    import json

    import numpy as np

    calls = []

    def fake_fwd_bwd(X, Y, points=None):
        calls.append(points)
        return 16384.0, 0.25  # cells, seconds

    monkeypatch.setattr(bench, "cpu_fwd_bwd", fake_fwd_bwd)
    monkeypatch.setattr(bench, "workload", lambda rank, *a: (np.zeros((2, 5, 8)), np.zeros((2, 5, 8))))
    bench.run_reference(argparse.Namespace(steps=3, warmup=2), 0, 1)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "cell-updates/s"
    assert line["higher_is_better"] is True
    assert line["steps"] == 3 and line["warmup"] == 2 and line["n_gpus"] == 1
    assert calls == [65, 65, 129, 129, 129]  # warm-up steps on shorter prefixes, timed steps at 129 points
    assert line["ms_per_step"] == pytest.approx(250.0)
    assert line["value"] == pytest.approx(16384.0 / 0.25)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # the GPU arm builds its line on the same metric string
    assert '"metric": METRIC' in inspect.getsource(bench.main)
    # other ranks print nothing
    bench.run_reference(argparse.Namespace(steps=1, warmup=0), 1, 2)
    assert capsys.readouterr().out == ""


def test_reference_arm_runs_from_the_command_line():
    """`python bench.py --impl reference` on this machine's cores: one JSON line as the last line
    of stdout, exit status 0, no GPU needed (one timed step of the oracle, about 10 s)."""
    import json
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["value"] == pytest.approx(16384 / (line["ms_per_step"] / 1e3), rel=1e-9)
