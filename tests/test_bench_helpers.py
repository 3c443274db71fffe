"""bench.py's host-side helpers on the CPU: the effective flop counts against
a count taken from the method's structure, the clock-sample parser, the
comparison with the stored oracle values, and the reference arm's line."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("m,n,b", [(1024, 1024, 32), (4096, 4096, 64), (700, 256, 16), (8192, 512, 32)])
def test_blocked_flops_from_the_visits(m, n, b):
    """A quasi-sweep visits (n/b)(n/2b) block pairs.  Each forms a 2b x 2b Gram
    block (4b^2 dot products of length m, 2m flops each) and updates an m x 2b
    and an n x 2b panel by a 2b x 2b matrix (2 flops per product term)."""
    visits = (n // b) * (n // (2 * b))
    per_visit = 2 * m * (2 * b) ** 2 + 2 * m * (2 * b) ** 2 + 2 * n * (2 * b) ** 2
    assert bench.flops_per_sweep(m, n) == visits * per_visit


@pytest.mark.parametrize("m,n", [(128, 128), (300, 200)])
def test_pointwise_flops_from_the_pairs(m, n):
    """n(n-1)/2 distinct pairs per sweep, counted as n^2/2: three dot products of
    length m (2m flops each), and a rotation of two G columns and two W columns,
    x <- (x + h t y) c and y <- (t x + y) c: 3 flops per entry of each column."""
    per_pair = 3 * 2 * m + 3 * 2 * m + 3 * 2 * n
    assert bench.pointwise_flops_per_sweep(m, n) == 0.5 * n * n * per_pair


def test_clock_sampler_summary(tmp_path):
    """The nvidia-smi CSV parser: the median SM clock, the maximum, and the
    throttle reasons reported Active."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()  # as if nvidia-smi had run
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_accuracy_vs_golden_branches():
    """The stored oracle values are compared only when G has the same bytes as
    the factor they were computed for; then their own values have error 0 and
    a planted relative error of 1e-10 is reported."""
    G, J = bench.make_input("graded1024")
    ref = np.loadtxt(bench.GOLDEN)
    out = bench.accuracy_vs_golden(G, J, ref[:, 0].copy())
    if "note" in out:  # this host's libm rounds G differently: nothing is compared
        assert "not compared" in out["note"]
        return
    assert out["sigma_max_rel_err"] == 0.0 and out["gate"] == "pass"
    s = ref[:, 0].copy()
    k = int(np.argmax(2 * ref[:, 1] <= 1e-12))  # a value held to 1e-12
    s[k] *= 1.0 + 1e-10
    out = bench.accuracy_vs_golden(G, J, s)
    assert abs(out["sigma_max_rel_err_where_2floor_below_1e-12"] - 1e-10) < 1e-12
    assert out["gate"] == "fail"
    s = ref[:, 0].copy()
    s[k] *= 1.0 + 0.9e-12
    assert bench.accuracy_vs_golden(G, J, s)["gate"] == "pass"
    # a value whose doubled floor is above 1e-12 may move by up to twice its floor
    loose = np.where(2 * ref[:, 1] > 1e-12)[0]
    if loose.size:
        j = int(loose[0])
        s = ref[:, 0].copy()
        s[j] *= 1.0 + 1.5 * ref[j, 1]
        assert bench.accuracy_vs_golden(G, J, s)["gate"] == "pass"
        s[j] = ref[j, 0] * (1.0 + 3.0 * ref[j, 1])
        assert bench.accuracy_vs_golden(G, J, s)["gate"] == "fail"


def test_stored_oracle_values_are_well_formed():
    """Every stored file: one row per column (sigma > 0, a floor u kappa_j
    >= u, since kappa_j >= 1), a sweep count and the SHA-256 of G."""
    import glob

    files = sorted(glob.glob(os.path.join(bench.GOLDEN_DIR, "*_sigma.txt")))
    assert files
    for path in files:
        name = os.path.basename(path)[:-len("_sigma.txt")]
        head = [ln for ln in open(path) if ln.startswith("#")]
        assert "sweeps=" in head[0] and head[1].startswith("# sha256(G)=")
        ref = np.loadtxt(path)
        assert ref.shape == (bench.WORKLOADS[name][0], 2)
        assert np.all(ref[:, 0] > 0) and np.all(ref[:, 1] >= 2.0 ** -53 * (1 - 1e-12))


@pytest.mark.parametrize("extra", [["--workload", "graded1024", "--form", "fp64"],
                                   ["--workload", "batch10k", "--count", "16"], []])
def test_reference_arm_line(extra):
    """The reference arm runs the oracle on the host alone and prints one
    JSON line with the GPU arm's metric, unit and workload string."""
    import json
    import subprocess
    import sys

    warm = "3" if extra else "0"  # the default workload's oracle sweep takes seconds here
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", warm] + extra, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "TFLOP/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["steps"] == 1 and d["warmup"] == int(warm) and d["n_gpus"] == 1
    if extra and extra[1] == "graded1024":
        assert d["metric"] == bench.metric_name("fp64")
        assert d["config"]["workload"] == bench.WORKLOADS["graded1024"][1]
    if not extra:  # the default line: the metric on the Haar 4096 factor, a bounded sample per step
        assert d["metric"] == bench.METRIC
        assert d["config"]["workload"] == bench.WORKLOADS["haar4096"][1]
        assert "first 2048 columns" in d["config"]["sample"]
