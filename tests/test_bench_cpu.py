"""The measurement code of bench.py on CPU: the compulsory-byte model behind the roofline figures,
the source check that voids a stale ncu traffic figure, the parsing of the clock samples, and the
defaults of a run (the schedule length and the end-to-end loop lengths)."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_byte_model_of_the_512_cubed_step():
    """Each kernel's inputs read once and outputs written once (ts = 4, cs = 8, ps = 32 bytes in the mixed
    form); the sum over the step's kernels is the design total the bench reports."""
    n = 512
    nc, nh, npart = n ** 3, n * n * (n // 2 + 1), n ** 3
    kb = {k: bench.kernel_bytes(k, n, npart, True) for k in bench.KERNELS}
    assert kb["project"] == 32 * npart + 4 * (nc + 1) + 12 * nc + 36 * nc
    assert kb["fft_fwd_y"] == kb["fft_fwd_z"] == 2 * 9 * 8 * nh
    assert kb["solve"] == (9 + 5 + 8) * 8 * nh               # 9 spectra in, 5 out, the h state read and written
    assert kb["fft_inv_x"] == 5 * 8 * nh + 5 * 4 * nc
    assert kb["kick_drift"] == 2 * 32 * npart + 5 * 4 * nc + 8 * nc
    assert sum(kb.values()) == 91997863944
    # FP64 doubles every field, complex and particle byte
    assert bench.kernel_bytes("solve", n, npart, False) == 2 * kb["solve"]
    assert bench.method_bytes_per_update(True) == 428.0 and bench.method_bytes_per_update(False) == 816.0


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    src = tmp_path / "paper_2607_17929_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("kernel source v1\n")
    (tmp_path / "profiles").mkdir()
    sha = hashlib.sha256(b"kernel source v1\n").hexdigest()[:12]
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        "# kernel precision ncap bytes source sha\n"
        f"project mixed 256 1000000 k.cu {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return src


def test_ncu_traffic_scales_by_units_and_voids_a_changed_kernel(fake_root):
    assert bench.ncu_traffic("project", 512, 512 ** 3, True) == 8 * 1000000.0   # 8x the units of the capture
    assert bench.ncu_traffic("project", 256, 256 ** 3, False) is None           # no FP64 capture
    assert bench.ncu_traffic("kick_drift", 512, 512 ** 3, True) is None          # no capture of this kernel
    (fake_root / "k.cu").write_text("kernel source v2\n")
    assert bench.ncu_traffic("project", 512, 512 ** 3, True) is None             # kernel changed since


def test_clock_summary_reports_median_clock_and_active_reasons(tmp_path):
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 780.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 760.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    open(c.path, "w").write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == 780.0
    assert not os.path.exists(c.path)


def test_clock_summary_without_samples_says_so(tmp_path):
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.path = str(tmp_path / "missing.csv")
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None


def test_default_run_keeps_the_100_step_schedule_and_times_e2e_over_the_timed_steps():
    """The default run steps the benchmark's own z = 100 -> 0 schedule of 100 steps, and its overlapped
    end-to-end loop runs as many steps as the device-timed region."""
    a = bench.parse_args([])
    assert (a.n, a.steps, a.warmup) == (512, 30, 5)
    assert a.e2e_async_steps == a.steps and a.e2e_steps == 10
    assert bench.schedule_length(a) == bench.N_STEPS_SCHEDULE == 100
    # the profiling commands (one overlapped step) and a long loop that no longer fits
    assert bench.parse_args(["--steps", "5", "--e2e-steps", "1", "--e2e-async-steps", "1"]).e2e_async_steps == 1
    long = bench.parse_args(["--e2e-async-steps", "80"])
    assert bench.schedule_length(long) == 5 + 30 + 2 * 11 + 81 + 2
