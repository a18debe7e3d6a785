"""bench.py's bookkeeping on CPU (no device): the stored ncu traffic is
reported only for the kernel source it was captured on and only for the full
workload; the roofline's peak comes from the measured file when there is one;
the clock samples taken during the timed region give the median SM clock and
every throttle reason seen."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KERNEL = """// the full pass
__global__ void k(int *x) { /* one thread */ x[0] = 1; }
"""


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A repository of one kernel source and one stored traffic figure."""
    csrc = tmp_path / "paper_2001_05291_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "kernels.cu").write_text(KERNEL)
    (csrc / "device_common.cuh").write_text("#pragma once\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))

    def store(digest, workload="large", traffic=123456789):
        (tmp_path / "profiles" / "t.md").write_text(
            f"# a summary\n\nsome text: with a colon\n\nkernel_source_digest: {digest}\n"
            f"workload: {workload}\ntraffic_bytes_per_launch: {traffic}\n")
    return csrc, store


class Args:
    missions = 0


class Inst:
    name = "large"


def test_comments_and_spacing_do_not_change_the_digest(tree):
    csrc, _ = tree
    d0 = bench.kernel_digest("swap_eval")
    (csrc / "kernels.cu").write_text("// other words\n\n" + KERNEL.replace("x[0] = 1; }", "x[0]   =  1; }  // set"))
    assert bench.kernel_digest("swap_eval") == d0
    (csrc / "kernels.cu").write_text(KERNEL.replace("x[0] = 1;", "x[0] = 2;"))
    assert bench.kernel_digest("swap_eval") != d0


def test_stored_traffic_only_for_the_captured_source_and_the_full_workload(tree):
    csrc, store = tree
    store(bench.kernel_digest("swap_eval"))
    assert bench.stored_traffic("t.md", Inst(), Args(), "swap_eval") == 123456789.0
    cut = Args()
    cut.missions = 200_000                      # a cut-down run: never the full figure
    assert bench.stored_traffic("t.md", Inst(), cut, "swap_eval") is None
    other = Inst()
    other.name = "province"
    assert bench.stored_traffic("t.md", other, Args(), "swap_eval") is None
    assert bench.stored_traffic("missing.md", Inst(), Args(), "swap_eval") is None
    (csrc / "kernels.cu").write_text(KERNEL.replace("x[0] = 1;", "x[0] = 3;"))   # the kernel changed
    assert bench.stored_traffic("t.md", Inst(), Args(), "swap_eval") is None


def test_committed_summaries_carry_the_fields_the_bench_reads():
    for fname, kernel in (("persist_traffic.md", "persist"), ("swap_eval_traffic.md", "swap_eval")):
        fields = {}
        with open(os.path.join(ROOT, "profiles", fname)) as fh:
            for line in fh:
                if ":" in line and not line.startswith((" ", "#")):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        assert fields["workload"] == "large"
        assert len(fields["kernel_source_digest"]) == 16
        assert float(fields["traffic_bytes_per_launch"]) > 1e9
        assert kernel in bench.KERNEL_SOURCES


def test_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6758.2, "bf16_tflops": 1900.0}))
    assert bench.load_peaks() == (6758.2, "measured")


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks(tmp_path, rows):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(", ".join(r) + "\n" for r in rows))
    c = bench.ClockSampler(0)
    c.proc, c.path = _Proc(), str(path)
    return c.stop()


def test_clock_samples_median_and_reasons(tmp_path):
    idle = ["0", "2070", "2070", "700.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    capped = ["0", "1980", "2070", "1399.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"]
    hot = ["0", "1500", "2070", "1390.5", "0x8", "Not Active", "Active", "Not Active", "Not Active"]
    got = _clocks(tmp_path, [idle, capped, idle, ["garbage"]])
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    got = _clocks(tmp_path, [hot, capped, hot])
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and got["sm_mhz"] == 1500.0
    assert _clocks(tmp_path, []) is None
    assert not (tmp_path / "clocks.csv").exists()   # the sample file is removed
