"""Host-side logic of bench.py (no GPU): the committed ncu traffic summaries are read
only while they match the current kernel sources, the clock sampler's parsing of
nvidia-smi rows, and the command line."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_summary_is_used_only_on_matching_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("kernel source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    h = bench.kernel_source_hash(("k.cuh",))
    (tmp_path / "profiles" / "t.txt").write_text(
        "# comment: the counters\nkernel_source_hash: %s\ndram_bytes_per_launch: 12345\n" % h)
    assert bench.ncu_traffic("t.txt", ("k.cuh",)) == 12345.0
    src.write_text("kernel source, changed\n")
    assert bench.ncu_traffic("t.txt", ("k.cuh",)) is None
    assert bench.ncu_traffic("missing.txt", ("k.cuh",)) is None


def test_committed_traffic_summaries_parse():
    for name, sources in [("spmm_powerlaw_kt32_g0_traffic.txt", bench.SPMM_STREAM_SOURCES),
                          ("spmv_er_large_traffic.txt", bench.SPMV_SOURCES)]:
        path = os.path.join(ROOT, "profiles", name)
        assert os.path.exists(path), name
        fields = dict(l.split(":", 1) for l in open(path) if ":" in l and not l.startswith("#"))
        assert float(fields["dram_bytes_per_launch"]) > 0
        assert len(fields["kernel_source_hash"].strip()) == 16


def test_clock_sampler_parses_rows():
    cs = bench.ClockSampler(0)

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class T:
        def join(self, timeout=None):
            pass

    cs.proc, cs.t = Done(), T()
    cs.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["0", "1980", "2070", "1400", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
               ["0", "2070", "2070", "950", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["garbled"]]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_command_line_help_runs_without_a_gpu():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0
    for opt in ("--workload", "--tuning", "--scale", "--eliminate", "--impl"):
        assert opt in r.stdout
