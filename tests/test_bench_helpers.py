"""Host logic of the benchmark's measurement (no GPU): the algorithmic bytes of one recovery behind the roofline
fraction, the per-step rows, and the rule that a committed ncu figure is reported only while the CUDA sources it
was taken on are unchanged."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_path_bytes_headline():
    # mesh 128^3: n = 2^21, m = 3 * 128^2 * 127, one off-tree edge per edge beyond the tree, k = floor(.10 n)
    n, side = 1 << 21, 128
    m = 3 * side * side * (side - 1)
    E = m - n + 1
    k = int(0.10 * n)
    assert (m, E, k) == (6242304, 4145153, 209715)
    # the CSR and parent, depth and D written and read, one 24-byte record written and read per off-tree edge,
    # the output ids
    assert bench.path_bytes(n, m, E, k) == 8 * (n + 1) + 24 * m + 4 * n + 40 * n + 48 * E + 4 * k == 458673412


def test_step_rows():
    avg = {s: 0.5 for s in ("classify", "tree", "score", "select", "sort", "accept", "budget")}
    avg["budget"] = 0.0
    by = {s: 1e6 for s in avg}
    rows = bench.step_list(avg, by, 4000.0)
    assert [r["step"] for r in rows] == list(avg)
    assert rows[0]["gbs"] == pytest.approx(2.0) and rows[0]["frac"] == pytest.approx(0.0005)
    assert rows[-1]["gbs"] is None and rows[-1]["frac"] is None


def _fake_tree(tmp_path, src: bytes):
    d = tmp_path / "paper_2508_20403_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "pdg_score.cu").write_bytes(src)
    (d / "other.cuh").write_bytes(b"// header\n")
    (tmp_path / "profiles").mkdir()
    return d


def test_recovery_traffic_only_for_unchanged_sources(tmp_path, monkeypatch):
    d = _fake_tree(tmp_path, b"__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.sources_digest()
    (tmp_path / "profiles" / "recovery_traffic_w.md").write_text(
        f"- dram bytes per recovery: 123456\n- sources sha256: `{digest}`\n")
    assert bench.ncu_recovery_traffic("w") == 123456.0
    (d / "pdg_score.cu").write_bytes(b"__global__ void k() { int x; }\n")  # the kernels changed since the capture
    assert bench.ncu_recovery_traffic("w") is None
    assert bench.ncu_recovery_traffic("missing") is None


def test_kernel_traffic_only_for_unchanged_kernel(tmp_path, monkeypatch):
    import hashlib

    src = b"__global__ void k_score() {}\n"
    d = _fake_tree(tmp_path, src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = hashlib.sha256(src).hexdigest()
    (tmp_path / "profiles" / "k_score_w.md").write_text(
        "- dram bytes per launch: 1000\n"
        "- dram bytes per launch (scaled to mesh 128^3 by off-tree edges, x 1.21459): 1215\n"
        f"- kernel source sha256: `{sha}`\n")
    assert bench.ncu_traffic("k_score", "w") == 1215.0  # the scaled figure wins when present
    (d / "other.cuh").write_bytes(b"// another header\n")  # only the kernel's own file counts
    assert bench.ncu_traffic("k_score", "w") == 1215.0
    (d / "pdg_score.cu").write_bytes(src + b"// edited\n")
    assert bench.ncu_traffic("k_score", "w") is None


class _FakeNvml:
    max_mhz = 2070.0

    def __init__(self, samples):
        self.samples = samples


def test_clock_record_from_nvml_samples():
    cs = bench.ClockSampler(0)
    bits = bench._NvmlSampler.BITS
    cs.nvml = _FakeNvml([(2070.0, 0), (2070.0, bits["sw_power_cap"]), (1965.0, bits["hw_slowdown"]), (2070.0, 0)])
    rec = cs.summary()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 4
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]
    cs.nvml = _FakeNvml([])
    assert cs.summary()["reasons"] == ["no samples"]


def test_clock_record_from_nvidia_smi_csv(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    cs.proc = object()  # the sampler ran
    rows = ["0, 2070, 2070, 905.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # unreadable sample
            "0, 2070, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active"]
    (tmp_path / "clocks.csv").write_text("\n".join(rows) + "\n")
    rec = cs.summary()
    assert rec["samples"] == 3 and rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["source"] == "nvidia-smi"
