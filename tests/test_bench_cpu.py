"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports for
a kernel comes from the committed ncu summary (bytes per atom of the
captured case times the atoms of the launch), and from nowhere once the
kernel sources differ from the ones the counters were taken on."""
import os

import pytest

import bench


def _summary(root, kernel, per_atom, sha):
    d = os.path.join(root, "profiles")
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, f"{kernel}.md"), "w") as f:
        f.write(f"# {kernel}\n\nReading.  A capture.\n\ntraffic_bytes_per_atom = {per_atom}\nsources_sha1 = {sha}\n")


def test_traffic_scales_the_captured_bytes_per_atom(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "0123abcd")
    _summary(str(tmp_path), "k_demo", 913.29, "0123abcd")
    assert bench.profiled_traffic("k_demo", 1_000_000) == pytest.approx(913.29e6)
    assert bench.profiled_traffic("k_demo", 262_144) == pytest.approx(913.29 * 262_144)
    assert bench.profiled_traffic("k_absent", 1000) is None


def test_no_traffic_once_the_kernel_sources_change(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "ffff0000")
    _summary(str(tmp_path), "k_demo", 500.0, "0123abcd")
    assert bench.profiled_traffic("k_demo", 1000) is None


def test_summary_without_a_figure_gives_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "0123abcd")
    os.makedirs(os.path.join(str(tmp_path), "profiles"))
    with open(os.path.join(str(tmp_path), "profiles", "k_demo.md"), "w") as f:
        f.write("sources_sha1 = 0123abcd\n")
    assert bench.profiled_traffic("k_demo", 1000) is None


@pytest.mark.parametrize("kernel", ["k_cv_fwd", "k_cv_avg", "k_adjoint", "k_force_pairs", "k_force_gather"])
def test_committed_summaries_record_their_figure_and_sources(kernel):
    with open(os.path.join(bench.ROOT, "profiles", f"{kernel}.md")) as f:
        text = f.read()
    lines = text.splitlines()
    assert any(line.startswith("traffic_bytes_per_atom = ") for line in lines)
    sha = [line.split("=", 1)[1].strip() for line in lines if line.startswith("sources_sha1 = ")]
    assert len(sha) == 1 and len(sha[0]) == 40
    assert "ncu " in text and "--clock-control none" in text
