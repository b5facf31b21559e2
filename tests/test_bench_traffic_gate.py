"""The gate on the recorded ncu counters in bench.py (CPU).

bench.py reports the DRAM traffic of the sweep kernel from a committed ncu
record only while the kernel's sources hash to the value the record was
taken on.  The hash covers the device code: aug_spmmv.cuh, the staged
kernel's file up to its host launch helpers, and the device-side interface
part of kpm_internal.h, without comments or blank lines.  These tests edit
copies of the sources and check that a device edit changes the hash, that
comment and host-helper edits do not, and that a record on other sources
reads as absent."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSRC = ("paper_1410_5242_gb300", "csrc")
STAGED = "aug_spmmv_staged.cu"


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    """A copy of the hashed sources, with bench.py pointed at it."""
    dst = tmp_path.joinpath(*CSRC)
    dst.mkdir(parents=True)
    for f in set(bench.KERNEL_SOURCES["fp32"]) | set(bench.KERNEL_SOURCES["fp64"]):
        shutil.copy(os.path.join(ROOT, *CSRC, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def edit(path, old, new):
    text = path.read_text()
    assert text.count(old) == 1, old
    path.write_text(text.replace(old, new))


def test_markers_are_in_the_sources():
    staged = open(os.path.join(ROOT, *CSRC, STAGED)).read()
    internal = open(os.path.join(ROOT, *CSRC, "kpm_internal.h")).read()
    assert staged.count(bench.HOST_BEGIN) == 1
    # the kernel itself lies before the host helpers
    assert staged.index("aug_spmmv_staged_kernel(") < staged.index(bench.HOST_BEGIN)
    assert internal.index(bench.INTERFACE_BEGIN) < internal.index(bench.INTERFACE_END)


def test_copy_hashes_like_the_tree(tree):
    h = bench.kernel_hash("fp32")
    assert h == bench.kernel_hash("fp64")
    assert len(h) == 12


def test_host_helper_and_comment_edits_keep_the_hash(tree):
    h0 = bench.kernel_hash("fp32")
    staged = tree / STAGED
    text = staged.read_text()
    staged.write_text(text + "\nstatic int kpm_gate_probe_host = 0;\n")
    assert bench.kernel_hash("fp32") == h0
    edit(staged, bench.HOST_BEGIN, bench.HOST_BEGIN + "\n// another comment line\n")
    assert bench.kernel_hash("fp32") == h0
    internal = tree / "kpm_internal.h"
    edit(internal, bench.INTERFACE_END, "int kpm_gate_probe_after_interface();\n"
         + bench.INTERFACE_END)
    assert bench.kernel_hash("fp32") != h0  # still inside the interface part
    edit(internal, "int kpm_gate_probe_after_interface();\n", "")
    assert bench.kernel_hash("fp32") == h0
    edit(internal, bench.INTERFACE_BEGIN, "// a comment\n" + bench.INTERFACE_BEGIN)
    assert bench.kernel_hash("fp32") == h0


def test_device_edits_change_the_hash(tree):
    h0 = bench.kernel_hash("fp32")
    staged = tree / STAGED
    text = staged.read_text()
    cut = text.index(bench.HOST_BEGIN)
    staged.write_text(text[:cut] + "__device__ int kpm_gate_probe_device;\n" + text[cut:])
    assert bench.kernel_hash("fp32") != h0
    staged.write_text(text)
    assert bench.kernel_hash("fp32") == h0
    cuh = tree / "aug_spmmv.cuh"
    cuh.write_text(cuh.read_text() + "\n__device__ int kpm_gate_probe_cuh;\n")
    assert bench.kernel_hash("fp64") != h0


def test_record_on_other_sources_reads_as_absent(tree, tmp_path, monkeypatch):
    h = bench.kernel_hash("fp32")
    rec = tmp_path / "traffic.txt"
    rec.write_text("# comment line\n"
                   "fp32_kernel_hash %s\nfp32_dram_bytes_per_launch 123456\n"
                   "fp64_kernel_hash 000000000000\nfp64_dram_bytes_per_launch 654321\n" % h)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.measured_traffic("fp32") == 123456.0
    assert bench.measured_traffic("fp64") is None
    assert "none" in bench.traffic_source("fp64", None)
    assert h in bench.traffic_source("fp32", 123456.0)
    staged = tree / STAGED
    text = staged.read_text()
    cut = text.index(bench.HOST_BEGIN)
    staged.write_text(text[:cut] + "__device__ int kpm_gate_probe_device;\n" + text[cut:])
    assert bench.measured_traffic("fp32") is None
