"""Host logic of bench.py that needs no GPU: the source regions its traffic
figures are tied to.  The committed ncu summaries under profiles/ carry the
hash of the kernel source they were measured on; bench.py reports a traffic
figure only while the source still hashes the same.  These checks keep that
link honest: each region's markers are present (so the hash covers the
kernel, not the whole file by accident), an edit inside a region changes its
hash while an edit elsewhere in the file does not, and the summaries match
the sources as committed."""
import os
import re

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_2110_07519_gb300", "csrc")
REGIONS = {
    "k_tc_screen": ("screen.cu", b"struct ScreenArgs {",
                    b"// ----------------------------------------------------------- recheck"),
    "k_lb_scan": ("query.cu", b"struct ScanCodes {",
                  b"// ------------------------------------------------------------ ED refine"),
}


@pytest.mark.parametrize("kernel", sorted(REGIONS))
def test_region_markers_present(kernel):
    name, a, b = REGIONS[kernel]
    text = open(os.path.join(CSRC, name), "rb").read()
    i, j = text.find(a), text.find(b)
    assert 0 <= i < j, (kernel, i, j)
    assert kernel.encode() in text[i:j]            # the kernel itself lies inside


@pytest.mark.parametrize("kernel", sorted(REGIONS))
def test_hash_follows_the_region_only(kernel, tmp_path, monkeypatch):
    name, a, b = REGIONS[kernel]
    root = tmp_path / "repo"
    csrc = root / "paper_2110_07519_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("screen.cu", "query.cu", "tc.cuh", "device_common.cuh"):
        (csrc / f).write_bytes(open(os.path.join(CSRC, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(root))
    base = bench.scan_source_sha(kernel)
    text = (csrc / name).read_bytes()
    # outside the region: the hash stays
    (csrc / name).write_bytes(b"// a comment above the region\n" + text)
    assert bench.scan_source_sha(kernel) == base
    # inside the region: the hash moves
    i = text.find(a) + len(a)
    (csrc / name).write_bytes(text[:i] + b" /* changed */" + text[i:])
    assert bench.scan_source_sha(kernel) != base


@pytest.mark.parametrize("kernel", sorted(REGIONS))
def test_committed_traffic_summaries_match_the_sources(kernel):
    text = open(os.path.join(bench.ROOT, "profiles", f"{kernel}_traffic.txt")).read()
    sha = re.search(r"source_sha:\s*(\w+)", text).group(1)
    assert sha == bench.scan_source_sha(kernel), \
        f"{kernel} changed since its traffic was captured: capture it again"
    per = float(re.search(r"dram_bytes_per_(?:series|word):\s*([0-9.eE+-]+)", text).group(1))
    assert bench.profiled_traffic(1000.0, kernel) == pytest.approx(per * 1000.0)
