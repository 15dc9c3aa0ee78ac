"""Host checks of bench.py's bookkeeping (no GPU)."""
import os
import re

import bench

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1503_03337_gb300", "csrc")


def local_includes(name, seen):
    """The csrc files a source includes, transitively."""
    if name in seen or not os.path.exists(os.path.join(CSRC, name)):
        return seen
    seen.add(name)
    for inc in re.findall(r'#include "([^"]+)"', open(os.path.join(CSRC, name)).read()):
        if "/" not in inc:
            local_includes(inc, seen)
    return seen


def test_kernel_source_hash_covers_step_sources():
    """The recorded DRAM traffic is reported only while the hash over the
    step kernel's sources matches; every file the single-domain step units
    include must therefore be part of that hash."""
    covered = set(re.findall(r'"(lbm_[a-z0-9_]+\.(?:cuh|cu|h))"',
                             open(bench.__file__).read().split("def kernel_source_hash")[1]
                             .split("def ")[0]))
    units = [f for f in os.listdir(CSRC) if re.fullmatch(r"lbm_step_q1[48][hb]?\.cu", f)]
    assert len(units) == 6
    needed = set()
    for u in units + ["lbm_step.cu"]:
        local_includes(u, needed)
    needed.discard("lbm_internal.h")  # host-side descriptor, no kernel code
    assert needed <= covered, sorted(needed - covered)


def test_recorded_traffic_needs_matching_hash(tmp_path, monkeypatch):
    """A traffic figure is reported under the current source hash only."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "1111111111111111")
    for recorded, expect in (("0000000000000000", None), ("1111111111111111", 299000000.0)):
        (prof / "step_kernel_dram_traffic.txt").write_text(
            "source_hash: %s\nQ18 f32 128^3: 299000000  (algorithmic 301989888)\n" % recorded)
        assert bench.recorded_traffic(18, "f32", 128) == expect
        assert bench.recorded_traffic(14, "f32", 128) is None
