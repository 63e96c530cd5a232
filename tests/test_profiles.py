"""The committed ncu summaries under profiles/ against the sources they describe.

bench.py reports a kernel's DRAM traffic, L1 data-pipe and issue fractions only
from a summary whose source key (a hash of the kernel's sources with comments
and whitespace removed) matches the code being built; these checks fail as soon
as the kernel sources change without a new capture, and check that every ncu
command in the summaries leaves the GPU clocks alone."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_march_records_match_the_march_sources():
    assert bench.recorded_traffic() is not None
    assert bench.recorded_value("l1_wavefronts_frac") is not None
    assert bench.recorded_value("issue_active_frac") is not None
    traffic = bench.recorded_traffic()
    # the quads the rays reach: between the volume once (0.54 GB) and all quads (2.2 GB)
    assert 0.5e9 < traffic < 2.2e9


def test_mesh_record_matches_the_mesh_sources():
    t = bench.recorded_traffic("mesh_workload.md", bench.MESH_SOURCES)
    assert t is not None and 0.5e9 < t < 2.6e9


def test_launch_list_names_the_current_march_key():
    key = bench.source_key(("vr_kernels.cu", "vr_device.cuh", "vr_internal.h"))
    text = open(os.path.join(PROFILES, "launches_paper_workload.md")).read()
    assert "source key %s" % key in text


def test_summaries_are_short_text_and_every_ncu_command_keeps_the_clocks():
    for name in os.listdir(PROFILES):
        path = os.path.join(PROFILES, name)
        assert name.endswith((".md", ".txt")), name
        assert os.path.getsize(path) < 32 * 1024, name
        text = open(path).read()
        # an ncu command may continue over backslash-ended lines
        joined = re.sub(r"\\\n\s*", " ", text)
        for line in joined.splitlines():
            for cmd in re.findall(r"\bncu\s+--[^`]*", line):
                if " -i " not in cmd:
                    assert "--clock-control none" in cmd, (name, cmd)
