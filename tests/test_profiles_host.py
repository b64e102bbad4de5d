"""The committed ncu summaries stay tied to the sources they describe (no GPU needed).

bench.py reports a kernel's DRAM traffic from profiles/traffic.json only while the digest
recorded there matches the current tile-kernel sources; these checks keep the committed
figures and their summaries consistent with that rule."""

import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_digest_matches_tile_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    sha = bench.tile_source_sha()
    for key, e in d.items():
        assert e["tile_sources_sha"] == sha, key
        assert e["dram_bytes_per_launch"] > 0, key
        assert os.path.exists(os.path.join(ROOT, e["summary"])), key
        assert bench._committed_traffic(key) == e["dram_bytes_per_launch"]


def test_profile_summaries_state_their_commands():
    """Every summary under profiles/ gives the command that made it, with the profiler's
    clock control left to the GPU (no clock locking) and only committed files run."""
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(ROOT, "profiles", name)) as f:
            text = f.read()
        assert "ncu " in text, name
        for line in text.splitlines():
            if line.strip().startswith("ncu "):
                assert "--clock-control none" in line, (name, line)
        assert "_work/" not in text, name
