"""The committed ncu summaries are short text, each with the full ncu command that made it (with
--clock-control none), running committed entry points only (bench.py or the package's
profile_case); the level-0 traffic record parses and holds what bench.py reads from it."""
import glob
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))


def test_profiles_are_short_text_with_their_commands():
    assert FILES
    for f in FILES:
        assert f.endswith((".md", ".txt")), f
        text = open(f).read()
        assert len(text.encode()) < 16 * 1024, f
        assert "ncu " in text and "--clock-control none" in text, f
        assert "_work" not in text, f
        for cmd in re.findall(r"python3? (?:-m )?(\S+)", text):
            assert cmd in ("bench.py", "paper_1212_6680_gb300.profile_case"), (f, cmd)


def test_traffic_record_parses():
    d = json.load(open(os.path.join(ROOT, "profiles", "plane_lean_traffic_level0_128cube.txt")))
    for key in ("dram_bytes_per_launch", "launches", "source_hash", "sources", "command"):
        assert key in d, key
    assert d["dram_bytes_per_launch"] == sum(d["launches"]) / len(d["launches"])
    assert len(d["source_hash"]) == 16
