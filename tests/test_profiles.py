"""The committed ncu summaries: short text files, each giving the command
that made it (every ncu invocation with --clock-control none, run on
committed files), and the engine summary carries the keys bench.py reads."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_profile_summaries():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))
    assert files
    for f in files:
        assert f.endswith((".txt", ".md")), f
        assert os.path.getsize(f) < 16_000, f
        text = open(f).read()
        assert "command" in text, f
        for ln in text.splitlines():
            # an ncu invocation (its options start on the line that names ncu)
            if "ncu --" in ln and ("python " in ln or ln.rstrip().endswith("\\")):
                assert "--clock-control none" in ln, (f, ln)


def test_engine_profile_keys():
    text = open(os.path.join(ROOT, "profiles", "k_engine_bench_ant1m_d6.txt")).read()
    keys = dict(re.findall(r"^# key (\S+) = (\S+)$", text, flags=re.M))
    assert int(keys["dram_bytes_per_step"]) > 0
    assert re.fullmatch(r"[0-9a-f]{64}", keys["engine_source_sha256"])
