"""Every profile summary under profiles/ names the command that made it, and
that command runs committed files only: each `python bench.py ...` line in
them parses with bench.py's own arguments, and every summary gives the ncu
clock flag that leaves the GPU's clocks alone."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def bench_commands(text):
    out = []
    for line in text.splitlines():
        m = re.search(r"python bench\.py([^\"\n`]*)", line)
        if m:
            out.append(shlex.split(m.group(1).replace("\\", " ")))
    return out


def test_there_are_profiles():
    assert len(PROFILES) >= 3


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_profile_commands_parse(path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    text = open(path).read()
    cmds = bench_commands(text)
    assert cmds, "no bench.py command"
    for args in cmds:
        monkeypatch.setattr(sys, "argv", ["bench.py", *args])
        bench.parse()                      # argparse exits on an unknown flag
    assert "--clock-control none" in text
    assert "_work" not in text and "gpurun" not in text
