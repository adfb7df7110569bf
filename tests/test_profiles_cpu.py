"""The ncu summaries under profiles/ stay reproducible (no GPU): each names
the command that made it, and every bench command in them uses only options
that bench.py defines."""

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _bench_options():
    src = open(os.path.join(ROOT, "bench.py")).read()
    return set(re.findall(r'add_argument\(\s*"(--[a-z0-9-]+)"', src))


def test_every_summary_gives_its_command():
    names = sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))
    assert names
    for f in names:
        txt = open(os.path.join(PROFILES, f)).read()
        assert "ncu " in txt and "--clock-control none" in txt, f
        assert "python bench.py" in txt, f


def test_bench_commands_use_defined_options():
    opts = _bench_options()
    assert {"--steps", "--warmup", "--seqs", "--only"} <= opts
    for f in sorted(os.listdir(PROFILES)):
        for line in open(os.path.join(PROFILES, f)):
            if "python bench.py" not in line:
                continue
            tail = line.split("python bench.py", 1)[1]
            used = set(re.findall(r"(?<![\w-])(--[a-z0-9-]+)", tail))
            assert used <= opts, (f, used - opts)
