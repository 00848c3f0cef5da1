"""The commands the profile summaries give run committed code: every `python bench.py ...`
command line in profiles/*.md parses with the benchmark's own argument parser, and every ncu
command leaves the GPU clocks alone (--clock-control none).  No GPU needed."""
import os
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands():
    cmds = []
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, name)).read().replace("\\\n", " ")
        for line in text.splitlines():
            line = line.strip()
            if line.startswith(("python ", "ncu ")):
                cmds.append((name, line))
    return cmds


def test_profile_commands_run_committed_code():
    sys.path.insert(0, ROOT)
    import bench
    cmds = _commands()
    bench_lines = 0
    for name, line in cmds:
        words = shlex.split(line)
        if words[0] == "ncu":
            assert "--clock-control" in words, (name, line)
            assert words[words.index("--clock-control") + 1] == "none", (name, line)
        if "bench.py" not in words:
            continue
        argv = words[len(words) - 1 - words[::-1].index("bench.py") + 1:]
        saved = sys.argv
        try:
            sys.argv = ["bench.py"] + argv
            bench.parse()  # argparse exits on an unknown flag or value
        finally:
            sys.argv = saved
        bench_lines += 1
    assert bench_lines >= 5, cmds
