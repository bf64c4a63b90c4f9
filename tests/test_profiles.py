"""The ncu summaries under profiles/ each give the command that made them;
every `python bench.py ...` in them must still be accepted by bench.py, and
every ncu command must keep the clocks unlocked."""
import glob
import os
import re
import shlex

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(path):
    """Indented command blocks of a summary, with backslash continuations joined."""
    text = open(path).read().replace("\\\n", " ")
    return [ln.strip() for ln in text.splitlines() if ln.startswith("    ") and ("ncu " in ln or "bench.py" in ln)]


def test_every_summary_gives_a_command_that_runs_committed_files():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert len(files) >= 5
    for path in files:
        if os.path.basename(path) == "README.md":
            continue
        cmds = _commands(path)
        assert cmds, f"{path}: no command given"
        for cmd in cmds:
            words = shlex.split(cmd)
            if words[0] == "ncu":
                assert "--clock-control" in words and words[words.index("--clock-control") + 1] == "none", cmd
            assert "python" in words and "bench.py" in words, cmd
            args = words[words.index("bench.py") + 1:]
            parsed = bench.make_parser().parse_args(args)
            assert set(parsed.parts.split(",")) <= set(bench.PARTS), cmd
            assert not re.search(r"_work|gpurun_out/\w+\.py", cmd), cmd
