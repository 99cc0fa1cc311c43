"""The ncu summaries under profiles/: each names the full command that made
it, that command runs committed files with options bench.py accepts, and
every ncu command in them leaves the GPU clocks alone (--clock-control
none)."""
import glob
import os
import re
import shlex
import shutil
import subprocess

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def commands(path):
    """The indented (code) lines of a summary, backslash continuations joined."""
    out, cur = [], ""
    for line in open(path, encoding="utf-8"):
        if not line.startswith("    "):
            if cur:
                out.append(cur)
                cur = ""
            continue
        text = line.strip()
        if text.endswith("\\"):
            cur += text[:-1] + " "
        else:
            out.append(cur + text)
            cur = ""
    if cur:
        out.append(cur)
    return [c for c in out if c]


def bench_args(cmd):
    """The arguments a command passes to bench.py."""
    tail = cmd.split("python bench.py", 1)[1]
    args = []
    for tok in shlex.split(tail):
        if tok in (";", "done", "&&", "|") or tok.startswith(">"):
            break
        args.append(tok)
    return args


def test_there_are_summaries():
    assert len(SUMMARIES) >= 4


@pytest.mark.parametrize("path", SUMMARIES, ids=os.path.basename)
def test_summary_commands(path):
    cmds = commands(path)
    runs = [c for c in cmds if "python bench.py" in c]
    assert runs, "no bench.py command in " + path
    parser = bench.arg_parser()
    for c in runs:
        parser.parse_args(bench_args(c))  # exits on an option bench.py does not take
    profiled = [c for c in cmds if c.startswith("ncu ") or " ncu " in c]
    assert profiled, "no ncu command in " + path
    for c in profiled:
        assert "--clock-control none" in c, c
    for c in cmds:  # committed files only: no scratch folders
        assert "_work/" not in c and "gpurun_out/" not in c, c


@pytest.mark.parametrize("path", SUMMARIES, ids=os.path.basename)
def test_summary_code_is_valid_shell(path):
    """The indented block parses as bash (bash -n runs nothing), and no
    variable assignment is continued onto an indented line (the indentation
    would end the assignment there)."""
    code = "".join(line[4:] for line in open(path, encoding="utf-8") if line.startswith("    "))
    assert not re.search(r"^[A-Za-z_][A-Za-z0-9_]*=\S*\\$", code, re.M), path
    bash = shutil.which("bash")
    if bash is None:
        pytest.skip("no bash")
    r = subprocess.run([bash, "-n"], input=code, text=True, capture_output=True)
    assert r.returncode == 0, r.stderr
