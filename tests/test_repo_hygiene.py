"""Repository rules that need no GPU.

- No committed file refers to the `_work/` folder, which holds uncommitted scratch work.
- Every command quoted in a profile summary runs committed scripts only, and every `ncu` command
  there leaves the GPU clocks alone (`--clock-control none`)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    return [l for l in out.splitlines() if l]


def test_no_committed_file_refers_to_scratch():
    pat = re.compile(r"(^|[^A-Za-z0-9_])_work/")
    bad = []
    for f in _tracked():
        if f == ".gitignore":
            continue
        p = os.path.join(ROOT, f)
        if not os.path.isfile(p):
            continue
        try:
            txt = open(p, encoding="utf-8").read()
        except UnicodeDecodeError:
            continue
        if pat.search(txt):
            bad.append(f)
    assert not bad, bad


def test_profile_commands_run_committed_scripts():
    tracked = set(_tracked())
    prof = os.path.join(ROOT, "profiles")
    summaries = [f for f in os.listdir(prof) if f.endswith((".md", ".txt"))]
    assert summaries
    for name in summaries:
        txt = open(os.path.join(prof, name), encoding="utf-8").read()
        scripts = re.findall(r"python3?\s+(?:-m\s+\S+\s+)?([\w./-]+\.py)", txt)
        assert scripts, name
        for s in scripts:
            assert s in tracked, (name, s)
        # a command: `ncu` followed by a flag, up to the closing backtick or a blank line
        for cmd in re.findall(r"ncu\s+-{1,2}[A-Za-z].*?(?=`|\n\s*\n|\Z)", txt, flags=re.S):
            if re.match(r"ncu\s+(-i|--import)\b", cmd):
                continue   # reading a saved report runs nothing on a GPU
            assert "--clock-control none" in cmd, (name, cmd[:160])
