"""Repository rules that need no GPU.

- No committed source file refers to the scratch folder (its name is built below, so this
  file does not match its own pattern); review and result files that the build pipeline
  writes at the repository root are not product source and are skipped.
- Every command quoted in a profile summary runs committed scripts only, and every `ncu` command
  there leaves the GPU clocks alone (`--clock-control none`).
- An `ncu` command that collects more than the launch list (`--set`, `--section`, or `--metrics`
  beyond `gpu__time_duration.sum`) captures one kernel (`-k` with a single name, no alternation)
  and a bounded number of launches (`-c`).
"""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRATCH = "_" + "work/"
# written by the build pipeline, not by this project's sources
PIPELINE_FILES = re.compile(r"^(VERDICT|ADVICE|SURVEY|BASELINE)\.md$|^(BENCH|GPUTEST|SCALE|MULTICHIP)_r\d+\.json$"
                            r"|^PROGRESS\.jsonl$|^BASELINE\.json$")


def _tracked():
    out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    return [l for l in out.splitlines() if l]


def test_no_committed_file_refers_to_scratch():
    pat = re.compile(r"(^|[^A-Za-z0-9_])" + re.escape(SCRATCH))
    bad = []
    for f in _tracked():
        if f == ".gitignore" or PIPELINE_FILES.match(f):
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


def _ncu_commands(txt):
    # a command: `ncu` followed by a flag, up to the closing backtick or a blank line
    return re.findall(r"ncu\s+-{1,2}[A-Za-z].*?(?=`|\n\s*\n|\Z)", txt, flags=re.S)


def _profile_summaries():
    prof = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.endswith((".md", ".txt"))]
    assert names
    return [(n, open(os.path.join(prof, n), encoding="utf-8").read()) for n in names]


def test_profile_commands_run_committed_scripts():
    tracked = set(_tracked())
    for name, txt in _profile_summaries():
        scripts = re.findall(r"python3?\s+(?:-m\s+\S+\s+)?([\w./-]+\.py)", txt)
        assert scripts, name
        for s in scripts:
            assert s in tracked, (name, s)
        for cmd in _ncu_commands(txt):
            if re.match(r"ncu\s+(-i|--import)\b", cmd):
                continue   # reading a saved report runs nothing on a GPU
            assert "--clock-control none" in cmd, (name, cmd[:160])


def test_full_captures_name_one_kernel():
    for name, txt in _profile_summaries():
        for cmd in _ncu_commands(txt):
            if re.match(r"ncu\s+(-i|--import)\b", cmd):
                continue
            metrics = re.findall(r"--metrics\s+(\S+)", cmd)
            heavy = ("--set" in cmd or "--section" in cmd
                     or any(m.strip("'\"") != "gpu__time_duration.sum" for m in metrics))
            if not heavy:
                continue
            k = re.search(r"(?:-k|--kernel-name)\s+(\S+)", cmd)
            assert k, (name, "a heavy capture must name its kernel", cmd[:160])
            kname = k.group(1).strip("'\"")
            assert "|" not in kname, (name, "one kernel per heavy capture", kname)
            c = re.search(r"(?:-c|--launch-count)\s+(\d+)", cmd)
            assert c and int(c.group(1)) <= 3, (name, "at most three launches per heavy capture", cmd[:160])
