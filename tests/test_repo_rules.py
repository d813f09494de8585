"""CPU checks of the repository's own rules.

* Every ncu command recorded under profiles/ leaves the GPU clocks alone
  (--clock-control none), and each summary names the command it came from.
* profiles/ holds short text summaries only, nothing that runs.
* No committed source, test or script reads the git-ignored working folder.
"""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def tracked():
    out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    if out.returncode != 0:          # not a git checkout: walk the tree instead
        files = []
        for d, dirs, fs in os.walk(ROOT):
            dirs[:] = [x for x in dirs if not x.startswith((".", "_")) and x != "gpurun_out"]
            files += [os.path.relpath(os.path.join(d, f), ROOT) for f in fs]
        return files
    return [f for f in out.stdout.split("\n") if f]


def test_profile_commands_leave_clocks_alone():
    names = sorted(f for f in os.listdir(PROFILES) if not f.startswith("."))
    assert names
    for f in names:
        assert f.endswith((".txt", ".md")), f
        text = open(os.path.join(PROFILES, f)).read()
        assert len(text) < 16_000, f
        assert re.search(r"^commands? \(", text, re.M), f"{f}: no command recorded"
        runs = [l for l in text.split("\n") if re.match(r"\s*ncu\s+-", l)]
        assert runs, f"{f}: no ncu command line"
        for l in runs:
            assert "--clock-control none" in l, (f, l)


def test_nothing_committed_reads_the_working_folder():
    for f in tracked():
        if f.endswith(".md") or f in (".gitignore", ".gpurunignore") or f.startswith(("profiles/",)):
            continue
        path = os.path.join(ROOT, f)
        if not os.path.isfile(path) or os.path.getsize(path) > 2_000_000:
            continue
        try:
            text = open(path, encoding="utf-8").read()
        except UnicodeDecodeError:
            continue
        if f == "tests/test_repo_rules.py":
            continue
        assert not re.search(r"(?<![\w.])_work\b", text), f


def test_no_top_level_tool_folders():
    for d in ("tools", "scripts"):
        assert not os.path.isdir(os.path.join(ROOT, d)), d
