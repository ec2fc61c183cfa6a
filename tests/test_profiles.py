"""CPU checks of the committed profile summaries: each names the full command
that produced it, and those commands run committed files only."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(text):
    for block in re.findall(r"```\n(.*?)```", text, flags=re.S):
        yield from (l.strip() for l in block.replace("\\\n", " ").splitlines() if l.strip())


def test_summaries_name_their_commands_and_run_committed_files():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for f in files:
        cmds = list(_commands(open(f).read()))
        assert cmds, f
        for c in cmds:
            assert c.startswith(("python ", "ncu ")), (f, c)
            for script in re.findall(r"python (\S+\.py)", c):
                assert os.path.isfile(os.path.join(ROOT, script)), (f, script)
            assert "_work" not in c and "/root/" not in c, (f, c)


def test_only_text_in_profiles():
    for f in glob.glob(os.path.join(ROOT, "profiles", "*")):
        assert os.path.splitext(f)[1] in (".md", ".txt", ".json"), f
        assert os.path.getsize(f) < 64 * 1024, f
