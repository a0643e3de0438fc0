"""The mistake-planting check itself works: a planted slip in a scratch copy of the oracle is caught
by the pins, and the repository's own oracle is left untouched.  (The whole list of plantings runs
with `python tests/plant_mistakes.py`, about ten minutes.)"""
import hashlib
import os

import plant_mistakes as PM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _digest(path):
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def test_a_planted_slip_is_caught(tmp_path):
    before = _digest("oracle/oracle.c")
    entry = next(m for m in PM.MUTATIONS if m[0] == "emission_peel_4pi")
    status, msg = PM.run(str(tmp_path / "scratch"), *entry)
    assert status == "caught", msg
    assert _digest("oracle/oracle.c") == before


def test_every_planting_matches_the_oracle_source_once():
    src = {p: open(os.path.join(ROOT, p)).read() for p in ("oracle/oracle.c", "oracle/oracle.py")}
    for name, path, old, new in PM.MUTATIONS:
        assert src[path].count(old) == 1, name
        assert old != new, name
