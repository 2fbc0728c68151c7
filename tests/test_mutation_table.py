"""The slips of tests/mutate_oracle.py still match the oracle's source text, so
the mutation check keeps testing what it names after the oracle is edited."""
import os

import mutate_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_slip_matches_the_oracle_source():
    src = open(os.path.join(ROOT, "oracle", "lb_oracle.c")).read()
    assert len(mutate_oracle.M) >= 40
    for name, text, repl, count in mutate_oracle.M:
        assert src.count(text) == count, name
        assert src.replace(text, repl) != src, name
