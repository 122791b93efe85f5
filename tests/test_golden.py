"""Every stored fixture under tests/golden/ says where its values come from
(a passage of the paper or a published reference) and is used by a test."""
import os
import re

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_fixtures_carry_a_citation_and_are_used():
    names = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
    assert names
    here = os.path.dirname(os.path.abspath(__file__))
    tests = "".join(open(os.path.join(here, f)).read() for f in os.listdir(here)
                    if f.startswith("test_") and f.endswith(".py") and f != "test_golden.py")
    for name in names:
        header = "".join(ln for ln in open(os.path.join(GOLDEN, name)) if ln.startswith("#"))
        assert re.search(r"arxiv 2608\.15253|\(\d{4}\)|'\d\d\b|\b(19|20)\d\d\b", header), name
        assert name in tests, name
