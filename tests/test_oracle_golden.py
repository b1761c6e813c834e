"""The oracle still reproduces its frozen trace (tests/golden/oracle_trace.json,
written by tests/golden/make_oracle_golden.py from oracle/ only)."""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_oracle_golden as G  # noqa: E402


def test_oracle_trace_is_unchanged():
    with open(os.path.join(HERE, "golden", "oracle_trace.json")) as f:
        want = json.load(f)["runs"]
    for name, spec in G.RUNS.items():
        assert want[name]["spec"] == spec
        assert G.trace(spec) == want[name]["trace"], name
