"""The oracle reproduces its committed snapshots (tests/golden/), bit for bit.

Run once on the CPU here and once (marked gpu) on the GPU host, whose CPU is
a different architecture: the oracle must give the same bits on both.
"""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def check():
    want = json.load(open(os.path.join(HERE, "golden", "oracle_snapshots.json")))
    got = [make_golden.snapshot(*c) for c in make_golden.cases()]
    assert got == want


def test_oracle_matches_snapshots():
    check()


@pytest.mark.gpu
def test_oracle_matches_snapshots_on_gpu_host():
    check()
