"""Golden fixtures under tests/golden/: two worked examples derived by hand
(their derivations are in the files) and one oracle regression file written
by tests/golden/make_golden.py."""
import os

import numpy as np
import pytest

import oracle
from workloads import config

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vals = line.split()
            out[k] = np.array([float(v) for v in vals])
    return out


@pytest.mark.parametrize("name", ["cartesian_2x3.txt", "keyed_join_2keys.txt"])
def test_hand_derived_examples(name):
    fx = read_fixture(name)
    A, B = fx["A"].reshape(-1, 1), fx["B"].reshape(-1, 1)
    kA, kB = fx["keyA"].astype(np.int32), fx["keyB"].astype(np.int32)
    for route in ("materialized", "reduced"):
        R, s = oracle.join_r_sigma(A, kA, B, kB, route=route)
        assert np.allclose(R.ravel(), fx["R"], rtol=1e-14, atol=1e-14), route
        assert np.allclose(s, fx["sigma"], rtol=1e-14), route


def test_c0_oracle_regression():
    fx = read_fixture("c0_oracle_R_sigma.txt")
    A, B = config("c0")
    assert oracle.join_rows(A.key, B.key) == int(fx["join_rows"][0])
    R, s = oracle.join_r_sigma(A.x, A.key, B.x, B.key, route="reduced")
    assert np.max(np.abs(R.ravel() - fx["R"])) < 1e-11
    assert np.max(np.abs(s - fx["sigma"])) < 1e-11
