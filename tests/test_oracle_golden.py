"""The stored plain-pipe wake (written by tests/golden/make_golden.py from the
oracle) is reproduced by the oracle as it stands, and obeys the loss-factor
identity of the energy law (19) at the full plain-pipe size."""
import os

import numpy as np
import pytest

from golden.make_golden import plain_pipe_wake

HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden(name="plain_pipe_24x24x96_wake.txt"):
    path = os.path.join(HERE, "golden", name)
    meta = {}
    vals = []
    with open(path) as f:
        for line in f:
            if line.startswith("# s0_m"):
                t = line[1:].split()
                meta = {t[i]: float(t[i + 1]) for i in range(0, len(t), 2)}
            elif not line.startswith("#"):
                vals.append(float(line))
    return np.array(vals), meta


def test_oracle_reproduces_stored_plain_pipe_wake():
    ref, meta = load_golden()
    wk, s0, ds, energy = plain_pipe_wake()
    assert s0 == pytest.approx(meta["s0_m"]) and ds == pytest.approx(meta["ds_m"])
    peak = np.max(np.abs(ref))
    assert np.max(np.abs(wk - ref)) <= 1e-12 * peak
    assert energy == pytest.approx(meta["field_energy_J"], rel=1e-12)
