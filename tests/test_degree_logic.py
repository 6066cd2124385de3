"""Host logic of the learned degree/bounds proposer (no GPU): input features and the decoding
of network outputs into a degree and bounds, with their safety clamps."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def degree():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_07820_gb300 import degree
    return degree


def test_features(degree):
    ev = np.linspace(-1.0, 0.5, 32)
    r1 = degree.Record(ev, np.full(32, 1e-3), 0.5, 100.0, 40, False)
    f = degree.features([r1], True)
    assert f.shape == (degree.N_IN,) and f[-1] == 1.0
    assert np.isclose(f[0], -0.75) and np.isclose(f[1], -0.75)            # log10(1e-3) / 4
    assert np.isclose(f[2], 1.5 / 101.0) and np.isclose(f[3], 1.5 / 101.0)
    assert np.isclose(f[4], 1.0) and f[5] == 0.0
    assert np.array_equal(f[0:6], f[6:12]) and np.array_equal(f[0:6], f[12:18])   # oldest repeated
    r2 = degree.Record(ev + 0.01, np.r_[np.full(24, 1e-6), np.full(8, 1.0)], 0.51, 110.0, 20, False)
    f = degree.features([r1, r2], False)
    assert f[-1] == 0.0
    assert np.isclose(f[0], -1.5)                  # largest residual of the lowest 3/4 only
    assert np.isclose(f[4], 0.5) and np.isclose(f[6 + 5], math.log(100.0 / 110.0))


def test_decode_and_clamps(degree):
    ev = np.linspace(-1.0, 0.5, 32)
    r = degree.Record(ev, np.full(32, 1e-3), 0.5, 100.0, 40, False)
    m, a, b, est = degree.decode(np.array([0.0, 0.0, 0.0]), r, 100.0)
    assert m == 16 and a == ev[-1] and np.isclose(est, 100.0) and np.isclose(b, 101.0)
    m, a, b, est = degree.decode(np.array([5.0, -3.0, -50.0]), r, 100.0)
    assert m == degree.DEG_MAX and a == ev[-1] and np.isclose(est, 100.0 * math.exp(-0.02))
    m, a, b, est = degree.decode(np.array([-5.0, 3.0, 50.0]), r, 100.0)
    assert m == degree.DEG_MIN and np.isclose(a, ev[-1] + 0.02 * 1.5) and np.isclose(est, 100.0 * math.exp(0.02))
    # the bound used never falls below a + spread
    m, a, b, est = degree.decode(np.array([0.0, 0.0, 0.0]), r, 0.1)
    assert b >= a + 1.5
