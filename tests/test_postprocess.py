"""Host-side post-processing: the Froude number of Eq. 59 (slope of the front
position over 2.5 <= t <= 10)."""
import numpy as np
import pytest

from paper_2112_08479_gb300.run import froude


def test_froude_exact_on_linear_front():
    t = np.linspace(0, 20, 201)
    x = 0.42 * t + 1.3
    assert froude(t, x) == pytest.approx(0.42, rel=1e-12)


def test_froude_uses_only_the_window():
    t = np.linspace(0, 20, 201)
    x = np.where(t < 2.5, 5 * t, 0.4 * t) + np.where(t > 10, 100 * (t - 10), 0)
    assert froude(t, x) == pytest.approx(0.4, rel=1e-12)
    assert froude(t, x, 0.0, 1.0) == pytest.approx(5.0, rel=1e-12)


def test_froude_none_without_samples():
    assert froude([0.0, 1.0], [0.0, 1.0]) is None
