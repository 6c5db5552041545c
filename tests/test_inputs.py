"""The seeded input generators that both sides draw from: deterministic per
seed, within their stated ranges, and with the properties the tests rely on
(unit finite-difference directions, pairwise distinct float32-exact values
for following populations through a streaming permutation)."""
import numpy as np

from paper_2112_08479_gb300 import inputs


def test_uniform_is_seeded_and_bounded():
    a = inputs.uniform((7, 50), 3, 0.25)
    assert np.array_equal(a, inputs.uniform((7, 50), 3, 0.25))
    assert not np.array_equal(a, inputs.uniform((7, 50), 4, 0.25))
    assert a.shape == (7, 50) and np.all(np.abs(a) <= 0.25)
    assert a.min() < -0.2 and a.max() > 0.2          # spans the range


def test_normal_is_seeded():
    a = inputs.normal(1000, 9, 2.0)
    assert np.array_equal(a, inputs.normal(1000, 9, 2.0))
    assert abs(a.std() - 2.0) < 0.2


def test_unit_direction_has_unit_norm():
    d = inputs.unit_direction((3, 4, 5), 11)
    assert d.shape == (3, 4, 5)
    assert abs(np.linalg.norm(d.ravel()) - 1.0) < 1e-12


def test_distinct_values_are_distinct_and_float32_exact():
    v = inputs.distinct_values((4, 6, 8), 5)
    flat = v.ravel()
    assert len(np.unique(flat)) == flat.size
    assert np.array_equal(flat.astype(np.float32).astype(np.float64), flat)
    assert np.all(np.abs(flat) < 1.0)
