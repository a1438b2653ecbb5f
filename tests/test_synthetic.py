"""The seeded input generators: links are SU(3) and near the unit matrix,
the sliced generator does not depend on the number of worker processes, and
the point sources are the 12 spin-colour unit vectors at one site."""
from __future__ import annotations

import numpy as np

import synthetic as syn


def _check_su3_near_unit(U, eps):
    I = np.eye(3)
    UU = U @ np.swapaxes(U.conj(), -1, -2)
    assert np.abs(UU - I).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-13
    # exp(i eps H), H ~ O(1): the distance from 1 scales with eps
    d = np.linalg.norm(U - I, axis=(-2, -1)).mean()
    assert 0.3 * eps < d < 5.0 * eps


def test_gauge_fields_are_su3_near_unit():
    for eps in (0.15, 0.3):
        _check_su3_near_unit(syn.gauge_field((4, 4, 4, 4), eps, 0), eps)
        _check_su3_near_unit(syn.gauge_field_sliced((4, 4, 2, 6), eps, 1), eps)


def test_sliced_generator_independent_of_workers():
    L = (4, 2, 2, 6)
    a = syn.gauge_field_sliced(L, 0.2, 7, workers=0)
    b = syn.gauge_field_sliced(L, 0.2, 7, workers=2)
    assert a.shape == (syn.volume(L), 4, 3, 3) and np.array_equal(a, b)
    assert not np.array_equal(a, syn.gauge_field_sliced(L, 0.2, 8))


def test_point_sources():
    L = (2, 2, 2, 2)
    b = syn.point_sources(L, site=3)
    assert b.shape == (12, 16, 4, 3)
    assert np.array_equal(b.reshape(12, -1)[:, 3 * 12:4 * 12], np.eye(12))
    assert np.count_nonzero(b) == 12
