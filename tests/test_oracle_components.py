"""Pins of the oracle's small-component filter (§Region of Interest
extraction: residual small connected components removed by area).

Against scipy's labelling with the 8-connected structuring element and a
bincount of the labels (an independent library route to the same set), and
closed forms: isolated pixels, a diagonal line (one 8-connected component
of its length), a checkerboard (one component), thresholds at exactly a
component's area."""
import numpy as np
import pytest

ndimage = pytest.importorskip("scipy.ndimage")


def _scipy_remove(m, min_area):
    lab, n = ndimage.label(m, structure=np.ones((3, 3), int))
    area = np.bincount(lab.ravel(), minlength=n + 1)
    keep = area >= min_area
    keep[0] = False
    return keep[lab].astype(np.uint8)


@pytest.mark.parametrize("seed,h,w,p,a", [(1, 40, 60, 0.3, 5), (2, 64, 64, 0.45, 12), (3, 1, 50, 0.6, 3),
                                          (4, 50, 1, 0.6, 2), (5, 128, 96, 0.55, 40)])
def test_matches_scipy_label_and_bincount(orc, seed, h, w, p, a):
    rng = np.random.default_rng(seed)
    m = (rng.random((h, w)) < p).astype(np.uint8)
    assert np.array_equal(orc.remove_small(m, a), _scipy_remove(m, a))


def test_isolated_pixels_and_thresholds(orc):
    m = np.zeros((10, 10), np.uint8)
    m[1, 1] = 1
    m[5:8, 5:8] = 1  # area 9
    assert np.array_equal(orc.remove_small(m, 1), m)
    assert np.array_equal(orc.remove_small(m, 0), m)
    r = orc.remove_small(m, 2)
    assert r[1, 1] == 0 and r[5:8, 5:8].all()
    assert orc.remove_small(m, 9)[5:8, 5:8].all()
    assert not orc.remove_small(m, 10).any()


def test_diagonal_and_checkerboard_are_single_8_connected_components(orc):
    d = np.eye(12, dtype=np.uint8)
    assert np.array_equal(orc.remove_small(d, 12), d)
    assert not orc.remove_small(d, 13).any()
    cb = (np.indices((9, 9)).sum(0) % 2 == 0).astype(np.uint8)  # 41 pixels, all diagonal neighbours
    assert np.array_equal(orc.remove_small(cb, 41), cb)
    assert not orc.remove_small(cb, 42).any()
