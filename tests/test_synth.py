"""Synthetic inputs: the approximated delta sources of Eq. 5.4 (input generation only)."""

import numpy as np

from paper_2003_02585_gb300 import synth


def test_delta_sources_unit_mass_bilinear_and_symmetric():
    n = (60, 60)
    h = 1.0 / 60
    f = synth.delta_sources(n, h, synth.TABLE5_POINTS)
    # four points of unit mass 1/(h1 h2) each
    assert np.isclose(f.sum() * h * h, 4.0)
    # (1/4, 1/4) lies midway between four cell-centred nodes: four equal weights per point
    assert np.count_nonzero(f) == 16
    assert np.allclose(f[f != 0], 0.25 / h ** 2)
    # the point set is symmetric under x -> 1 - x and y -> 1 - y, and so is the field
    assert np.array_equal(f, f[::-1, :]) and np.array_equal(f, f[:, ::-1])


def test_delta_source_off_node_weights():
    n = (10, 10)
    h = 0.1
    f = synth.delta_sources(n, h, [(0.32, 0.5)])
    # x: 0.32 / 0.1 - 0.5 = 2.7 -> nodes 2 (weight 0.3) and 3 (0.7); y: midway between 4 and 5
    assert np.isclose(f[4, 2], 0.3 * 0.5 / h ** 2) and np.isclose(f[5, 3], 0.7 * 0.5 / h ** 2)
    assert np.isclose(f.sum() * h * h, 1.0)
