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


def test_section51_mesh_source_and_medium():
    """Section 5.1 recipe: mesh geometry of the printed tables, the smooth source of Eq. (5.1)
    (unit mass: 16 k^2 / pi^3 * pi / (4 k / pi)^2 = 1), its four mirror images, and the smooth
    two-layer wave speed (c = 1 below 0.65, 0.8 above 0.66, monotone ramp between)."""
    from paper_2003_02585_gb300 import synth
    assert synth.conv_mesh(270) == (240, 15, 1.0 / 270)
    assert synth.conv_mesh(1080) == (960, 60, 1.0 / 1080)
    n_int, pml, h = synth.conv_mesh(540)
    n = (n_int, n_int)
    f1 = synth.smooth_source(n, h)
    f4 = synth.smooth_source(n, h, symmetric=True)
    assert abs(f1.sum() * h * h - 1.0) < 1e-6
    assert abs(f4.sum() * h * h - 4.0) < 1e-6
    # mirror symmetry of the four-source field about the centre of B_L (= centre of the interior)
    assert np.allclose(f4, f4[::-1, :]) and np.allclose(f4, f4[:, ::-1])
    c = synth.medium_smooth_two_layer(n, h)
    x2 = (np.arange(n_int) + 0.5) * h + synth.CONV_OFFSET
    assert np.all(c[x2 < 0.65] == 1.0) and np.allclose(c[x2 > 0.66], 0.8)
    ramp = c[(x2 >= 0.65) & (x2 <= 0.66), 0]
    assert ramp.size > 0 and np.all(np.diff(ramp) < 0)
    assert np.all(c == c[:, :1])   # layered along x2 only


def test_gaussian_patch_equals_the_full_field():
    """The serving client evaluates sources on their compact support only
    (synth.gaussian_source_patch); placed into a zero field it must equal gaussian_source."""
    from paper_2003_02585_gb300 import synth
    rng = np.random.default_rng(0)
    for n in ((256, 256), (100, 60), (24, 40, 16)):
        h = 1.0 / n[0]
        for _ in range(4):
            c = rng.uniform(0.0, 1.0, len(n)) * np.array(n) * h
            full = synth.gaussian_source(n, h, c, 2 * h)
            sl, vals = synth.gaussian_source_patch(n, h, c, 2 * h)
            placed = np.zeros_like(full)
            placed[sl] = vals
            assert np.array_equal(placed, full)
