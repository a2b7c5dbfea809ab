"""The jet observables of Sec. 3 recover the parameters of analytic fields:
Gaussian radial profiles exp(-k (r/(z - z0))^2) and a linear inverse
centre-line decay."""
import numpy as np
import pytest

from paper_2403_15773_gb300 import jetstats


def self_similar_field(nx=96, ny=96, nz=200, k=75.0, z0=-10.0, slope=1 / 6.5 / 16, a=1.0):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy = nx / 2, ny / 2
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    uc = 1.0 / (a + slope * z)
    return uc * np.exp(-k * r2 / (z - z0) ** 2), uc


@pytest.mark.parametrize("k", [75.0, 80.0, 200.0])
def test_gaussian_exponent_recovered(k):
    f, _ = self_similar_field(k=k)
    z = 150
    r, prof = jetstats.radial_profile(f, z, 48.0, 48.0, dr=1.0)
    kf = jetstats.gaussian_exponent(r, prof, z, -10.0)
    assert abs(kf / k - 1.0) < 0.03


def test_inverse_centerline_slope_recovered():
    slope = 1.0 / (6.5 * 16)
    f, uc = self_similar_field(slope=slope)
    c = jetstats.centerline(f, 48.0, 48.0)
    assert np.allclose(c, uc[:, 48, 48])
    s = jetstats.inverse_slope(np.arange(f.shape[0]), c, 40, 190)
    assert abs(s / slope - 1.0) < 1e-9


def test_centerline_bilinear_between_nodes():
    f = np.zeros((3, 4, 4))
    f[:, 1, 1], f[:, 1, 2], f[:, 2, 1], f[:, 2, 2] = 1.0, 2.0, 3.0, 4.0
    assert np.allclose(jetstats.centerline(f, 1.5, 1.5), 2.5)
