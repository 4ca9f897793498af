"""The stencil study's anisotropy measures on synthetic angular data (no GPU)."""
import numpy as np
import pytest

from paper_2604_14938_gb300.stencil_study import analytic_T, anisotropy


@pytest.mark.parametrize("eps,phase", [(0.0, 0.0), (0.05, 0.0), (0.12, 0.3)])
def test_fourfold_amplitude_and_bin_ratio(eps, phase):
    rng = np.random.default_rng(4)
    # uneven angular sampling (denser near the diagonals) must not bias the measure
    th = np.concatenate([rng.uniform(-np.pi, np.pi, 4000), np.pi / 4 + rng.normal(0, 0.05, 3000)])
    th = (th + np.pi) % (2 * np.pi) - np.pi
    ratio = 0.9 * (1 + eps * np.cos(4 * (th - phase)))
    mm, four = anisotropy(th, ratio, 72)
    assert four == pytest.approx(eps, abs=2e-3)
    # bin means of a smooth pattern: min / max close to (1 - eps) / (1 + eps)
    assert mm == pytest.approx((1 - eps) / (1 + eps), abs=0.01)


def test_analytic_field():
    x = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.9], [0.8, 0.5, 0.5]])
    T = analytic_T(x, 0.3, 100.0, 373.15)
    np.testing.assert_allclose(T, [373.15, 373.15 + 100 * 0.1, 373.15])
