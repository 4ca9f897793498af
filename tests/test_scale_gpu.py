"""Mesh scale and placement on the GPU: the interface geometry runs in (hi, lo) FP32 pairs with
positions relative to each cell's apex, so a mesh of small cells far from the origin and a mesh of
large cells must meet the same parity bars as the unit mesh (the oracle works in FP64 throughout)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import case, close, gpu_step

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _transformed(m, scale, offset):
    return dataclasses.replace(m, vx=m.vx * scale + offset[0], vy=m.vy * scale + offset[1], vz=m.vz * scale + offset[2])


@pytest.mark.parametrize("scale,offset", [(1e-3, (1.0, -2.0, 0.5)), (1e3, (0.0, 0.0, 0.0)), (1.0, (1e2, 1e2, 1e2))])
def test_geometry_and_source_at_any_scale(scale, offset):
    m0, a, T, Tb = case("voronoi_spheres")
    m = _transformed(m0, scale, offset)
    M, g = gpu_step(m, a, T, Tb)
    O = oracle.Oracle(m)
    r = O.run(a, T, Tb, synth.PROPS)
    V = O.geometry()["cell_vol"]
    I = g["iface_idx"]
    assert np.array_equal(I, np.where((a > 1e-12) & (a < 1 - 1e-12))[0])
    worst = 0.0
    for c in I:
        geo = O.liquid_volume(c, g["phi_v"], g["iso"][c])
        worst = max(worst, abs(geo["VL"] / V[c] - a[c]))
        h = V[c] ** (1 / 3)
        assert geo["area"] == pytest.approx(g["A_int"][c], rel=1e-9, abs=1e-13 * h * h)
        vn = np.linalg.norm(geo["vec_area"])
        if vn > 1e-9 * geo["area"]:
            np.testing.assert_allclose(g["n_int"][c], -geo["vec_area"] / vn, atol=1e-8)
        if geo["area"] > 0:
            np.testing.assert_allclose(g["x_gamma"][c], geo["centroid"], rtol=0, atol=1e-9 * h)
    assert worst <= 1e-10, worst
    for k in ("mdot", "Q"):
        ok, err = close(g[k], r["pc"][k])
        assert ok, (k, err)
