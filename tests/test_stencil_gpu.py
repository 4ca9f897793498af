"""GPU parity of the least-squares variants of the stencil-anisotropy study (options.lsq_variant):
the CUDA study kernel through the C ABI against the oracle's variants, on the same reconstruction
and crossing points.

Bars: gradients relative 1e-8 (Euclidean norm, floored at 1e-3 of the largest), widened to 100
times the oracle's own movement under one-ulp centroid rounding where the weighted or shortened
stencils are ill-conditioned; cond(G_P) within 1e-10 + 1e-12 cond relative (both sides lose about
an ulp times cond in the smallest eigenvalue); the singular flags exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import case, gpu_step, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = ["hex_sphere", "voronoi_spheres", "tet_sphere", "pipe_film"]
VARIANTS = [8, 9, 10, 12, 14, 15]


def spread(O, a, pc, T, Tb, variant, draws=2, seed=0):
    """The oracle's own gradient change under one-ulp centroid rounding, row by row."""
    g = O.geometry()
    cen0 = g["cell_cen"].copy()
    base = O.lsq_study(a, pc, T, Tb, synth.PROPS, variant)
    rng = np.random.default_rng(seed)
    out = np.zeros(len(cen0))
    try:
        for _ in range(draws):
            s = rng.integers(-1, 2, cen0.shape)
            g["cell_cen"][:] = np.where(s > 0, np.nextafter(cen0, np.inf),
                                        np.where(s < 0, np.nextafter(cen0, -np.inf), cen0))
            out = np.maximum(out, rel_err(O.lsq_study(a, pc, T, Tb, synth.PROPS, variant)["grad"], base["grad"]))
    finally:
        g["cell_cen"][:] = cen0
    return base, out


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_lsq_variant_parity(name, variant):
    m, a, T, Tb = case(name)
    M, g = gpu_step(m, a, T, Tb, lsq_variant=variant)
    O = oracle.Oracle(m)
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    band = pc["in_band"].astype(bool)
    assert np.array_equal(g["band_stamp"] == g["counts"]["step"], band)
    r, sp = spread(O, a, pc, T, Tb, variant)
    e = rel_err(g["grad"][band], r["grad"][band])
    allow = np.maximum(1e-8, 100 * sp[band])
    assert np.all(e <= allow), float((e / allow).max())
    assert np.array_equal(g["status"][band] & 8, r["status"][band] & 8)
    ok = band & np.isfinite(r["cond"])
    ce = np.abs(g["lsq_cond"][ok] - r["cond"][ok]) / r["cond"][ok]
    assert np.all(ce <= 1e-10 + 1e-12 * r["cond"][ok]), float(ce.max())


def test_default_variant_is_the_path():
    """Variant 8 (cond only) gives the path's own gradients to rounding; downstream outputs follow."""
    m, a, T, Tb = case("voronoi_spheres")
    M, g0 = gpu_step(m, a, T, Tb)
    _, g8 = gpu_step(m, a, T, Tb, dev_mesh=M, lsq_variant=8)
    band = g0["band_stamp"] == g0["counts"]["step"]
    assert np.all(rel_err(g8["grad"][band], g0["grad"][band]) <= 1e-12)
    np.testing.assert_allclose(g8["totals"], g0["totals"], rtol=1e-11)
