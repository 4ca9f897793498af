"""The thread-per-cell root search (one lane per cell: cells of at most 24 tetrahedra, learned and
interval-cubic modes, root phase in FP32-pair arithmetic) against the oracle, and its hand-over of
cells to the FP64 lane-group path.

Bars as in the parity tests: the oracle's cut volume at the GPU isovalue matches alpha to 1e-10
on every interface cell, the interface area matches the oracle's at that isovalue to 1e-9, and the
mass transfer equals the lane-group path's to the 1e-8 parity bar."""
import numpy as np
import pytest

import oracle
from gpu_helpers import EPS, case, close, gpu_step

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14938_gb300 as vof  # noqa: E402

CASES = ["hex_sphere", "voronoi_film", "voronoi_spheres", "tet_sphere", "prism_sphere", "pipe_film"]


def _check_residual_and_area(m, a, g):
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    I = g["iface_idx"]
    assert np.array_equal(I, np.where((a > EPS) & (a < 1 - EPS))[0])
    worst = 0.0
    for c in I:
        if g["status"][c] & 1:
            continue
        geo = O.liquid_volume(c, g["phi_v"], g["iso"][c])
        worst = max(worst, abs(geo["VL"] / V[c] - a[c]))
        assert geo["area"] == pytest.approx(g["A_int"][c], rel=1e-9, abs=1e-13 * V[c] ** (2 / 3))
    assert worst <= 1e-10, worst
    cnt = g["counts"]
    assert cnt["n_not_converged"] == 0 and cnt["n_fallback"] == 0


@pytest.mark.parametrize("mode", ["learned", "cubic"])
@pytest.mark.parametrize("name", CASES)
def test_one_lane_per_cell_meets_the_bar(name, mode):
    m, a, T, Tb = case(name)
    M = vof.Mesh(m)
    if mode == "learned":
        assert vof.load_default_mlp(M)
    rm = vof.ROOT_LEARNED if mode == "learned" else vof.ROOT_CUBIC
    _, g1 = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=rm, group_size=1)
    _check_residual_and_area(m, a, g1)
    # one FP64-equivalent pass per cell on these meshes (the interval holding the refined point)
    assert g1["counts"]["evals_total"] <= 2 * len(g1["iface_idx"])
    _, g4 = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=rm, group_size=4)
    ok, err = close(g1["mdot"], g4["mdot"])
    assert ok, err
    np.testing.assert_allclose(g1["totals"], g4["totals"], rtol=1e-8)


@pytest.mark.parametrize("name", ["hex_sphere", "tet_sphere", "pipe_film"])
def test_handed_over_cells_equal_the_lane_group_path(name):
    """root_narrow = 2 makes every interval too narrow for the pairs: every cell goes to the slow
    list, and the lane-group kernel that takes it (four lanes per cell) gives exactly what it gives
    when it runs the bin itself."""
    m, a, T, Tb = case(name)
    M = vof.Mesh(m)
    _, gs = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_CUBIC, group_size=1, root_narrow=2.0)
    _, g4 = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_CUBIC, group_size=4)
    I = gs["iface_idx"]
    assert len(I) > 0
    for k in ("iso", "status", "evals", "A_int"):
        assert np.array_equal(gs[k][I], g4[k][I]), k
    assert np.array_equal(gs["mdot"], g4["mdot"])
    _check_residual_and_area(m, a, gs)


def test_root_narrow_is_validated():
    m, a, T, Tb = case("tet_sphere")
    M = vof.Mesh(m)
    for bad in (0.0, 2.0 ** -21, 2.5, float("nan")):
        with pytest.raises(vof.VofError):
            gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_CUBIC, root_narrow=bad)
