"""The interval-cubic root mode (the exact cubic of the root's vertex interval) on the GPU: the cut
volume at its isovalue matches alpha (checked by the oracle), the isovalue agrees with the oracle's
own interval-cubic root where the interface has area, the downstream steps from it agree with the
oracle, and it takes one or two FP64 passes per cell."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import EPS, close, case, gpu_step

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14938_gb300 as vof  # noqa: E402

CASES = ["hex_sphere", "voronoi_film", "voronoi_spheres", "tet_sphere", "prism_sphere", "pipe_film"]


@pytest.mark.parametrize("name", CASES)
def test_interval_cubic_mode(name):
    m, a, T, Tb = case(name)
    M, g = gpu_step(m, a, T, Tb, root_mode=vof.ROOT_CUBIC)
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    I = g["iface_idx"]
    assert np.array_equal(I, np.where((a > EPS) & (a < 1 - EPS))[0])
    rc = O.reconstruct(a, g["phi_v"], cells=I, method="cubic")
    worst = 0.0
    for c in I:
        if g["status"][c] & 1:
            continue
        geo = O.liquid_volume(c, g["phi_v"], g["iso"][c])
        worst = max(worst, abs(geo["VL"] / V[c] - a[c]))
        u = np.unique(g["phi_v"][[int(v) for f, _ in m.cell_faces(c) for v in m.face_loop(f)]])
        if geo["area"] > 1e-6 * V[c] ** (2 / 3):
            assert abs(g["iso"][c] - rc["iso"][c]) <= 1e-8 * (u[-1] - u[0]), c
        assert geo["area"] == pytest.approx(g["A_int"][c], rel=1e-9, abs=1e-13 * V[c] ** (2 / 3))
    assert worst <= 1e-10, worst
    cnt = g["counts"]
    assert cnt["n_not_converged"] == 0
    assert cnt["evals_total"] <= 2 * len(I), cnt["evals_total"] / len(I)
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    for k in ("mdot", "q_l", "q_v"):
        ok, err = close(g[k][I], pc[k][I], rel=1e-10)
        assert ok, (k, err)


def test_interval_cubic_needs_no_mlp_and_matches_bisection():
    """No MLP is attached: the mode refines from 1 - alpha on the FP32 pipe. Its mass transfer
    equals the bisection path's to the parity bar."""
    m, a, T, Tb = case("voronoi_spheres")
    M = vof.Mesh(m)
    _, gc = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_CUBIC)
    _, gb = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_BISECT)
    ok, err = close(gc["mdot"], gb["mdot"])
    assert ok, err
    assert gc["counts"]["evals_total"] * 10 < gb["counts"]["evals_total"]


def test_interval_cubic_takes_the_mlp_guess():
    """With an MLP attached the interval is picked from the learned guess: fewer FP32 evaluations,
    the same single FP64 pass, the same bars."""
    m, a, T, Tb = case("voronoi_film")
    M = vof.Mesh(m)
    _, g0 = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_CUBIC)
    assert vof.load_default_mlp(M)
    _, g1 = gpu_step(m, a, T, Tb, dev_mesh=M, root_mode=vof.ROOT_CUBIC)
    assert g1["counts"]["evals32_total"] < g0["counts"]["evals32_total"]
    assert g1["counts"]["evals_total"] <= 2 * len(g1["iface_idx"])
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    for c in g1["iface_idx"]:
        assert abs(O.liquid_volume(c, g1["phi_v"], g1["iso"][c])["VL"] / V[c] - a[c]) <= 1e-10
    ok, err = close(g1["mdot"], g0["mdot"])
    assert ok, err


@pytest.mark.parametrize("name", ["hex_sphere", "voronoi_film", "tet_sphere", "pipe_film"])
def test_fixed_isovalue_mode(name):
    """The paper's own reconstruction (iso-surface at alpha_iso = 0.5):
    the geometry at 0.5 and the downstream steps match the oracle's, and the interface
    heat-transfer coefficients a_f = k_phi A_int,f / d_f of both sides of every crossing face next
    to the band match too."""
    m, a, T, Tb = case(name)
    M, g = gpu_step(m, a, T, Tb, root_mode=vof.ROOT_FIXED, htc=1)
    O = oracle.Oracle(m)
    I = g["iface_idx"]
    live = I[(g["status"][I] & 1) == 0]
    assert np.all(g["iso"][live] == 0.5)
    assert g["counts"]["evals_total"] == 0
    rf = O.reconstruct(a, g["phi_v"], cells=I, method="fixed")
    V = O.geometry()["cell_vol"]
    for c in live:
        assert rf["A_int"][c] == pytest.approx(g["A_int"][c], rel=1e-9, abs=1e-13 * V[c] ** (2 / 3))
        if rf["A_int"][c] > 1e-9 * V[c] ** (2 / 3):
            np.testing.assert_allclose(g["n_int"][c], rf["n_int"][c], atol=1e-8)
            np.testing.assert_allclose(g["x_gamma"][c], rf["x_gamma"][c], atol=1e-9 * V[c] ** (1 / 3))
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    for k in ("mdot", "q_l", "q_v"):
        ok, err = close(g[k][I], pc[k][I], rel=1e-10)
        assert ok, (k, err)
    band = pc["in_band"].astype(bool)
    exp = pc["crossing"].astype(bool) & (band[m.face_owner] | band[np.maximum(m.face_neigh, 0)])
    assert np.array_equal(g["face_stamp"] == g["counts"]["step"], exp)
    for k in ("a_own", "a_neigh"):
        ok, err = close(g[k][exp], pc[k][exp], rel=1e-10)
        assert ok, (k, err)
    # each band cell's energy-matrix terms: its own side's a_f and a_f T_sat summed over its
    # detached faces
    for k in ("htc_diag", "htc_rhs"):
        ok, err = close(g[k][band], pc[k][band], rel=1e-10)
        assert ok, (k, err)


@pytest.mark.parametrize("name", ["voronoi_film", "prism_sphere"])
def test_energy_matrix_terms_volume_matched(name):
    """Eq. interface_htc's energy-matrix terms (options.htc = 1) on the volume-matched
    reconstruction: per band cell, the diagonal sum of a_f and the right-hand side sum of
    a_f T_sat over its detached faces match the oracle's, computed from the GPU's reconstruction."""
    m, a, T, Tb = case(name)
    M, g = gpu_step(m, a, T, Tb, root_mode=vof.ROOT_BISECT, htc=1)
    O = oracle.Oracle(m)
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    band = pc["in_band"].astype(bool)
    assert np.array_equal(band, g["band_stamp"] == g["counts"]["step"])
    assert np.count_nonzero(pc["htc_diag"][band]) > 0
    assert not np.any(pc["htc_diag"][~band])
    for k in ("htc_diag", "htc_rhs"):
        ok, err = close(g[k][band], pc[k][band], rel=1e-10)
        assert ok, (k, err)
