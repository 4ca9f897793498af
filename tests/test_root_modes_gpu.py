"""The interval-cubic root mode (the scope's next step for the root search) on the GPU: the cut
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
