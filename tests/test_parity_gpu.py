"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Bars: |V_L^oracle(c_GPU)/V - alpha| <= 1e-10 on every interface cell (the oracle
re-evaluates the GPU's isovalue, since several c can be correct to rounding); relative error
<= 1e-8 on gradients, heat rates and mdot (relative to max(|x|, 1e-3 max|x|): a plain relative
error wherever |x| >= 1e-3 max|x|, and a deliberate absolute term of 1e-11 max|x| below that, where
q_l + q_v cancels and a plain relative error is undefined); integer and index outputs bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import EPS, case, close, gpu_step

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = ["hex_sphere", "voronoi_film", "voronoi_spheres", "tet_sphere", "prism_sphere", "pipe_film"]


@pytest.fixture(scope="module", params=CASES)
def run(request):
    m, a, T, Tb = case(request.param)
    M, g = gpu_step(m, a, T, Tb, htc=1)
    O = oracle.Oracle(m)
    r = O.run(a, T, Tb, synth.PROPS)
    return request.param, m, a, T, Tb, g, O, r


def test_selection_and_band_exact(run):
    name, m, a, T, Tb, g, O, r = run
    I = np.where((a > EPS) & (a < 1 - EPS))[0]
    assert g["counts"]["n_iface"] == len(I)
    assert np.array_equal(g["iface_idx"], I)
    step = g["counts"]["step"]
    assert np.array_equal(g["band_stamp"] == step, r["pc"]["in_band"].astype(bool))
    assert g["counts"]["n_band"] == r["pc"]["in_band"].sum()


def test_vertex_field(run):
    name, m, a, T, Tb, g, O, r = run
    I = np.where((a > EPS) & (a < 1 - EPS))[0]
    vs = np.unique(np.concatenate([m.face_vert[m.face_vert_off[f]:m.face_vert_off[f + 1]]
                                   for c in I for f, _ in m.cell_faces(c)]))
    np.testing.assert_allclose(g["phi_v"][vs], r["phi"][vs], rtol=0, atol=1e-14)


def test_isovalue_residual_and_geometry(run):
    """a2/a3: the oracle's cut volume at the GPU isovalue matches alpha to 1e-10; the interface
    geometry matches the oracle's geometry at that isovalue."""
    name, m, a, T, Tb, g, O, r = run
    V = O.geometry()["cell_vol"]
    I = g["iface_idx"]
    assert np.array_equal(g["status"][I] & 1, r["recon"]["status"][I] & 1)
    worst = 0.0
    for c in I:
        if g["status"][c] & 1:
            continue
        geo = O.liquid_volume(c, g["phi_v"], g["iso"][c])
        worst = max(worst, abs(geo["VL"] / V[c] - a[c]))
        assert geo["area"] == pytest.approx(g["A_int"][c], rel=1e-9, abs=1e-13 * V[c] ** (2 / 3))
        vn = np.linalg.norm(geo["vec_area"])
        if vn > 1e-9 * geo["area"]:
            np.testing.assert_allclose(g["n_int"][c], -geo["vec_area"] / vn, atol=1e-8)
        if geo["area"] > 0:
            np.testing.assert_allclose(g["x_gamma"][c], geo["centroid"], atol=1e-9 * V[c] ** (1 / 3))
    assert worst <= 1e-10, worst
    assert g["counts"]["n_not_converged"] == 0


def test_crossing_faces(run):
    """a4: crossing points, distances and projected areas on crossing faces next to the band."""
    name, m, a, T, Tb, g, O, r = run
    pc = r["pc"]
    band = pc["in_band"].astype(bool)
    exp = pc["crossing"].astype(bool) & (band[m.face_owner] | band[np.maximum(m.face_neigh, 0)])
    got = g["face_stamp"] == g["counts"]["step"]
    assert np.array_equal(got, exp)
    for k in ("d_own", "d_neigh", "A_int_f", "a_own", "a_neigh"):
        ok, err = close(g[k][exp], pc[k][exp])
        assert ok, (k, err)
    ok, err = close(g["x_f"][exp], pc["x_f"][exp])
    assert ok, ("x_f", err)


def test_gradients_and_source(run):
    """a5/a6/a7: modified least squares on the band, per-side gradients, q_l, q_v, mdot, Q and
    the totals against the oracle's own full pipeline."""
    name, m, a, T, Tb, g, O, r = run
    pc = r["pc"]
    band = pc["in_band"].astype(bool)
    I = g["iface_idx"]
    ok, err = close(g["grad"][band], pc["grad"][band])
    assert ok, ("grad", err)
    for k in ("grad_l", "grad_v", "q_l", "q_v"):
        ok, err = close(g[k][I], pc[k][I])
        assert ok, (k, err)
    for k, ko in (("mdot", "mdot"), ("Q", "Q")):
        ok, err = close(g[k], pc[ko])
        assert ok, (k, err)
    np.testing.assert_allclose(g["totals"], pc["totals"], rtol=1e-8)
    assert np.array_equal(g["status"][I] & 16, pc["status"][I] & 16)


def test_downstream_given_gpu_reconstruction(run):
    """With the GPU reconstruction fed to the oracle, the downstream steps agree to 1e-10."""
    name, m, a, T, Tb, g, O, r = run
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    I = g["iface_idx"]
    for k in ("mdot", "q_l", "q_v"):
        ok, err = close(g[k][I], pc[k][I], rel=1e-10)
        assert ok, (k, err)
    np.testing.assert_allclose(g["totals"], pc["totals"], rtol=1e-10)


@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
def test_group_sizes_agree(G):
    """Every lanes-per-cell mapping of the root search meets the same bar."""
    m, a, T, Tb = case("voronoi_spheres")
    M, g = gpu_step(m, a, T, Tb, group_size=G)
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    for c in g["iface_idx"]:
        assert abs(O.liquid_volume(c, g["phi_v"], g["iso"][c])["VL"] / V[c] - a[c]) <= 1e-10


@pytest.mark.parametrize("mode", [oracle.XF_LINEAR, oracle.XF_AS_PRINTED])
def test_crossing_modes(mode):
    m, a, T, Tb = case("voronoi_film")
    M, g = gpu_step(m, a, T, Tb, xf_mode=mode)
    r = oracle.Oracle(m).run(a, T, Tb, synth.PROPS, xf_mode=mode)
    ok, err = close(g["mdot"], r["pc"]["mdot"])
    assert ok, err


def test_edge_empty_interface():
    m = synth.voronoi_bcc(5, seed=3)
    a = np.ones(m.n_cells)
    T = np.full(m.n_cells, 380.0)
    M, g = gpu_step(m, a, T, None)
    assert g["counts"]["n_iface"] == 0 and g["counts"]["n_band"] == 0
    assert np.all(g["mdot"] == 0) and np.all(g["totals"] == 0)


def test_edge_degenerate_and_uniform():
    """alpha = 0.3 everywhere: every cell is an interface cell with a constant vertex field
    (degenerate range: A_int = 0, mdot = 0); no face crosses 1/2."""
    m = synth.hex_box(6)
    a = np.full(m.n_cells, 0.3)
    T, Tb = synth.temperature(m, {}, dict(kind="linear", T0=370.0, g=[1.0, 2.0, 3.0]))
    M, g = gpu_step(m, a, T, Tb, htc=1)
    assert g["counts"]["n_iface"] == m.n_cells
    assert g["counts"]["n_degenerate"] == m.n_cells
    assert np.all(g["A_int"] == 0) and np.all(g["mdot"] == 0)
    np.testing.assert_allclose(g["grad"], np.broadcast_to([1.0, 2.0, 3.0], (m.n_cells, 3)), atol=1e-9)


def test_edge_single_cell_and_ties():
    """One interface cell whose vertex values include exact ties with the bisection midpoints."""
    m = synth.hex_box(4)
    a = np.zeros(m.n_cells)
    a[21] = 0.5
    a[m.n_cells // 2:] = np.where(a[m.n_cells // 2:] == 0, 1.0, a[m.n_cells // 2:])
    T = np.full(m.n_cells, synth.T_SAT)
    M, g = gpu_step(m, a, T, None, vertex_mode=1)
    r = oracle.Oracle(m).run(a, T, None, synth.PROPS, vertex_mode=1)
    I = g["iface_idx"]
    V = oracle.Oracle(m).geometry()["cell_vol"]
    for c in I:
        if not g["status"][c] & 1:
            assert abs(oracle.Oracle(m).liquid_volume(c, g["phi_v"], g["iso"][c])["VL"] / V[c] - a[c]) <= 1e-10
    assert np.all(g["mdot"] == 0) and np.all(r["pc"]["mdot"] == 0)


def test_repeated_steps_are_bitwise_reproducible():
    m, a, T, Tb = case("voronoi_film")
    M, g1 = gpu_step(m, a, T, Tb)
    _, g2 = gpu_step(m, a, T, Tb, dev_mesh=M)
    for k in ("iso", "A_int", "mdot", "grad", "totals"):
        assert np.array_equal(g1[k], g2[k]), k
    assert g2["counts"]["step"] == g1["counts"]["step"] + 1


def test_host_buffer_step_matches_device_step():
    import paper_2604_14938_gb300 as vof
    m, a, T, Tb = case("voronoi_film")
    M, g = gpu_step(m, a, T, Tb, htc=1)
    pin = lambda x: torch.as_tensor(np.ascontiguousarray(x)).pin_memory()
    ha, hT, hTb = pin(a), pin(T), pin(Tb)
    hm = torch.empty(m.n_cells, dtype=torch.float64).pin_memory()
    ht = torch.empty(2, dtype=torch.float64).pin_memory()
    M.step_host(ha, hT, hTb, synth.PROPS, hm, ht, vof.default_options())
    assert np.array_equal(hm.numpy(), g["mdot"])
    assert np.array_equal(ht.numpy(), g["totals"])


def test_host_buffer_step_from_pageable_memory():
    """Host buffers that are not pinned take the plain copies (the boundary gather needs a mapped
    view); the results are those of the device step."""
    import paper_2604_14938_gb300 as vof
    m, a, T, Tb = case("pipe_film")
    M, g = gpu_step(m, a, T, Tb, htc=1)
    hm, ht = torch.empty(m.n_cells, dtype=torch.float64), torch.empty(2, dtype=torch.float64)
    M.step_host(torch.as_tensor(a), torch.as_tensor(T), torch.as_tensor(np.ascontiguousarray(Tb)), synth.PROPS, hm, ht,
                vof.default_options())
    assert np.array_equal(hm.numpy(), g["mdot"])
    assert np.array_equal(ht.numpy(), g["totals"])


def test_iteration_cap_sets_status_not_a_fault():
    """A forced bisection cap leaves NOT_CONVERGED bits and counts; the step completes."""
    m, a, T, Tb = case("voronoi_spheres")
    M, g = gpu_step(m, a, T, Tb, max_bisect=3)
    I = g["iface_idx"]
    nc = g["counts"]["n_not_converged"]
    assert nc > 0
    assert nc == int(np.sum((g["status"][I] & 2) != 0))
    assert np.all(g["evals"][I] <= 3)
    assert np.all(np.isfinite(g["mdot"]))


def test_non_finite_and_out_of_range_alpha():
    """NaN and alpha outside [0, 1] never select a cell; the rest of the step is unchanged."""
    m, a, T, Tb = case("voronoi_film")
    M, g0 = gpu_step(m, a, T, Tb)
    a2 = a.copy()
    bulk = np.where((a == 0) | (a == 1))[0][:50]
    a2[bulk[:25]] = np.nan
    a2[bulk[25:]] = np.where(a[bulk[25:]] == 0, -0.5, 1.5)
    _, g1 = gpu_step(m, a2, T, Tb, dev_mesh=M)
    assert g1["counts"]["n_iface"] == g0["counts"]["n_iface"]
    assert np.array_equal(g1["iface_idx"], g0["iface_idx"])
