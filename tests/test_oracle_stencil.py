"""The oracle's least-squares variants for the stencil-anisotropy study (standard stencil,
inverse-distance weights, vertex neighbours; cond(G_P)) against closed forms, exactness and a
library routine (no GPU).

Pins:
- S1 the Jacobi eigenvalues of a symmetric 3x3 matrix equal numpy's eigvalsh.
- S2 a linear temperature gives the exact gradient with every standard-stencil variant (weighted
  or not, face or vertex neighbours) on every cell type: least squares reproduce linear fields.
- S3 with a planar interface on which T = T_sat, the modified face stencil stays exact, weighted or
  not.
- S4 cond(G_P) in closed form on a uniform hex mesh: 1 away from the interface for the face and
  vertex stencils; 2 / (1 + t^2) next to a plane normal to an axis that shortens one face vector
  to t h; and 1 there again with the weights 1/|r|^2, which turn every entry into the outer product
  of its unit direction.
- S5 variant 0 is the path's own least squares (R7).
- S6 T = x y^2 at an interior cell of a uniform hex mesh: the face stencil (weighted or not) gives
  d/dx = y^2 exactly; the 26-cell vertex stencil gives y^2 + 2h^2/3, and with the weights 1/|r|^2
  y^2 + 7h^2/13 (sums over the 3 x 3 x 3 block written out).
- S7 a corner cell with two crossing faces shortened to t = 1/2 and 2/3 (linear interpolation of
  alpha): cond = 2 / (1 + 1/4); the standard stencils stay exact when T_sat is off the field.
"""
import numpy as np
import pytest

import oracle
import synth

from test_oracle_pins import MESHES

VARIANTS_STD = [1, 3, 5, 7]


def test_S1_eigenvalues_match_library():
    rng = np.random.default_rng(2)
    for _ in range(500):
        B = rng.normal(size=(3, 3))
        A = B @ B.T * rng.uniform(1e-4, 1e4)
        np.testing.assert_allclose(oracle.sym3_eigenvalues(A), np.linalg.eigvalsh(A), rtol=1e-12,
                                   atol=1e-13 * np.abs(A).max())


@pytest.mark.parametrize("kind", sorted(MESHES))
def test_S2_linear_field_exact_standard_variants(kind):
    m = MESHES[kind]()
    O = oracle.Oracle(m)
    g = np.array([3.0, -2.0, 0.5])
    T, Tb = synth.temperature(m, {}, dict(kind="linear", T0=370.0, g=g))
    a = np.full(m.n_cells, 0.3)
    rec = O.reconstruct(a, O.vertex_field(a))
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    for v in VARIANTS_STD:
        r = O.lsq_study(a, pc, T, Tb, synth.PROPS, v)
        np.testing.assert_allclose(r["grad"], np.broadcast_to(g, r["grad"].shape), rtol=0, atol=1e-9)


def plane_case(n=8, axis=0):
    """A hex mesh with a planar interface normal to an axis, liquid on the high side, and the same
    linear T on both sides with T = T_sat on the plane."""
    m = synth.hex_box(n)
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    xg = 0.4 + 0.37 / n
    lo = np.floor(cen[:, axis] * n) / n
    a = np.clip((lo + 1 / n - xg) * n, 0, 1)
    gvec = np.zeros(3)
    gvec[axis] = 7.0
    T, Tb = synth.temperature(m, {}, dict(kind="linear", T0=synth.T_SAT - 7.0 * xg, g=gvec))
    pc = O.run(a, T, Tb, synth.PROPS)["pc"]
    return m, O, cen, a, T, Tb, pc, gvec, xg


@pytest.mark.parametrize("variant", [0, 2])
def test_S3_modified_face_stencil_exact_on_plane(variant):
    m, O, cen, a, T, Tb, pc, gvec, xg = plane_case()
    r = O.lsq_study(a, pc, T, Tb, synth.PROPS, variant)
    band = pc["in_band"].astype(bool)
    np.testing.assert_allclose(r["grad"][band], np.broadcast_to(gvec, (band.sum(), 3)), atol=1e-9)


@pytest.mark.parametrize("variant", [0, 2, 4, 6])
def test_S3_modified_stencils_exact_on_tilted_plane(variant):
    """alpha linear in the signed distance to a tilted plane (within four cells of it), so that the
    linear interpolation of alpha along any centroid connection lands on the plane; T linear with
    T = T_sat there: every modified stencil, face or vertex, weighted or not, is exact."""
    n = 8
    h = 1.0 / n
    m = synth.hex_box(n)
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    nrm = np.array([0.6, -0.3, 0.74])
    nrm /= np.linalg.norm(nrm)
    d = (cen - 0.5) @ nrm - 0.013
    a = np.clip(0.5 + d / (8 * h), 0.0, 1.0)
    gvec = 9.0 * nrm
    prof = dict(kind="linear", T0=synth.T_SAT - gvec @ (0.5 + 0.013 * nrm), g=gvec)
    T, Tb = synth.temperature(m, {}, prof)
    pc = O.run(a, T, Tb, synth.PROPS, xf_mode=oracle.XF_LINEAR)["pc"]
    r = O.lsq_study(a, pc, T, Tb, synth.PROPS, variant)
    band = pc["in_band"].astype(bool)
    assert pc["crossing"].sum() > 0
    np.testing.assert_allclose(r["grad"][band], np.broadcast_to(gvec, (band.sum(), 3)), atol=1e-9)


def test_S4_condition_numbers_closed_form():
    n = 8
    m, O, cen, a, T, Tb, pc, gvec, xg = plane_case(n)
    h = 1.0 / n
    interior = np.all((cen > h) & (cen < 1 - h), axis=1)
    # the modified face stencil: a cell whose +x or -x face crosses the plane
    band = pc["in_band"].astype(bool)
    r0 = O.lsq_study(a, pc, T, Tb, synth.PROPS, 0)
    r2 = O.lsq_study(a, pc, T, Tb, synth.PROPS, 2)
    near = band & interior & (np.abs(cen[:, 0] - xg) < h)
    far = band & interior & (np.abs(cen[:, 0] - xg) >= h)
    assert near.sum() > 0 and far.sum() > 0
    t = np.abs(cen[near, 0] - xg) / h
    np.testing.assert_allclose(r0["cond"][near], 2 / (1 + t ** 2), rtol=1e-10)
    np.testing.assert_allclose(r2["cond"][near], 1.0, rtol=1e-10)
    for v in (0, 1, 2, 3):
        np.testing.assert_allclose(O.lsq_study(a, pc, T, Tb, synth.PROPS, v)["cond"][far], 1.0, rtol=1e-10)
    # the vertex stencil of an interior cell with no crossing (every cell an interface cell of one
    # phase): 26 neighbours, symmetric
    a1 = np.full(m.n_cells, 0.3)
    pc1 = O.phase_change(a1, O.reconstruct(a1, O.vertex_field(a1)), T, Tb, synth.PROPS)
    assert pc1["in_band"].all()
    for v in (4, 5, 6, 7):
        np.testing.assert_allclose(O.lsq_study(a1, pc1, T, Tb, synth.PROPS, v)["cond"][interior], 1.0, rtol=1e-10)


def test_S5_variant_zero_is_the_path_least_squares():
    from gpu_helpers import case
    m, a, T, Tb = case("voronoi_spheres")
    O = oracle.Oracle(m)
    pc = O.run(a, T, Tb, synth.PROPS)["pc"]
    r = O.lsq_study(a, pc, T, Tb, synth.PROPS, 0)
    band = pc["in_band"].astype(bool)
    scale = np.abs(pc["grad"][band]).max()
    np.testing.assert_allclose(r["grad"][band], pc["grad"][band], rtol=1e-10, atol=1e-10 * scale)
    assert np.array_equal(r["status"][band] & 8, pc["status"][band] & 8)


@pytest.mark.parametrize("variant,extra", [(0, 0.0), (2, 0.0), (4, 2 / 3), (6, 7 / 13)])
def test_S6_vertex_stencil_closed_form(variant, extra):
    n = 6
    h = 1.0 / n
    m = synth.hex_box(n)
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    T = cen[:, 0] * cen[:, 1] ** 2 * 40.0 + 300.0
    a = np.full(m.n_cells, 0.3)
    pc = O.phase_change(a, O.reconstruct(a, O.vertex_field(a)), T, None, synth.PROPS)
    r = O.lsq_study(a, pc, T, None, synth.PROPS, variant)
    interior = np.all((cen > h) & (cen < 1 - h), axis=1)
    y = cen[interior, 1]
    np.testing.assert_allclose(r["grad"][interior, 0], 40.0 * (y ** 2 + extra * h * h), rtol=1e-11)


def test_S7_corner_cell_and_standard_stencil():
    n = 6
    h = 1.0 / n
    m = synth.hex_box(n)
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    i, j = np.floor(cen[:, 0] * n).astype(int), np.floor(cen[:, 1] * n).astype(int)
    a = np.where((i >= 3) & (j >= 3), 0.9, np.where(i >= 3, 0.3, np.where(j >= 3, 0.1, 0.2)))
    g = np.array([5.0, -3.0, 2.0])
    T, Tb = synth.temperature(m, {}, dict(kind="linear", T0=360.0, g=g))
    props = dict(synth.PROPS, T_sat=synth.T_SAT + 1.0)  # off the field: only the standard stencil is exact
    rec = O.reconstruct(a, O.vertex_field(a))
    pc = O.phase_change(a, rec, T, Tb, props, xf_mode=oracle.XF_LINEAR)
    corner = np.where((i == 3) & (j == 3) & (np.abs(cen[:, 2] - 0.5) < h))[0]
    assert len(corner) == 2
    r0 = O.lsq_study(a, pc, T, Tb, props, 0)
    np.testing.assert_allclose(r0["cond"][corner], 2 / (1 + 0.25), rtol=1e-10)
    np.testing.assert_allclose(O.lsq_study(a, pc, T, Tb, props, 2)["cond"][corner], 1.0, rtol=1e-10)
    band = pc["in_band"].astype(bool)
    for v in VARIANTS_STD:
        rs = O.lsq_study(a, pc, T, Tb, props, v)
        np.testing.assert_allclose(rs["grad"][band], np.broadcast_to(g, (band.sum(), 3)), atol=1e-9)
    assert np.abs(r0["grad"][corner] - g).max() > 1e-3
