"""The oracle checked against what the paper and the mathematics fix (no GPU).

Each test names the pin it applies: closed forms (tetrahedron cut volume, Appendix C stencil
formulas, 1D Stefan flux), textbook constructions computed by an independent routine (half-space
clip of a convex cell via Qhull), invariants (reference-point independence, monotonicity,
continuity), and the paper's printed values (tests/golden/appendix_c_boost.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
spatial = pytest.importorskip("scipy.spatial")


def cell_vertex_ids(m, c):
    vs = set()
    for f, _ in m.cell_faces(c):
        vs.update(int(v) for v in m.face_loop(f))
    return sorted(vs)


def cell_edges(m, c):
    es = set()
    for f, _ in m.cell_faces(c):
        L = m.face_loop(f)
        for i in range(len(L)):
            a, b = int(L[i]), int(L[(i + 1) % len(L)])
            es.add((min(a, b), max(a, b)))
    return sorted(es)


def xyz(m, ids):
    return np.stack([m.vx[ids], m.vy[ids], m.vz[ids]], 1)


def halfspace_clip(m, c, n, d):
    """Volume of {x in cell: n.x <= d} and area of the section, by Qhull (independent of R2)."""
    ids = cell_vertex_ids(m, c)
    P = xyz(m, ids)
    pos = {v: i for i, v in enumerate(ids)}
    s = P @ n - d
    pts = [P[i] for i in range(len(ids)) if s[i] <= 0]
    cut = []
    for a, b in cell_edges(m, c):
        sa, sb = s[pos[a]], s[pos[b]]
        if sa * sb < 0:
            t = sa / (sa - sb)
            cut.append(P[pos[a]] + t * (P[pos[b]] - P[pos[a]]))
    vol = spatial.ConvexHull(np.array(pts + cut)).volume
    # section area: project the cut points onto the plane
    C = np.array(cut)
    u = np.cross(n, [1.0, 0, 0] if abs(n[0]) < 0.9 else [0, 1.0, 0])
    u /= np.linalg.norm(u)
    w = np.cross(n, u)
    area = spatial.ConvexHull(np.stack([C @ u, C @ w], 1)).volume
    return vol, area, spatial.ConvexHull(P).volume


MESHES = {
    "hex": lambda: synth.hex_box(4),
    "tet": lambda: synth.tet_box(3),
    "prism": lambda: synth.prism_box(3),
    "voronoi": lambda: synth.voronoi_bcc(4, seed=7),
    "pipe": lambda: synth.pipe(spacing=0.25, layers=3, length=0.75, seed=3),
}


@pytest.mark.parametrize("kind", sorted(MESHES))
def test_P1_planar_interface_exact(kind):
    """P1: a linear vertex field phi = d - n.x with alpha = exact half-space fraction reproduces
    c = 0, n_int = -n (vapour -> liquid), A_int = section area (the method reproduces planar
    interfaces exactly)."""
    m = MESHES[kind]()
    O = oracle.Oracle(m)
    rng = np.random.default_rng(11)
    P = xyz(m, np.arange(m.n_verts))
    cells = rng.choice(m.n_cells, size=min(12, m.n_cells), replace=False)
    for c in cells:
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        ids = cell_vertex_ids(m, c)
        proj = P[ids] @ n
        d = proj.min() + (proj.max() - proj.min()) * rng.uniform(0.15, 0.85)
        phi = d - P @ n
        vol, area, V = halfspace_clip(m, c, n, d)
        alpha = np.zeros(m.n_cells)
        alpha[c] = vol / V
        r = O.reconstruct(alpha, phi, cells=[c])
        h = (V) ** (1 / 3)
        assert r["status"][c] == 0
        assert abs(r["iso"][c]) <= 1e-9 * h
        assert r["A_int"][c] == pytest.approx(area, rel=1e-9)
        np.testing.assert_allclose(r["n_int"][c], -n, atol=1e-9)
        # the centroid of the section lies on the plane
        assert abs(r["x_gamma"][c] @ n - d) <= 1e-9 * h


def test_P2_tet_closed_form():
    """P2: for a linear field on a tetrahedron the liquid fraction {phi >= c} is the third divided
    difference of (t - c)_+^3 over the vertex values (Curry-Schoenberg B-spline), i.e.
    sum_i (phi_i - c)_+^3 / prod_{j != i} (phi_i - phi_j); one vertex above c gives V l1 l2 l3."""
    m = synth.tet_box(1)
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    rng = np.random.default_rng(3)
    for trial in range(20):
        phi = rng.uniform(-1, 1, m.n_verts)
        for c in range(m.n_cells):
            ids = cell_vertex_ids(m, c)
            f = phi[ids]
            for cc in np.linspace(f.min(), f.max(), 23)[1:-1]:
                expect = sum(max(f[i] - cc, 0.0) ** 3 / np.prod([f[i] - f[j] for j in range(4) if j != i])
                             for i in range(4))
                got = O.liquid_volume(c, phi, cc)["VL"] / V[c]
                assert got == pytest.approx(expect, abs=1e-12)
    # the product form for a single vertex above c
    phi = np.array([0.0] * m.n_verts)
    c = 0
    ids = cell_vertex_ids(m, c)
    phi[ids] = [1.0, 0.2, 0.1, -0.3]
    cc = 0.6
    lam = [(1.0 - cc) / (1.0 - x) for x in (0.2, 0.1, -0.3)]
    assert O.liquid_volume(c, phi, cc)["VL"] / V[c] == pytest.approx(np.prod(lam), rel=1e-13)


def _idw_cells(m, reg, n=15, seed=0):
    a = synth.alpha(m, reg, mode="subtet", level=2)
    O = oracle.Oracle(m)
    phi = O.vertex_field(a)
    I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0]
    rng = np.random.default_rng(seed)
    return O, a, phi, rng.choice(I, size=min(n, len(I)), replace=False)


def test_P3_invariants_voronoi():
    """P3: V_L independent of the reference point; V_L(phi_min) = V, V_L(phi_max) = 0;
    non-increasing in c; continuous where c passes a vertex value (the iso-polygon fan centre is
    the perimeter-weighted centroid, so coinciding cut points carry no weight)."""
    m = synth.voronoi_bcc(6, seed=2)
    reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.31)])
    O, a, phi, cells = _idw_cells(m, reg)
    V = O.geometry()["cell_vol"]
    rng = np.random.default_rng(5)
    for c in cells:
        f = np.unique(phi[cell_vertex_ids(m, c)])
        lo, hi = f.min(), f.max()
        assert O.liquid_volume(c, phi, lo)["VL"] == pytest.approx(V[c], rel=1e-13)
        assert abs(O.liquid_volume(c, phi, hi)["VL"]) <= 1e-13 * V[c]
        cc = rng.uniform(lo, hi)
        x0 = O.geometry()["cell_cen"][c] + rng.normal(size=3) * V[c] ** (1 / 3)
        assert O.liquid_volume(c, phi, cc, x0=x0)["VL"] == pytest.approx(O.liquid_volume(c, phi, cc)["VL"],
                                                                        abs=1e-13 * V[c])
        scan = np.linspace(lo, hi, 400)
        vl = np.array([O.liquid_volume(c, phi, s)["VL"] for s in scan])
        assert np.all(np.diff(vl) <= 1e-13 * V[c])
        # continuity at every vertex value: the gap across it vanishes linearly with the offset
        d = 1e-8 * (hi - lo)
        for v in f[1:-1]:
            gap = [O.liquid_volume(c, phi, v - e)["VL"] - O.liquid_volume(c, phi, v + e)["VL"] for e in (d, d / 100)]
            assert gap[1] >= -1e-9 * V[c]  # the cone centre drifts: monotone up to ~1e-9 V
            assert abs(gap[1]) <= abs(gap[0]) / 20 + 1e-13 * V[c]


def _tet_root(f, alpha):
    """Closed-form isovalue of a linear field on a tetrahedron: the root of
    sum_i (f_i - c)_+^3 / prod_{j != i}(f_i - f_j) = alpha on the bracketing vertex interval."""
    fs = np.sort(f)[::-1]
    den = [np.prod([f[i] - f[j] for j in range(4) if j != i]) for i in range(4)]

    def F(c):
        return sum(max(f[i] - c, 0.0) ** 3 / den[i] for i in range(4))

    for k in range(3):
        hi, lo = fs[k], fs[k + 1]
        if F(lo) >= alpha >= F(hi):
            act = [i for i in range(4) if f[i] >= hi]
            poly = np.zeros(4)
            for i in act:  # (f_i - c)^3 / den_i as a polynomial in c
                poly += np.array([-1.0, 3 * f[i], -3 * f[i] ** 2, f[i] ** 3]) / den[i]
            poly[3] -= alpha
            roots = [r.real for r in np.roots(poly) if abs(r.imag) < 1e-7 and lo - 1e-12 <= r.real <= hi + 1e-12]
            return min(roots, key=lambda r: abs(F(r) - alpha))
    raise AssertionError("no bracket")


def test_P4_bisection_matches_closed_form_root():
    """P4: on tetrahedra with a linear field the bisection root equals the closed-form root of the
    cut-volume cubic, and |V_L(c)/V - alpha| <= 1e-12 (the root's volume tolerance)."""
    m = synth.tet_box(2)
    O = oracle.Oracle(m)
    rng = np.random.default_rng(8)
    phi = rng.uniform(-1, 1, m.n_verts)
    a = rng.uniform(0.01, 0.99, m.n_cells)
    r = O.reconstruct(a, phi)
    V = O.geometry()["cell_vol"]
    for c in range(m.n_cells):
        f = phi[cell_vertex_ids(m, c)]
        assert abs(O.liquid_volume(c, phi, r["iso"][c])["VL"] / V[c] - a[c]) <= 1e-12
        assert abs(r["iso"][c] - _tet_root(f, a[c])) <= 1e-10 * (f.max() - f.min())


def test_P3_exact_at_vertex_values():
    """P3: at c equal to a vertex value the cut volume of a tetrahedron equals the closed form
    sum_i (f_i - c)_+^3 / prod_j (f_i - f_j) (no jump there), and on a Voronoi cell it equals the
    mean of its values just below and just above."""
    m = synth.tet_box(2)
    O = oracle.Oracle(m)
    phi = np.random.default_rng(21).uniform(-1, 1, m.n_verts)
    V = O.geometry()["cell_vol"]
    for c in range(m.n_cells):
        f = phi[cell_vertex_ids(m, c)]
        den = [np.prod([f[i] - f[j] for j in range(4) if j != i]) for i in range(4)]
        for x in f:
            exact = sum(max(f[i] - x, 0.0) ** 3 / den[i] for i in range(4))
            assert O.liquid_volume(c, phi, x)["VL"] / V[c] == pytest.approx(exact, abs=1e-13)
    m = synth.voronoi_bcc(5, seed=11)
    reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.3)])
    O, a, phi, cells = _idw_cells(m, reg, n=10, seed=2)
    V = O.geometry()["cell_vol"]
    for c in cells:
        f = np.unique(phi[cell_vertex_ids(m, c)])
        e = 1e-9 * (f[-1] - f[0])
        for x in f[1:-1]:
            mid = 0.5 * (O.liquid_volume(c, phi, x - e)["VL"] + O.liquid_volume(c, phi, x + e)["VL"])
            assert abs(O.liquid_volume(c, phi, x)["VL"] - mid) <= 1e-8 * V[c]


def test_P11_interval_cubic_matches_closed_form_root():
    """P11 (interval cubic): on tetrahedra with a linear field the interval-cubic root
    equals the closed-form root of the tetrahedron's cut-volume cubic, with |V_L(c)/V - alpha| <=
    1e-12, after at most one bisection step over the four vertex values and two interior samples
    (plus the final check)."""
    m = synth.tet_box(2)
    O = oracle.Oracle(m)
    rng = np.random.default_rng(18)
    phi = rng.uniform(-1, 1, m.n_verts)
    a = rng.uniform(0.01, 0.99, m.n_cells)
    r = O.reconstruct(a, phi, method="cubic")
    V = O.geometry()["cell_vol"]
    for c in range(m.n_cells):
        f = phi[cell_vertex_ids(m, c)]
        assert r["status"][c] == 0
        assert abs(O.liquid_volume(c, phi, r["iso"][c])["VL"] / V[c] - a[c]) <= 1e-12
        assert abs(r["iso"][c] - _tet_root(f, a[c])) <= 1e-10 * (f.max() - f.min())
        assert r["evals"][c] <= 2 + 2 + 1


@pytest.mark.parametrize("kind", ["voronoi", "hex", "tet"])
def test_P11_interval_cubic_residual_and_evaluations(kind):
    """P11: on every interface cell of a curved interface the interval-cubic root meets
    |V_L(c)/V - alpha| <= 1e-12, agrees with the bisection root (the root is unique where the
    interface has area), and takes ceil(log2(distinct vertex values - 1)) + 3 evaluations at most."""
    m = MESHES[kind]()
    reg = dict(type="spheres", spheres=[(0.47, 0.52, 0.5, 0.33)])
    O, a, phi, cells = _idw_cells(m, reg, n=60, seed=3)
    V = O.geometry()["cell_vol"]
    rc = O.reconstruct(a, phi, cells=cells, method="cubic")
    rb = O.reconstruct(a, phi, cells=cells)
    for c in cells:
        u = np.unique(phi[cell_vertex_ids(m, c)])
        assert rc["status"][c] == 0
        assert abs(O.liquid_volume(c, phi, rc["iso"][c])["VL"] / V[c] - a[c]) <= 1e-12
        assert rc["evals"][c] <= int(np.ceil(np.log2(max(len(u) - 1, 1)))) + 3
        if rc["A_int"][c] > 1e-6 * V[c] ** (2 / 3):
            assert abs(rc["iso"][c] - rb["iso"][c]) <= 1e-8 * (u[-1] - u[0])
        assert rc["evals"][c] < rb["evals"][c]


def test_P4_residual_voronoi():
    """P4: every converged Voronoi cell meets |V_L(c)/V - alpha| <= 1e-12 in a few tens of
    evaluations."""
    m = synth.voronoi_bcc(6, seed=4)
    reg = dict(type="film", z0=0.43, a=0.05)
    O, a, phi, cells = _idw_cells(m, reg, n=40)
    V = O.geometry()["cell_vol"]
    r = O.reconstruct(a, phi, cells=cells)
    for c in cells:
        assert r["status"][c] == 0
        assert abs(O.liquid_volume(c, phi, r["iso"][c])["VL"] / V[c] - a[c]) <= 1e-12
        assert r["evals"][c] <= 60


@pytest.mark.parametrize("kind", sorted(MESHES))
def test_P5_linear_field_exact_unmodified(kind):
    """P5: a linear temperature gives the exact gradient with the unmodified stencil on every cell
    type (no face crosses alpha = 1/2; boundary faces enter as virtual neighbours)."""
    m = MESHES[kind]()
    O = oracle.Oracle(m)
    g = np.array([3.0, -2.0, 0.5])
    T, Tb = synth.temperature(m, {}, dict(kind="linear", T0=370.0, g=g))
    a = np.full(m.n_cells, 0.3)
    phi = O.vertex_field(a)
    rec = O.reconstruct(a, phi)
    pc = O.phase_change(a, rec, T, Tb, synth.PROPS)
    assert pc["in_band"].all()
    np.testing.assert_allclose(pc["grad"], np.broadcast_to(g, pc["grad"].shape), rtol=0, atol=1e-9)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_P5_linear_field_exact_modified(axis):
    """P5: with the interface-modified stencil the gradient stays exact when T_sat = T(x_f): a
    planar interface normal to an axis on a hex mesh, the same linear T on both sides."""
    n = 8
    m = synth.hex_box(n)
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    xg = 0.4 + 0.37 / n
    lo = np.floor(cen[:, axis] * n) / n
    a = np.clip((lo + 1 / n - xg) * n, 0, 1)   # liquid on the high side
    gvec = np.zeros(3)
    gvec[axis] = 7.0
    prof = dict(kind="linear", T0=synth.T_SAT - 7.0 * xg, g=gvec)
    T, Tb = synth.temperature(m, {}, prof)
    r = O.run(a, T, Tb, synth.PROPS)
    pc = r["pc"]
    band = pc["in_band"].astype(bool)
    assert band.sum() > 0
    np.testing.assert_allclose(pc["grad"][band], np.broadcast_to(gvec, (band.sum(), 3)), atol=1e-9)
    # R4 and R5 in the same setting: both interface cells of a crossing face carry the same plane,
    # so the crossing point lies on x_axis = x_g whichever is chosen; and the other side's gradient,
    # an upwind average of equal neighbour gradients, is that gradient again: q_l and q_v follow in
    # closed form (n = +e_axis, the liquid side high; A_int = the cross-section 1/n^2)
    cross = np.where(pc["crossing"])[0]
    assert len(cross) == n * n
    # the plane's position carries the root's volume tolerance 1e-12 (in units of the cell width)
    np.testing.assert_allclose(pc["x_f"][cross][:, axis], xg, rtol=0, atol=2e-12 / n)
    I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0]
    for k in ("grad_l", "grad_v"):
        np.testing.assert_allclose(pc[k][I], np.broadcast_to(gvec, (len(I), 3)), atol=1e-9)
    np.testing.assert_allclose(pc["q_l"][I], synth.PROPS["k_l"] * 7.0 / n ** 2, rtol=1e-10)
    np.testing.assert_allclose(pc["q_v"][I], -synth.PROPS["k_v"] * 7.0 / n ** 2, rtol=1e-10)
    assert not np.any(pc["status"][I] & oracle.ST_NO_SIDE)


def _column(d_over_h, T_P, T_far, Ts=373.15, h=1.0, standard=False):
    """1D hex column of five cells: vapour | vapour | P | liquid | liquid; the interface between
    the second cell and P sits d from x_P (alpha-interpolated x_f, Eq. front_interpolation read
    as linear interpolation)."""
    m = synth.hex_box(5, 1, 1, lo=(0, 0, 0), hi=(5 * h, h, h))
    O = oracle.Oracle(m)
    t = 1 - d_over_h  # x_f = x_left + t h, so |x_f - x_P| = d
    if 0.5 / t < 1:
        a_left, aP = 0.0, 0.5 / t
    else:  # t = (a_left - 1/2)/(a_left - a_P) with a_P = 0.9
        aP = 0.9
        a_left = (0.5 - t * aP) / (1 - t)
    a = np.array([0.0, a_left, aP, 1.0, 1.0])
    if standard:
        a = np.array([0.2, 0.2, 0.3, 0.3, 0.3])
    T = np.array([Ts, Ts, T_P, T_far, T_far])
    Tb = np.full(m.n_faces, T_P)  # transverse virtual neighbours at T_P leave g_x untouched
    phi = O.vertex_field(a)
    rec = O.reconstruct(a, phi)
    pc = O.phase_change(a, rec, T, Tb, dict(synth.PROPS, T_sat=Ts), xf_mode=oracle.XF_LINEAR)
    return pc["grad"][2, 0]


@pytest.mark.parametrize("dh", [0.1, 0.3, 0.5, 0.7])
def test_P6_appendix_c_modified_stencil(dh):
    """P6: Appendix C, Eq. (g_fm): g_fm = ((T_P - T_sat) d + (T_far - T_P) h)/(d^2 + h^2), and
    Eq. (g_std) for the standard stencil."""
    h, Ts, TP, Tf = 1.0, 373.15, 374.0, 376.5
    d = dh * h
    g = _column(dh, TP, Tf, Ts, h)
    assert g == pytest.approx(((TP - Ts) * d + (Tf - TP) * h) / (d * d + h * h), rel=1e-13)
    gs = _column(dh, TP, Tf, Ts, h, standard=True)
    # standard stencil with the inner neighbour in the vapour at T_sat
    assert gs == pytest.approx((Tf - Ts) / (2 * h), rel=1e-13)


def test_P6_appendix_c_heat_sink_limit_golden():
    """P6: heat-sink limit 2h^2/(d^2+h^2), against the values the paper prints (golden file)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "appendix_c_boost.txt")) if l.strip() and l[0] != "#"]
    Ts, Tf = 373.15, 378.15
    for dh, ratio, tol in ((float(a), float(b), float(c)) for a, b, c in rows):
        dh_eff = max(dh, 1e-7)
        g_fm = _column(dh_eff, Ts, Tf, Ts)
        g_std = (Tf - Ts) / 2.0
        assert g_fm / g_std == pytest.approx(2 / (1 + dh_eff ** 2), rel=1e-12)
        assert abs(g_fm / g_std - ratio) <= tol


@pytest.mark.parametrize("lam", [0.2, 0.5, 0.8])
def test_P6_appendix_c_truncation(lam):
    """P6: Eq. (lsq_truncation): for neighbours at -h and +lam h and a quadratic field the 1D LSQ
    gradient errs by -h (1 - lam^3)/(2 (1 + lam^2)) phi''."""
    h = 1.0
    Ts = 373.15
    xP = 2.5
    xf = xP + lam * h
    c2 = -3.0  # phi''
    c1 = 4.0

    def T(x):  # quadratic through (x_f, T_sat)
        return Ts + c1 * (x - xf) + 0.5 * c2 * (x - xf) ** 2

    m = synth.hex_box(5, 1, 1, lo=(0, 0, 0), hi=(5.0, 1.0, 1.0))
    O = oracle.Oracle(m)
    # owner = P (cell 2), neighbour = cell 3; t = (a_o - 1/2)/(a_o - a_n) = lam
    aP = 0.5 + 0.4 * lam
    an = aP - (aP - 0.5) / lam  # = 0.1 + 0.4 lam, vapour
    a = np.array([aP, aP, aP, an, 0.0])
    Tc = np.array([T(0.5), T(1.5), T(xP), Ts, Ts])
    Tb = np.full(m.n_faces, T(xP))
    phi = O.vertex_field(a)
    rec = O.reconstruct(a, phi)
    pc = O.phase_change(a, rec, Tc, Tb, dict(synth.PROPS, T_sat=Ts), xf_mode=oracle.XF_LINEAR)
    g_true = c1 + c2 * (xP - xf)
    err = -h * (1 - lam ** 3) / (2 * (1 + lam ** 2)) * c2
    assert pc["grad"][2, 0] - g_true == pytest.approx(err, rel=1e-11)


def _stefan(xg_frac, mode=oracle.XF_RECON):
    L, n, W = 2e-3, 20, 3
    h = L / n
    m = synth.hex_box(n, W, W, lo=(0, 0, 0), hi=(L, W * h, W * h))
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    xg = 5 * h + xg_frac * h
    lo = np.round(cen[:, 0] / h - 0.5) * h
    a = np.clip((lo + h - xg) / h, 0, 1)
    dT = 10.0
    T, Tb = synth.temperature(m, {}, dict(kind="stefan", x_g=xg, dT=dT))
    r = O.run(a, T, Tb, synth.PROPS, xf_mode=mode)
    I = (a > 1e-12) & (a < 1 - 1e-12)
    return r, I, O.geometry()["cell_vol"], xg, dT


@pytest.mark.parametrize("frac", [0.23, 0.5 + 1e-3, 0.81])
def test_P7_stefan_flux(frac):
    """P7: planar vapour layer with T linear from T_sat + dT at the wall to T_sat at x_g, liquid at
    T_sat: mdot V / A_int = k_v dT / (h_lv x_g), q_l = 0 exactly (Sec. 3.1 Stefan problem; the
    instantaneous flux of its linear vapour profile)."""
    r, I, V, xg, dT = _stefan(frac)
    pc, rec = r["pc"], r["recon"]
    assert I.sum() == 9
    flux = pc["mdot"][I] * V[I] / rec["A_int"][I]
    expect = synth.PROPS["k_v"] * dT / (synth.PROPS["h_lv"] * xg)
    np.testing.assert_allclose(flux, expect, rtol=1e-12)
    assert np.all(pc["q_l"][I] == 0.0)
    np.testing.assert_allclose(rec["n_int"][I], np.broadcast_to([1.0, 0, 0], (9, 3)), atol=1e-12)


@pytest.mark.parametrize("frac", [0.23, 0.81])
def test_P12_interface_htc_stefan(frac):
    """P12 (Eq. interface_htc): on the planar Stefan layer the one crossing face per row
    of cells is the face next to the interface cell; its interface area projected onto the face is
    the face area h^2, and each side's coefficient is k_phi h^2 / d with d the distance from that
    cell's centre to the plane x = x_g; every other face has none."""
    r, I, V, xg, dT = _stefan(frac)
    pc = r["pc"]
    m = synth.hex_box(20, 3, 3, lo=(0, 0, 0), hi=(2e-3, 3e-4, 3e-4))
    cen = oracle.Oracle(m).geometry()["cell_cen"]
    h = 1e-4
    cross = np.where(pc["crossing"])[0]
    assert len(cross) == 9
    for f in cross:
        o, n = m.face_owner[f], m.face_neigh[f]
        for cell, got in ((o, pc["a_own"][f]), (n, pc["a_neigh"][f])):
            liquid = cen[cell, 0] > xg
            k = synth.PROPS["k_l"] if liquid else synth.PROPS["k_v"]
            assert got == pytest.approx(k * h * h / abs(cen[cell, 0] - xg), rel=1e-12)
    others = np.setdiff1d(np.arange(m.n_faces), cross)
    assert not np.any(pc["a_own"][others]) and not np.any(pc["a_neigh"][others])


@pytest.mark.parametrize("frac", [0.23, 0.81])
def test_P12_energy_matrix_terms_stefan(frac):
    """P12 (Eq. interface_htc in the energy equation): on the planar Stefan layer each
    cell next to the interface has exactly one detached face, so its diagonal term is k_phi h^2 / d
    (d its centre's distance to the plane x = x_g) and its right-hand side that times T_sat; every
    other cell has none."""
    r, I, V, xg, dT = _stefan(frac)
    pc = r["pc"]
    m = synth.hex_box(20, 3, 3, lo=(0, 0, 0), hi=(2e-3, 3e-4, 3e-4))
    cen = oracle.Oracle(m).geometry()["cell_cen"]
    h = 1e-4
    touched = set()
    for f in np.where(pc["crossing"])[0]:
        touched |= {int(m.face_owner[f]), int(m.face_neigh[f])}
    assert len(touched) == 18
    for c in range(m.n_cells):
        if c in touched:
            k = synth.PROPS["k_l"] if cen[c, 0] > xg else synth.PROPS["k_v"]
            assert pc["htc_diag"][c] == pytest.approx(k * h * h / abs(cen[c, 0] - xg), rel=1e-12)
            assert pc["htc_rhs"][c] == pytest.approx(pc["htc_diag"][c] * synth.T_SAT, rel=1e-15)
        else:
            assert pc["htc_diag"][c] == 0.0 and pc["htc_rhs"][c] == 0.0


def test_P12_energy_matrix_terms_two_faces():
    """P12 with a cell detached on two faces, worked by hand. Cells [0, 1], [1, 3], [3, 4] along x
    (unit cross-section, centroids x = 1/2, 2, 7/2), alpha = 0.3 | 0.9 | 0.1, all interface cells,
    linear crossing points (Eq. front_interpolation read as linear interpolation): the face x = 1
    has t = 1/3, so x_f = 1 and d = 1/2 | 1; the face x = 3 has t = 1/2, so x_f = 11/4 and
    d = 3/4 | 3/4. Each face's projected area comes from its owner's plane: 1 on the first
    (normal e_x), 0.8 |n . e_x| = 0.8/sqrt2 on the second (normal (1, 1, 0)/sqrt2). So the
    diagonal terms are 2 k_v, k_l + k_l 0.8/(0.75 sqrt2) and k_v 0.8/(0.75 sqrt2); the right-hand
    sides are those times T_sat."""
    m = stretched_hex([0.0, 1.0, 3.0, 4.0], [0.0, 1.0], [0.0, 1.0])
    cells = [box_cell(m, (0, 0, 0), (1, 1, 1)), box_cell(m, (1, 0, 0), (3, 1, 1)), box_cell(m, (3, 0, 0), (4, 1, 1))]
    a = np.zeros(m.n_cells)
    a[cells] = [0.3, 0.9, 0.1]
    assert all(int(m.face_owner[_shared_face(m, cells[i], cells[i + 1])]) == cells[i] for i in range(2))
    rec = _two_cell_recon(m, cells, [(1.0, (1, 0, 0), (0.9, 0.5, 0.5)), (0.8, (1, 1, 0), (2.9, 0.5, 0.5)),
                                     (0.5, (-1, 0, 0), (3.1, 0.5, 0.5))])
    T = np.full(m.n_cells, synth.T_SAT)
    pc = oracle.Oracle(m).phase_change(a, rec, T, None, synth.PROPS, xf_mode=oracle.XF_LINEAR)
    kl, kv = synth.PROPS["k_l"], synth.PROPS["k_v"]
    g = 0.8 / (0.75 * math.sqrt(2.0))
    for c, want in zip(cells, (2 * kv, kl + kl * g, kv * g)):
        assert pc["htc_diag"][c] == pytest.approx(want, rel=1e-14)
        assert pc["htc_rhs"][c] == pytest.approx(want * synth.T_SAT, rel=1e-14)


def test_P12_fixed_isovalue_planar():
    """P12: with the vertex field linear in x the alpha_iso = 0.5 surface is the plane
    where that field is 0.5; its area in each cut cell is the cell's cross-section (1/3)^2, its
    normal -x (vapour at high x), and the cells it misses have no interface."""
    m = synth.hex_box(6, 3, 3)
    O = oracle.Oracle(m)
    h = 1 / 6  # cell size along x; 1/3 across
    phi = 0.9 - 1.3 * m.vx  # linear, decreasing in x: the liquid (phi >= c) lies at low x
    a = np.full(m.n_cells, 0.5)
    rec = O.reconstruct(a, phi, method="fixed", alpha_iso=0.5)
    x_iso = (0.9 - 0.5) / 1.3
    cen = O.geometry()["cell_cen"]
    for c in range(m.n_cells):
        cut = abs(cen[c, 0] - x_iso) < h / 2
        assert rec["status"][c] == 0 and rec["iso"][c] == 0.5
        if cut:
            assert rec["A_int"][c] == pytest.approx(1 / 9, rel=1e-12)
            np.testing.assert_allclose(rec["n_int"][c], [-1.0, 0, 0], atol=1e-12)
            assert rec["x_gamma"][c][0] == pytest.approx(x_iso, rel=1e-12)
        else:
            assert rec["A_int"][c] == 0.0


def test_P7_stefan_linear_xf_is_not_exact():
    """P7: with the alpha-interpolated crossing point the flux is not exact."""
    r, I, V, xg, dT = _stefan(0.23, mode=oracle.XF_LINEAR)
    flux = r["pc"]["mdot"][I] * V[I] / r["recon"]["A_int"][I]
    expect = synth.PROPS["k_v"] * dT / (synth.PROPS["h_lv"] * xg)
    assert np.all(np.abs(flux / expect - 1) > 1e-4)


def test_P8_sphere_area_convergence():
    """P8: sum of A_int over the interface cells tends to 4 pi R^2 under refinement h = 1/16,
    1/32, 1/64. With a signed-distance vertex field the error falls at an average order >= 1.5
    (alpha from 64^3 midpoint samples per cell; the sampling error of alpha, not the
    reconstruction, limits the observed order); with the inverse-distance field the error is
    recorded, not gated."""
    R, c0 = 0.25, np.array([0.5, 0.5, 0.5])
    reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, R)])
    err_sd, err_idw = [], []
    for n in (16, 32, 64):
        m = synth.hex_box(n)
        O = oracle.Oracle(m)
        a = synth.alpha(m, reg, mode="hexgrid", level=6)
        P = xyz(m, np.arange(m.n_verts))
        phi_sd = np.linalg.norm(P - c0, axis=1) - R
        rec = O.reconstruct(a, phi_sd)
        err_sd.append(abs(rec["A_int"].sum() - 4 * np.pi * R * R))
        rec2 = O.reconstruct(a, O.vertex_field(a))
        err_idw.append(abs(rec2["A_int"].sum() - 4 * np.pi * R * R))
    assert err_sd[0] > err_sd[1] > err_sd[2], err_sd
    assert math.log2(err_sd[0] / err_sd[2]) / 2 >= 1.5, err_sd
    # inverse-distance field of a sharp alpha stays curved at the cell scale: recorded, bounded
    # (measured 2.6e-2, 2.1e-2, 2.2e-2 of 0.785 at n = 16, 32, 64)
    assert max(err_idw) < 0.05 * 4 * np.pi * R * R, err_idw


def test_P9_special_cases(hex_sphere):
    """P9: vapour at T_sat gives q_v = 0 exactly; T = T_sat everywhere gives mdot = 0 exactly."""
    m, reg, a, T, Tb = hex_sphere
    O = oracle.Oracle(m)
    r = O.run(a, T, Tb, synth.PROPS)
    I = (a > 1e-12) & (a < 1 - 1e-12)
    assert np.all(r["pc"]["q_v"][I] == 0.0)
    assert np.all(r["pc"]["mdot"][I] >= 0.0)
    Tc = np.full(m.n_cells, synth.T_SAT)
    r2 = O.phase_change(a, r["recon"], Tc, np.full(m.n_faces, synth.T_SAT), synth.PROPS)
    assert np.all(r2["mdot"] == 0.0) and r2["totals"][0] == 0.0


def test_R1_uniform_hex_is_the_plain_mean():
    """R1, a special case with a textbook answer: on a uniform hex mesh an interior vertex is
    equidistant from its eight cell centroids, so the inverse-distance field is their plain mean;
    a boundary vertex of a face's centre line is equidistant from its two or four cells too."""
    m = synth.hex_box(4)
    O = oracle.Oracle(m)
    a = np.random.default_rng(5).uniform(size=m.n_cells)
    phi = O.vertex_field(a)
    cells_of = [[] for _ in range(m.n_verts)]
    for c in range(m.n_cells):
        for v in cell_vertex_ids(m, c):
            cells_of[v].append(c)
    for v, cs in enumerate(cells_of):
        assert phi[v] == pytest.approx(np.mean(a[cs]), rel=1e-14), v
    np.testing.assert_allclose(phi, O.vertex_field(a, mode=1), rtol=1e-14)


def test_R1_vertex_field_invariants():
    """R1 (parity unpinned; invariants only): constant alpha gives a constant field; each vertex
    value lies between the min and max alpha of its cells."""
    m = synth.voronoi_bcc(5, seed=9)
    O = oracle.Oracle(m)
    assert np.allclose(O.vertex_field(np.full(m.n_cells, 0.37)), 0.37, atol=1e-15)
    a = np.random.default_rng(1).uniform(size=m.n_cells)
    phi = O.vertex_field(a)
    lo = np.full(m.n_verts, np.inf)
    hi = np.full(m.n_verts, -np.inf)
    for c in range(m.n_cells):
        ids = cell_vertex_ids(m, c)
        lo[ids] = np.minimum(lo[ids], a[c])
        hi[ids] = np.maximum(hi[ids], a[c])
    assert np.all(phi >= lo - 1e-15) and np.all(phi <= hi + 1e-15)


def test_R8_pairwise_tree():
    """R8: the total is the fixed pairwise tree over the zero-padded power of two."""
    a = np.array([1e16, 1.0, -1e16, 1.0, 3.0])
    t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + 0.0) + (0.0 + 0.0))
    assert oracle.pairwise_sum(a) == t
    b = np.random.default_rng(0).normal(size=1000)
    assert oracle.pairwise_sum(b) == pytest.approx(math.fsum(b), abs=1e-12)
    assert oracle.pairwise_sum(np.zeros(0)) == 0.0


def test_geometry_closed_cells():
    """Oracle geometry: cell volumes sum to the box volume and centroids of a hex grid are exact."""
    for kind, mk in MESHES.items():
        m = mk()
        g = oracle.Oracle(m).geometry()
        if kind != "pipe":
            assert g["cell_vol"].sum() == pytest.approx(1.0, rel=1e-12)
        assert np.all(g["cell_vol"] > 0)
    m = synth.hex_box(4)
    g = oracle.Oracle(m).geometry()
    i = np.arange(4)
    exp = np.stack(np.meshgrid((i + 0.5) / 4, (i + 0.5) / 4, (i + 0.5) / 4, indexing="ij")[::-1], -1).reshape(-1, 3)
    np.testing.assert_allclose(g["cell_cen"], exp, atol=1e-15)


def stretched_hex(xs, ys, zs):
    """A hex mesh whose grid lines sit at the given node coordinates (a uniform hex box with each
    coordinate mapped piecewise linearly onto the nodes): cells of different sizes, exact box
    centroids."""
    m = synth.hex_box(len(xs) - 1, len(ys) - 1, len(zs) - 1)
    for attr, nodes in (("vx", xs), ("vy", ys), ("vz", zs)):
        u = np.linspace(0.0, 1.0, len(nodes))
        setattr(m, attr, np.interp(getattr(m, attr), u, np.asarray(nodes, np.float64)))
    return m


def box_cell(m, lo, hi):
    """The cell of a stretched hex mesh whose vertices span the box [lo, hi] (found by its vertices)."""
    for c in range(m.n_cells):
        P = xyz(m, cell_vertex_ids(m, c))
        if np.allclose(P.min(0), lo) and np.allclose(P.max(0), hi):
            return c
    raise KeyError((lo, hi))


def vertex_at(m, x):
    d = (m.vx - x[0]) ** 2 + (m.vy - x[1]) ** 2 + (m.vz - x[2]) ** 2
    v = int(np.argmin(d))
    assert d[v] == 0.0
    return v


def test_R1_inverse_distance_unequal_cells():
    """R1 on cells of four different sizes, worked by hand. Grid lines x = 0, 1, 3 and y = 0, 1/2, 2,
    one layer 0 <= z <= 1. The vertex (1, 1/2, 0) touches the four cells, whose box centroids are
    (1/2, 1/4, 1/2), (2, 1/4, 1/2), (1/2, 5/4, 1/2) and (2, 5/4, 1/2), at distances 3/4, sqrt(21)/4,
    sqrt(17)/4 and sqrt(29)/4; so phi_v = (a0/3 + a1/sqrt21 + a2/sqrt17 + a3/sqrt29) /
    (1/3 + 1/sqrt21 + 1/sqrt17 + 1/sqrt29). The boundary vertex (1, 0, 0) touches the first two cells
    at distances 3/4 and sqrt(21)/4: phi_v = (a0/3 + a1/sqrt21)/(1/3 + 1/sqrt21). A corner vertex
    takes its one cell's alpha. Weights 1/|x|^2 or the plain mean give other values."""
    m = stretched_hex([0.0, 1.0, 3.0], [0.0, 0.5, 2.0], [0.0, 1.0])
    O = oracle.Oracle(m)
    cells = [box_cell(m, (0, 0, 0), (1, 0.5, 1)), box_cell(m, (1, 0, 0), (3, 0.5, 1)),
             box_cell(m, (0, 0.5, 0), (1, 2, 1)), box_cell(m, (1, 0.5, 0), (3, 2, 1))]
    a = np.zeros(m.n_cells)
    a[cells] = [0.2, 0.9, 0.55, 0.05]
    phi = O.vertex_field(a)
    w = np.array([1 / 3, 1 / math.sqrt(21), 1 / math.sqrt(17), 1 / math.sqrt(29)])
    assert phi[vertex_at(m, (1, 0.5, 0))] == pytest.approx((w @ a[cells]) / w.sum(), rel=1e-14)
    assert phi[vertex_at(m, (1, 0, 0))] == pytest.approx((0.2 / 3 + 0.9 / math.sqrt(21)) / w[:2].sum(), rel=1e-14)
    assert phi[vertex_at(m, (3, 2, 1))] == 0.05
    # the same vertex with the plain average (vertex_mode 1)
    assert O.vertex_field(a, mode=1)[vertex_at(m, (1, 0.5, 0))] == pytest.approx(np.mean(a[cells]), rel=1e-14)


def _two_cell_recon(m, cells, planes):
    """A reconstruction given by hand: planes[k] = (A_int, n_int, x_gamma) of cells[k]."""
    nc = m.n_cells
    rec = dict(status=np.zeros(nc, np.int32), A_int=np.zeros(nc), n_int=np.zeros((nc, 3)), x_gamma=np.zeros((nc, 3)))
    for c, (A, n, xg) in zip(cells, planes):
        rec["A_int"][c] = A
        rec["n_int"][c] = np.asarray(n, np.float64) / np.linalg.norm(n)
        rec["x_gamma"][c] = xg
    return rec


def _shared_face(m, p, q):
    for f in range(m.n_faces):
        if {int(m.face_owner[f]), int(m.face_neigh[f])} == {p, q}:
            return f
    raise KeyError((p, q))


@pytest.mark.parametrize("case", ["owner_nearer", "neighbour_nearer", "owner_outside", "both_outside"])
def test_R4_two_interface_cells_nearest_plane(case):
    """R4 when both cells of a crossing face are interface cells with different planes, worked by
    hand. Cells [0, 1] and [1, 3] along x (unit cross-section), centroids x = 1/2 and x = 2, so the
    centroid segment is x = 1/2 + 3/2 t; the face centroid is at x = 1. alpha = 0.7 | 0.3 (liquid on
    the left: n_int = -e_x). A plane x = p crosses at t = (p - 1/2)/(3/2), at distance |p - 1| from
    the face centroid; the plane nearer the face centroid gives x_f, one whose t leaves [0, 1] does
    not count, and with neither the linear interpolation t = (0.7 - 0.5)/(0.7 - 0.3) = 1/2 applies.
    The projected area A_int,f = |A_int n_int . n_f| follows the plane that was used. Tilted planes
    (normal (-1, -1, 0)) cross the centre line y = 1/2 at the same x."""
    m = stretched_hex([0.0, 1.0, 3.0], [0.0, 1.0], [0.0, 1.0])
    p, q = box_cell(m, (0, 0, 0), (1, 1, 1)), box_cell(m, (1, 0, 0), (3, 1, 1))
    a = np.zeros(m.n_cells)
    a[p], a[q] = 0.7, 0.3
    xp, xq = {"owner_nearer": (0.8, 1.5), "neighbour_nearer": (0.6, 1.1), "owner_outside": (0.2, 1.9),
              "both_outside": (0.1, 2.9)}[case]
    # cell p: axis-normal plane, area 1; cell q: tilted plane through (xq, 1/2, 1/2), area 0.5
    rec = _two_cell_recon(m, [p, q], [(1.0, (-1, 0, 0), (xp, 0.5, 0.5)), (0.5, (-1, -1, 0), (xq, 0.5, 0.5))])
    T = np.full(m.n_cells, synth.T_SAT)
    pc = oracle.Oracle(m).phase_change(a, rec, T, None, synth.PROPS)
    f = _shared_face(m, p, q)
    assert pc["crossing"][f] == 1
    tp, tq = (xp - 0.5) / 1.5, (xq - 0.5) / 1.5
    cand = [(abs(x - 1.0), x, A) for x, t, A in ((xp, tp, 1.0), (xq, tq, 0.5 / math.sqrt(2))) if 0 <= t <= 1]
    o = int(m.face_owner[f])
    if cand:
        _, x_exp, Af_exp = min(cand)
    else:  # linear interpolation; the projected area then comes from the owner's plane
        x_exp, Af_exp = 0.5 + 1.5 * 0.5, 1.0 if o == p else 0.5 / math.sqrt(2)
    want = {"owner_nearer": 0.8, "neighbour_nearer": 1.1, "owner_outside": 1.9, "both_outside": 1.25}[case]
    assert x_exp == want
    np.testing.assert_allclose(pc["x_f"][f], [x_exp, 0.5, 0.5], rtol=0, atol=1e-15)
    d_o, d_n = (x_exp - 0.5, 2.0 - x_exp) if o == p else (2.0 - x_exp, x_exp - 0.5)
    assert pc["d_own"][f] == pytest.approx(d_o, rel=1e-14)
    assert pc["d_neigh"][f] == pytest.approx(d_n, rel=1e-14)
    assert pc["A_int_f"][f] == pytest.approx(Af_exp, rel=1e-14)
