"""The oracle's pseudo-time extrapolation (Eq. extrapolation, the full solve) against closed forms
and an independent steady-state solve (no GPU).

Pins:
- E1 closed form: when every inflow neighbour of every unknown is a cell of the side (a planar
  interface along a hex-mesh axis), each unknown relaxes geometrically,
  x_k = x* + (1 - c)^k (x_0 - x*), with c = dtau W / V and x* the inflow neighbour's gradient, and a
  solve stops at the first k whose largest change c (1 - c)^(k-1) |x_0 - x*| is below tol; dtau on a
  uniform hex mesh is h/2 (centroid to boundary-face centroid), so c = 1/2.
- E2 steady state: run to convergence, the iterate solves the steady upwind equations
  sum_f w_f (x_Q - x_P) = 0 at every unknown with inflow, solved here directly (dense linear solve
  per component) on a tilted planar interface whose unknowns feed one another.
- E3 a constant gradient field is a fixed point: every solve stops after its first iteration.
- E4 with a pseudo-time step beyond every cell's Courant limit (c = 1), an unknown whose inflow
  neighbours all belong to the side takes the weighted mean of R5's single sweep in one step.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import case


def hex_setup(n, normal, offset, rng):
    """A uniform n^3 hex mesh with a planar interface n_int . (x - x0) = 0 (n_int from vapour to
    liquid): alpha from the signed distance of the cell centroid, interface cells within one cell
    of the plane, n_int the plane normal there, and a seeded random gradient field."""
    m = synth.hex_box(n)
    O = oracle.Oracle(m)
    cen = O.geometry()["cell_cen"]
    nrm = np.asarray(normal, float) / np.linalg.norm(normal)
    d = (cen - 0.5) @ nrm - offset
    h = 1.0 / n
    alpha = np.clip(0.5 + 0.45 * d / h, 0.0, 1.0)
    alpha[np.abs(d) >= h] = np.where(d[np.abs(d) >= h] > 0, 1.0, 0.0)
    iface = ((alpha > 0) & (alpha < 1)).astype(np.uint8)
    alpha[(iface == 1) & (alpha == 0.5)] = 0.55
    n_int = np.where(iface[:, None] == 1, nrm[None, :], 0.0)
    grad = rng.normal(size=(m.n_cells, 3)) * 50.0
    return m, O, cen, alpha, iface, n_int, grad


def neighbours(m, c):
    """(face, neighbour, outward area from c) of every interior face of cell c."""
    out = []
    for f, rev in m.cell_faces(c):
        o, q = int(m.face_owner[f]), int(m.face_neigh[f])
        if q < 0:
            continue
        out.append((f, q if o == c else o, -1.0 if rev else 1.0))
    return out


def test_E1_closed_form_axis_plane():
    rng = np.random.default_rng(3)
    n = 8
    m, O, cen, alpha, iface, n_int, grad = hex_setup(n, (0, 0, -1), 0.03, rng)
    h = 1.0 / n
    assert O.extrap_dtau() == pytest.approx(h / 2, rel=1e-13)
    tol = 1e-3
    r = O.extrapolate(alpha, iface, n_int, grad, max_iter=120, tol=tol)
    liquid = alpha > 0.5
    I = np.where(iface == 1)[0]
    assert len(I) > 0 and np.any(liquid[I]) and np.any(~liquid[I])
    c = 0.5
    for side in (0, 1):  # 0 liquid side (unknowns: vapour interface cells), 1 vapour side
        U = I[liquid[I] == (side == 1)]
        # the single inflow neighbour: one layer towards the side's bulk (-n for the liquid side)
        step = np.array([0, 0, 1.0]) * h * (1 if side == 0 else -1)
        star = np.empty((len(U), 3))
        for t, P in enumerate(U):
            target = cen[P] - step
            Q = np.argmin(np.linalg.norm(cen - target, axis=1))
            assert np.linalg.norm(cen[Q] - target) < 1e-9
            assert liquid[Q] == (side == 0)  # a cell of the side
            star[t] = grad[Q]
        x0 = grad[U]
        for j in range(3):
            amp = np.abs(x0[:, j] - star[:, j]).max()
            K = next((k for k in range(1, 121) if c * (1 - c) ** (k - 1) * amp < tol), 120)
            assert r["iters"][3 * side + j] == K, (side, j)
            want = star[:, j] + (1 - c) ** K * (x0[:, j] - star[:, j])
            np.testing.assert_allclose(r["g_other"][U, j], want, rtol=1e-12, atol=1e-12 * amp)
    assert not np.any(r["status"] & 16)


def upwind_system(m, alpha, iface, n_int, grad, face_area, side):
    """The steady upwind equations of one side as a dense system A x = B over its unknowns U (rows
    of unknowns without inflow: x = start value), and each unknown's inflow weight sum W."""
    liquid = alpha > 0.5
    sigma = 1.0 if side == 0 else -1.0
    U = np.where((iface == 1) & (liquid == (side == 1)))[0]
    pos = {int(P): i for i, P in enumerate(U)}
    A = np.zeros((len(U), len(U)))
    B = np.zeros((len(U), 3))
    for i, P in enumerate(U):
        for f, Q, sign in neighbours(m, int(P)):
            w = sigma * sign * float(n_int[P] @ face_area[f])
            if not w > 0:
                continue
            if liquid[Q] == (side == 0):
                A[i, i] += w
                B[i] += w * grad[Q]
            elif Q in pos:
                A[i, i] += w
                A[i, pos[Q]] -= w
    W = np.diag(A).copy()
    for i, P in enumerate(U):
        if A[i, i] == 0:  # no inflow: keeps its start value
            A[i, i] = 1.0
            B[i] = grad[P]
    return U, A, B, W


def steady_state(m, alpha, iface, n_int, grad, face_area, side):
    """Direct solve of the steady upwind equations of one side (dense, per component)."""
    U, A, B, _ = upwind_system(m, alpha, iface, n_int, grad, face_area, side)
    return U, np.linalg.solve(A, B)


@pytest.mark.parametrize("normal", [(1.0, 0.5, -2.0), (-0.3, 1.0, 0.4)])
def test_E2_steady_state_tilted_plane(normal):
    rng = np.random.default_rng(11)
    m, O, cen, alpha, iface, n_int, grad = hex_setup(8, normal, 0.02, rng)
    fa = O.geometry()["face_area"]
    r = O.extrapolate(alpha, iface, n_int, grad, max_iter=1000, tol=0.0)
    coupled = 0
    for side in (0, 1):
        U, X = steady_state(m, alpha, iface, n_int, grad, fa, side)
        np.testing.assert_allclose(r["g_other"][U], X, rtol=1e-10, atol=1e-10 * np.abs(X).max())
        # the unknowns must feed one another somewhere, or this pin would not test the coupling
        liquid = alpha > 0.5
        sigma = 1.0 if side == 0 else -1.0
        for P in U:
            for f, Q, sign in neighbours(m, int(P)):
                if sigma * sign * float(n_int[P] @ fa[f]) > 0 and iface[Q] and liquid[Q] == liquid[P]:
                    coupled += 1
    assert coupled > 0


@pytest.mark.parametrize("iters", [1, 2, 5])
def test_E5_transient_is_the_jacobi_step(iters):
    """The first iterates, against the explicit step in matrix form, x <- x + F (B - A x) with
    F = diag(min(dtau, V/W) / V) (0 where W = 0): every unknown from the previous iterate."""
    rng = np.random.default_rng(11)
    m, O, cen, alpha, iface, n_int, grad = hex_setup(8, (1.0, 0.5, -2.0), 0.02, rng)
    g = O.geometry()
    dtau = O.extrap_dtau()
    r = O.extrapolate(alpha, iface, n_int, grad, max_iter=iters, tol=0.0)
    for side in (0, 1):
        U, A, B, W = upwind_system(m, alpha, iface, n_int, grad, g["face_area"], side)
        V = g["cell_vol"][U]
        F = np.where(W > 0, np.minimum(dtau, V / np.where(W > 0, W, 1.0)) / V, 0.0)
        x = grad[U].copy()
        for _ in range(iters):
            x = x + F[:, None] * (B - A @ x)
        np.testing.assert_allclose(r["g_other"][U], x, rtol=1e-11, atol=1e-11 * np.abs(x).max())
    assert list(r["iters"]) == [iters] * 6


def test_E3_constant_gradient_is_a_fixed_point():
    m, a, T, Tb = case("voronoi_film")
    O = oracle.Oracle(m)
    rec = O.run(a, T, Tb, synth.PROPS)["recon"]
    iface = ((a > 1e-12) & (a < 1 - 1e-12) & (rec["A_int"] > 0)).astype(np.uint8)
    g = np.tile([3.0, -7.5, 120.25], (m.n_cells, 1))
    r = O.extrapolate(a, iface, rec["n_int"], g)
    assert list(r["iters"]) == [1] * 6
    np.testing.assert_array_equal(r["g_other"][iface == 1], g[iface == 1])


def test_E4_unit_courant_step_is_r5_where_inflow_is_known():
    m, a, T, Tb = case("voronoi_film")
    O = oracle.Oracle(m)
    run = O.run(a, T, Tb, synth.PROPS)
    rec, pc = run["recon"], run["pc"]
    big = O.phase_change(a, rec, T, Tb, synth.PROPS, extrap=dict(dtau=1e30, max_iter=120, tol=1e-9))
    fa = O.geometry()["face_area"]
    liquid = a > 0.5
    I = np.where((a > 1e-12) & (a < 1 - 1e-12) & (rec["A_int"] > 0))[0]
    checked = 0
    for P in I:
        sigma = -1.0 if liquid[P] else 1.0  # the other side
        feeds = [Q for f, Q, sign in neighbours(m, int(P))
                 if sigma * sign * float(rec["n_int"][P] @ fa[f]) > 0]
        if not feeds or any(liquid[Q] == liquid[P] and Q in set(I) for Q in feeds):
            continue
        other = "grad_v" if liquid[P] else "grad_l"
        scale = max(np.abs(pc[other][P]).max(), np.abs(pc["grad"][P]).max())
        np.testing.assert_allclose(big[other][P], pc[other][P], rtol=1e-12, atol=1e-12 * scale)
        checked += 1
    assert checked >= 50, checked  # 76 of the 411 interface cells of this film take no unknown inflow
