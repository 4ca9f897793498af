"""Helpers shared by the GPU tests: seeded cases, one GPU step through the C ABI, and the
comparison rule for floating-point outputs."""
import numpy as np

import synth

EPS = 1e-12


def close(gpu, orc, rel=1e-8):
    """|gpu - orc| <= rel * max(|orc|, 1e-3 max|orc|), elementwise (a plain relative error is
    undefined where q_l ~ -q_v)."""
    gpu, orc = np.asarray(gpu, float), np.asarray(orc, float)
    if orc.size == 0:
        return True, 0.0
    floor = 1e-3 * np.abs(orc).max() if orc.size else 0.0
    scale = np.maximum(np.abs(orc), floor)
    scale = np.where(scale == 0, 1.0, scale)
    err = np.abs(gpu - orc) / scale
    return bool(np.all(err <= rel)), float(err.max())


def case(name):
    """(mesh, alpha, T, T_bnd) of a seeded small case."""
    if name == "hex_sphere":
        m = synth.hex_box(32)
        reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.25)])
        a = synth.alpha(m, reg, mode="hexgrid", level=3)
        prof = dict(kind="radial", dT=5.0)
    elif name == "voronoi_film":
        m = synth.voronoi_bcc(14, seed=1)
        reg = dict(type="film", z0=0.3, a=0.03)
        a = synth.alpha(m, reg, mode="subtet", level=2)
        prof = dict(kind="film", dT=10.0)
    elif name == "voronoi_spheres":
        m = synth.voronoi_bcc(12, seed=5)
        reg = dict(type="spheres", spheres=[(0.3, 0.35, 0.4, 0.17), (0.7, 0.62, 0.6, 0.2)])
        a = synth.alpha(m, reg, mode="subtet", level=2)
        prof = dict(kind="radial", dT=5.0)
    elif name == "tet_sphere":
        m = synth.tet_box(10)
        reg = dict(type="spheres", spheres=[(0.45, 0.5, 0.55, 0.3)])
        a = synth.alpha(m, reg, mode="subtet", level=2)
        prof = dict(kind="radial", dT=5.0)
    elif name == "prism_sphere":
        m = synth.prism_box(12)
        reg = dict(type="spheres", spheres=[(0.5, 0.45, 0.5, 0.28)])
        a = synth.alpha(m, reg, mode="subtet", level=2)
        prof = dict(kind="radial", dT=5.0)
    elif name == "pipe_film":
        m = synth.pipe(spacing=0.1, layers=16, radius=1.0, length=1.0, seed=5)
        reg = dict(type="pipe", r0=0.9, a=0.04, lam=0.5, t=0.0)
        a = synth.alpha(m, reg, mode="subtet", level=2)
        prof = dict(kind="pipe", dT=8.0, radius=1.0)
    elif name == "voronoi_many_spheres":  # about 15.0k interface cells
        from synth.workloads import spheres
        m = synth.voronoi_bcc(36, seed=7)
        reg = dict(type="spheres", spheres=spheres(np.random.default_rng(7), 130, 0.04, 0.09))
        a = synth.alpha(m, reg, mode="subtet", level=1)
        prof = dict(kind="radial", dT=5.0)
    else:
        raise KeyError(name)
    T, Tb = synth.temperature(m, reg, prof)
    return m, a, T, Tb


def gpu_step(m, a, T, Tb, props=None, dev_mesh=None, n_cells=None, **opt):
    """Runs one step through the C ABI; returns (device mesh, dict of numpy outputs). `m` may be
    None when `dev_mesh` and `n_cells` are given."""
    import torch
    import paper_2604_14938_gb300 as vof
    props = props or synth.PROPS
    M = dev_mesh or vof.Mesh(m)
    nc = m.n_cells if m is not None else n_cells
    d = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    ta, tT = d(a), d(T)
    tTb = None if Tb is None else d(Tb)
    mdot = torch.empty(nc, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(mdot)
    tot = torch.empty(2, dtype=torch.float64, device="cuda")
    M.step(ta, tT, tTb, props, mdot, Q, tot, vof.default_options(**opt))
    torch.cuda.synchronize()
    out = {k: M.field(k).cpu().numpy() for k in vof.FIELDS}
    out.update(mdot=mdot.cpu().numpy(), Q=Q.cpu().numpy(), totals=tot.cpu().numpy(), counts=M.counts())
    return M, out


def rel_err(x, y):
    """Per-element (per-row for vectors: Euclidean norm) error of x against y, relative to
    max(|y|, 1e-3 max|y|)."""
    x, y = np.asarray(x, float), np.asarray(y, float)
    if y.ndim == 2:
        dn, yn = np.linalg.norm(x - y, axis=1), np.linalg.norm(y, axis=1)
    else:
        dn, yn = np.abs(x - y), np.abs(y)
    if yn.size == 0:
        return dn
    scale = np.maximum(yn, 1e-3 * yn.max())
    return dn / np.where(scale == 0, 1.0, scale)


def ulp_spread(O, a, rec, T, Tb, props, keys, draws=2, seed=0, **pc_kw):
    """The oracle's own conditioning, cell by cell: the largest rel_err of its downstream outputs
    when every cell centroid is moved by at most one ulp (random sign). Returns (unperturbed
    outputs, {key: spread per row}); pc_kw goes to the oracle's phase_change."""
    g = O.geometry()
    cen0 = g["cell_cen"].copy()
    pc0 = O.phase_change(a, rec, T, Tb, props, **pc_kw)
    rng = np.random.default_rng(seed)
    spread = {k: np.zeros(len(pc0[k])) for k in keys}
    try:
        for _ in range(draws):
            s = rng.integers(-1, 2, cen0.shape)
            g["cell_cen"][:] = np.where(s > 0, np.nextafter(cen0, np.inf), np.where(s < 0, np.nextafter(cen0, -np.inf), cen0))
            pc = O.phase_change(a, rec, T, Tb, props, **pc_kw)
            for k in keys:
                spread[k] = np.maximum(spread[k], rel_err(pc[k], pc0[k]))
    finally:
        g["cell_cen"][:] = cen0
    return pc0, spread


def within(gpu, orc, spread, rel=1e-8, factor=100.0):
    """(ok, worst ratio): rel_err(gpu, orc) <= max(rel, factor * spread) row by row. Where the
    oracle's own answer moves by more than rel/factor under one-ulp input rounding (an
    ill-conditioned least-squares stencil), the allowance grows with it."""
    e = rel_err(gpu, orc)
    allow = np.maximum(rel, factor * np.asarray(spread))
    r = e / allow
    return bool(np.all(r <= 1.0)), float(r.max()) if r.size else 0.0
