"""The seeded workloads at their full sizes: the meshes, alpha and temperature fields that the
benchmark times and the full-size parity tests check. Inputs only: nothing here computes any
part of the reconstruction or the phase-change source.

    film250k    jittered-BCC Voronoi, 2 x 50^3 cells, wavy liquid film
    sphere32    uniform hex 32^3, one vapour sphere R = 0.25 at the centre
    batch64     64 meshes of four kinds, log-uniform sizes 8k-500k cells, 1-6 spheres each
    voronoi2m   jittered-BCC Voronoi, 2 x 100^3 cells (spacing 0.01), 200 vapour spheres with
                R ~ U[0.01, 0.05]: the application case of the learned isovalue guess
    pipe8m      extruded jittered 2D Voronoi disk, 600 layers (about 7.9M cells), wall film with
                axial waves moving one layer per step (the benchmark default: the largest
                single-GPU case, learned and batched over 100 resident steps)
"""
from __future__ import annotations

import numpy as np

from . import alpha, hex_box, pipe, prism_box, temperature, tet_box, voronoi_bcc

NAMES = ("film250k", "sphere32", "batch64", "voronoi2m", "pipe8m")


def spheres(rng, k, r_lo=0.05, r_hi=0.2):
    """k non-overlapping spheres with R ~ U[r_lo, r_hi] inside the unit box (rejection)."""
    out = []
    while len(out) < k:
        R = rng.uniform(r_lo, r_hi)
        c = rng.uniform(R, 1 - R, 3)
        if all(np.linalg.norm(c - np.array(o[:3])) > R + o[3] for o in out):
            out.append((float(c[0]), float(c[1]), float(c[2]), float(R)))
    return out


def workload(name: str, layers: int = 600):
    """(mesh or list of meshes, alpha, T, T_bnd, description, extra). For a list of meshes the
    fields are concatenated in mesh order. `layers` shortens the pipe (same cross-section and
    layer height 0.01, so every layer's cells are those of the full pipe): a smaller case of the
    same kernels for profiling."""
    if name == "film250k":
        m = voronoi_bcc(50, jitter=0.25, seed=1)
        reg = dict(type="film", z0=0.3, a=0.03)
        a = alpha(m, reg, mode="subtet", level=3)
        T, Tb = temperature(m, reg, dict(kind="film", dT=10.0))
        return m, a, T, Tb, ("jittered-BCC Voronoi 2x50^3=250k cells (seed 1, +-h/4), wavy film "
                             "z<0.3+0.03sin(2pi x)sin(2pi y), T linear to T_sat+10 K at the wall"), {}
    if name == "sphere32":
        m = hex_box(32)
        reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.25)])
        a = alpha(m, reg, mode="hexgrid", level=3)
        T, Tb = temperature(m, reg, dict(kind="radial", dT=5.0))
        return m, a, T, Tb, "hex 32^3 unit cube, vapour sphere R=0.25 at the centre, alpha from 8^3 samples", {}
    if name == "batch64":
        rng = np.random.default_rng(3)
        meshes, As, Ts, Tbs, kinds = [], [], [], [], []
        for i in range(64):
            size = float(np.exp(rng.uniform(np.log(8e3), np.log(5e5))))
            kind = ["hex", "tet", "prism", "voronoi"][int(rng.integers(0, 4))]
            if kind == "hex":
                m = hex_box(max(2, round(size ** (1 / 3))))
            elif kind == "tet":
                m = tet_box(max(2, round((size / 6) ** (1 / 3))))
            elif kind == "prism":
                m = prism_box(max(2, round((size / 2) ** (1 / 3))))
            else:
                m = voronoi_bcc(max(2, round((size / 2) ** (1 / 3))), seed=int(rng.integers(0, 2 ** 31)))
            reg = dict(type="spheres", spheres=spheres(rng, int(rng.integers(1, 7))))
            a = alpha(m, reg, mode="hexgrid" if kind == "hex" else "subtet", level=3 if kind == "hex" else 2)
            T, Tb = temperature(m, reg, dict(kind="radial", dT=5.0))
            meshes.append(m); As.append(a); Ts.append(T); Tbs.append(Tb); kinds.append(kind)
        return (meshes, np.concatenate(As), np.concatenate(Ts), np.concatenate(Tbs),
                f"64 meshes (seed 3), sizes log-uniform 8k-500k cells ({sum(m.n_cells for m in meshes)} cells), "
                "kinds uniform over hex/Kuhn-tet/prism/jittered-BCC Voronoi, 1-6 spheres R~U[0.05,0.2], radial T",
                {"kinds": {k: kinds.count(k) for k in set(kinds)}})
    if name == "voronoi2m":
        rng = np.random.default_rng(100)
        m = voronoi_bcc(100, jitter=0.25, seed=100)
        reg = dict(type="spheres", spheres=spheres(rng, 200, 0.01, 0.05))
        a = alpha(m, reg, mode="subtet", level=2)
        T, Tb = temperature(m, reg, dict(kind="radial", dT=5.0))
        return m, a, T, Tb, ("jittered-BCC Voronoi 2x100^3=2M cells (seed 100, +-h/4), 200 non-overlapping vapour "
                             "spheres R~U[0.01,0.05], alpha from 64 sub-tetrahedra per fan tetrahedron, radial T"), {}
    if name == "pipe8m":
        m = pipe(spacing=0.01537, layers=layers, radius=1.0, length=6.0 * layers / 600, seed=5)
        reg = dict(type="pipe", r0=0.9, a=0.04, lam=0.5, t=0.0)
        a = alpha(m, reg, mode="subtet", level=2)
        T, Tb = temperature(m, reg, dict(kind="pipe", dT=8.0, radius=1.0))
        return m, a, T, Tb, (f"extruded jittered 2D Voronoi disk (radius 1, {layers} layers over length "
                             f"{6.0 * layers / 600:g}, {m.n_cells} cells), wall film r > 0.9 - 0.04 sin(2pi(z-t)/0.5) "
                             "moving one layer (dz = 0.01 = phase velocity x dt) per step, T_sat+8 K at the wall"), \
            {"layers": layers}
    raise KeyError(f"unknown workload {name}")
