"""Stencil-anisotropy study (Sec. 3, "Origin of the gradient anisotropy", Fig. stencil_polar): the
least-squares gradient of Appendix B applied to an analytical temperature field around a sphere,
for the standard and interface-modified stencils, with and without inverse-distance weights, on
face and vertex neighbours, on a hexahedral and a polyhedral mesh.

The field: T = T_sat + G (r - R) in the liquid (r > R) and T_sat in the vapour sphere, so the
exact gradient magnitude next to the interface is G. The cells: liquid band cells within 1.5 cell
widths of the sphere, in the equatorial slab |z - z_c| < h. Per variant the script bins
|grad T| / G by the azimuth and reports the bin means' minimum / maximum ratio (the paper's
anisotropy measure), the relative amplitude of the bin means' four-fold Fourier mode, the mean
ratio and the median cond(G_P). On a Voronoi mesh the vertex stencil equals the face stencil: the
four cells around a Voronoi vertex form a Delaunay tetrahedron, so every two of them share a face.
Everything runs on the GPU through the library (one step per variant).

    python -m paper_2604_14938_gb300.stencil_study [--n 64] [--json out.json]
"""
import argparse
import json

import numpy as np

VARIANTS = {  # name -> options.lsq_variant bits (8: cond(G_P) as well)
    "standard": 1 | 8,
    "modified": 0 | 8,
    "standard, inverse-distance": 1 | 2 | 8,
    "modified, inverse-distance": 2 | 8,
    "standard, vertex stencil": 1 | 4 | 8,
    "modified, vertex stencil": 4 | 8,
}


def sphere_case(kind: str, n: int, R: float, seed: int = 3):
    """Mesh, alpha (vapour sphere of radius R at the box centre), cell and face centroids."""
    import synth
    if kind == "hex":
        m = synth.hex_box(n)
        a = synth.alpha(m, dict(type="spheres", spheres=[(0.5, 0.5, 0.5, R)]), mode="hexgrid", level=3)
    else:  # polyhedral: jittered-BCC Voronoi with about the same cell count
        m = synth.voronoi_bcc(max(4, int(round(n / 2 ** (1 / 3)))), seed=seed)
        a = synth.alpha(m, dict(type="spheres", spheres=[(0.5, 0.5, 0.5, R)]), mode="subtet", level=2)
    return m, a


def analytic_T(x: np.ndarray, R: float, G: float, T_sat: float) -> np.ndarray:
    r = np.linalg.norm(x - 0.5, axis=1)
    return np.where(r > R, T_sat + G * (r - R), T_sat)


def anisotropy(theta: np.ndarray, ratio: np.ndarray, bins: int) -> tuple[float, float]:
    """(min / max of the azimuth-bin means of ratio, relative amplitude of the bin means'
    four-fold Fourier mode). The bin means weigh every bin alike, so that the mesh's uneven
    angular sampling does not enter; the amplitude of m(theta) = m0 (1 + eps cos 4 (theta - c))
    is eps."""
    k = np.clip(((theta + np.pi) / (2 * np.pi) * bins).astype(int), 0, bins - 1)
    filled = [b for b in range(bins) if np.any(k == b)]
    means = np.array([ratio[k == b].mean() for b in filled])
    centres = -np.pi + (np.array(filled) + 0.5) * (2 * np.pi / bins)
    four = 2 * np.abs(np.mean((means - means.mean()) * np.exp(4j * centres))) / means.mean()
    return float(means.min() / means.max()), float(four)


def study(kind: str = "hex", n: int = 64, R: float = 0.3, G: float = 1000.0, bins: int = 24) -> dict:
    import torch
    import synth
    from . import Mesh, default_options

    m, a = sphere_case(kind, n, R)
    M = Mesh(m)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    cen = M.field("cell_cen").cpu().numpy()
    fcen = M.field("face_cen").cpu().numpy()
    T_sat = synth.PROPS["T_sat"]
    T, Tb = analytic_T(cen, R, G, T_sat), analytic_T(fcen, R, G, T_sat)
    ta, tT, tTb = dev(a), dev(T), dev(Tb)
    mdot = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    Q, tot = torch.empty_like(mdot), torch.empty(2, dtype=torch.float64, device="cuda")
    h = (1.0 / m.n_cells) ** (1 / 3)
    rr = np.linalg.norm(cen - 0.5, axis=1)
    theta = np.arctan2(cen[:, 1] - 0.5, cen[:, 0] - 0.5)
    out = {"mesh": kind, "n_cells": int(m.n_cells), "h": h, "R": R, "G": G, "variants": {}}
    for name, bits in VARIANTS.items():
        M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, default_options(lsq_variant=bits))
        torch.cuda.synchronize()
        band = (M.field("band_stamp").cpu().numpy() == M.counts()["step"])
        sel = band & (a > 0.5) & (rr > R) & (rr - R < 1.5 * h) & (np.abs(cen[:, 2] - 0.5) < h)
        g = M.field("grad").cpu().numpy()[sel]
        ratio = np.linalg.norm(g, axis=1) / G
        mm, four = anisotropy(theta[sel], ratio, bins)
        cond = M.field("lsq_cond").cpu().numpy()[sel]
        out["variants"][name] = dict(cells=int(sel.sum()), mean_ratio=float(ratio.mean()),
                                     min_over_max=mm, fourfold=four,
                                     median_cond=float(np.median(cond)), max_cond=float(cond.max()))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64, help="hexahedra per box edge (the polyhedral mesh matches the count)")
    ap.add_argument("--R", type=float, default=0.3)
    ap.add_argument("--json", default="")
    args = ap.parse_args()
    res = [study("hex", args.n, args.R), study("voronoi", args.n, args.R)]
    print("| mesh | variant | cells | mean |grad T| / G | bin min / max | four-fold amplitude | median cond | max cond |")
    print("|---|---|---|---|---|---|---|---|")
    for r in res:
        for name, v in r["variants"].items():
            print(f"| {r['mesh']} {r['n_cells']} | {name} | {v['cells']} | {v['mean_ratio']:.4f} | "
                  f"{v['min_over_max']:.3f} | {v['fourfold']:.4f} | {v['median_cond']:.2f} | {v['max_cond']:.1f} |")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
