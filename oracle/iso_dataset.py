"""Training set for the isovalue-guess MLP, labelled by the oracle — TEST INFRASTRUCTURE ONLY.

Samples are interface cells of seeded meshes (jittered-BCC Voronoi, uniform hex, Kuhn tets)
cut by random planes and random groups of spheres. Each cell's vertex field is the oracle's
inverse-distance field of the sampled alpha, and its label is the oracle's bisection isovalue
as a normalised position t = (c - phi_min)/(phi_max - phi_min).

Features (40 per cell; the definition the GPU kernel restates):
  0      alpha
  1      number of faces / 32
  2..33  vertex values normalised to [0, 1] over the cell's range, sorted descending, padded
         to 32 with the last (smallest) value
  34..36 bounding-box extents / V^(1/3)
  37..39 (vertex mean - bounding-box centre) / V^(1/3)
Cells with more than 32 vertices or a degenerate range are not samples.

Run as a script to write an .npz with float32 features X [n, 40] and labels t [n]:
  python -m oracle.iso_dataset --samples 2000000 --seeds 0-9 --jobs 10 --out iso_train.npz
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

N_FEAT = 40
MAX_V = 32


def cell_features(m, c: int, phi: np.ndarray, alpha: float, V: float):
    """Features of one cell, or None when it has more than 32 vertices or a degenerate range."""
    vs = set()
    nf = 0
    for k in range(m.cell_face_off[c], m.cell_face_off[c + 1]):
        f = int(m.cell_face[k]) & 0x7FFFFFFF
        vs.update(int(v) for v in m.face_vert[m.face_vert_off[f]:m.face_vert_off[f + 1]])
        nf += 1
    vs = np.array(sorted(vs))
    if len(vs) > MAX_V:
        return None
    p = phi[vs]
    lo, hi = p.min(), p.max()
    if hi - lo < 1e-14:
        return None
    u = np.sort((p - lo) / (hi - lo))[::-1]
    u = np.concatenate([u, np.full(MAX_V - len(u), u[-1])])
    P = np.stack([m.vx[vs], m.vy[vs], m.vz[vs]], 1)
    bmin, bmax = P.min(0), P.max(0)
    s = V ** (1.0 / 3.0)
    ext = (bmax - bmin) / s
    off = (P.mean(0) - 0.5 * (bmin + bmax)) / s
    return np.concatenate([[alpha, nf / 32.0], u, ext, off])


def features(m, cells, phi, alpha, vol):
    """[len(cells), 40] features (rows of NaN where a cell is not a sample)."""
    out = np.full((len(cells), N_FEAT), np.nan)
    for i, c in enumerate(cells):
        f = cell_features(m, int(c), phi, float(alpha[c]), float(vol[c]))
        if f is not None:
            out[i] = f
    return out


def random_region(rng):
    if rng.uniform() < 0.5:
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        return dict(type="plane", n=tuple(n), d=float(n @ rng.uniform(0.3, 0.7, 3)))
    k = int(rng.integers(1, 4))
    return dict(type="spheres", spheres=[tuple(rng.uniform(0.25, 0.75, 3)) + (float(rng.uniform(0.08, 0.3)),)
                                         for _ in range(k)])


def make(seed: int, samples: int, log=sys.stderr):
    import oracle
    import synth

    rng = np.random.default_rng(seed)
    X, T = [], []
    got = 0
    t0 = time.time()
    while got < samples:
        kind = ["voronoi", "hex", "tet"][int(rng.integers(0, 3))]
        n = int(rng.integers(10, 22))
        if kind == "voronoi":
            m = synth.voronoi_bcc(n, seed=int(rng.integers(0, 2 ** 31)))
        elif kind == "hex":
            m = synth.hex_box(n)
        else:
            m = synth.tet_box(max(6, n // 2))
        O = oracle.Oracle(m)
        vol = O.geometry()["cell_vol"]
        for _ in range(4):
            reg = random_region(rng)
            a = synth.alpha(m, reg, mode="subtet", level=2)
            phi = O.vertex_field(a)
            I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0]
            if len(I) == 0:
                continue
            F = features(m, I, phi, a, vol)
            ok = ~np.isnan(F[:, 0])
            I, F = I[ok], F[ok]
            r = O.reconstruct(a, phi, cells=I)
            conv = r["status"][I] == 0
            I, F = I[conv], F[conv]
            lo = np.array([phi[list(_verts(m, c))].min() for c in I])
            hi = np.array([phi[list(_verts(m, c))].max() for c in I])
            t = (r["iso"][I] - lo) / (hi - lo)
            X.append(F.astype(np.float32))
            T.append(t.astype(np.float32))
            got += len(I)
            if got >= samples:
                break
        print(f"seed {seed}: {got}/{samples} samples, {time.time() - t0:.0f} s", file=log, flush=True)
    X = np.concatenate(X)[:samples]
    T = np.concatenate(T)[:samples]
    return X, T


def _verts(m, c):
    vs = set()
    for k in range(m.cell_face_off[c], m.cell_face_off[c + 1]):
        f = int(m.cell_face[k]) & 0x7FFFFFFF
        vs.update(int(v) for v in m.face_vert[m.face_vert_off[f]:m.face_vert_off[f + 1]])
    return vs


def _one(args):
    seed, per = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return make(seed, per)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=2_000_000)
    ap.add_argument("--seeds", default="0-9")
    ap.add_argument("--jobs", type=int, default=1, help="worker processes (one seed each)")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    a, b = (int(x) for x in args.seeds.split("-"))
    seeds = list(range(a, b + 1))
    per = args.samples // len(seeds)
    if args.jobs > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(args.jobs) as pool:
            res = pool.map(_one, [(s, per) for s in seeds])
    else:
        res = [make(s, per) for s in seeds]
    np.savez(args.out, X=np.concatenate([r[0] for r in res]), t=np.concatenate([r[1] for r in res]),
             seeds=np.array(seeds))


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
