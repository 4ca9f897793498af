"""Seeded synthetic inputs shared by the oracle and the CUDA library.

Meshes (uniform hex, Kuhn 6-tet split hex, 2-prism split hex, jittered-BCC Voronoi clipped to a
box, extruded jittered 2D Voronoi pipe) come from ``libsynth.so`` (``synth.cpp``); the volume
fraction ``alpha`` is the sampled liquid fraction of an analytic interface, and the temperature
is an analytic profile evaluated at cell centroids and boundary-face centroids.

This module holds none of the method's arithmetic: it only writes inputs. Both consumers derive
their own geometry from the primitive arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

T_SAT = 373.15
PROPS = dict(k_l=0.68, k_v=0.025, h_lv=2.26e6, T_sat=T_SAT)


def build(force: bool = False) -> str:
    """Compiles libsynth.so next to this file (g++, OpenMP) and returns its path."""
    so = os.path.join(_HERE, "libsynth.so")
    src = os.path.join(_HERE, "synth.cpp")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        vp, dp, i64p, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p
        for name in ("synth_hex", "synth_tet", "synth_prism"):
            f = getattr(lib, name)
            f.restype = vp
            f.argtypes = [ctypes.c_int] * 3 + [dp, dp]
        lib.synth_voronoi_bcc.restype = vp
        lib.synth_voronoi_bcc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, dp, dp]
        lib.synth_voronoi_sites.restype = vp
        lib.synth_voronoi_sites.argtypes = [dp, ctypes.c_int64, ctypes.c_double, dp, dp]
        lib.synth_pipe.restype = vp
        lib.synth_pipe.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64]
        lib.synth_sizes.argtypes = [vp, ctypes.c_void_p]
        lib.synth_copy.argtypes = [vp] + [ctypes.c_void_p] * 9
        lib.synth_free.argtypes = [vp]
        mesh_args = [ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, vp]
        lib.synth_alpha.argtypes = mesh_args + [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.synth_points.argtypes = mesh_args + [vp, vp]
        _LIB = lib
    return _LIB


@dataclass
class Mesh:
    """Primitive polyhedral mesh arrays (host, numpy). See synth.cpp for the format."""
    kind: str
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    face_vert_off: np.ndarray
    face_vert: np.ndarray
    face_owner: np.ndarray
    face_neigh: np.ndarray
    cell_face_off: np.ndarray
    cell_face: np.ndarray
    conform_errors: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return len(self.cell_face_off) - 1

    @property
    def n_faces(self) -> int:
        return len(self.face_owner)

    @property
    def n_verts(self) -> int:
        return len(self.vx)

    def _args(self):
        p = lambda a: a.ctypes.data
        return [self.n_cells, p(self.vx), p(self.vy), p(self.vz), self.n_verts, p(self.face_vert_off),
                p(self.face_vert), self.n_faces, p(self.cell_face_off), p(self.cell_face)]

    def cell_faces(self, c: int):
        """(face id, reversed) pairs of cell c."""
        out = []
        for e in self.cell_face[self.cell_face_off[c]:self.cell_face_off[c + 1]]:
            e = int(e)
            out.append((e & 0x7FFFFFFF, e < 0))
        return out

    def face_loop(self, f: int) -> np.ndarray:
        return self.face_vert[self.face_vert_off[f]:self.face_vert_off[f + 1]]


def _take(h, kind: str, **meta) -> Mesh:
    lib = _lib()
    sz = np.zeros(6, np.int64)
    lib.synth_sizes(h, sz.ctypes.data)
    nc, nf, nv, nfv, ncf, err = (int(x) for x in sz)
    m = Mesh(kind, np.empty(nv), np.empty(nv), np.empty(nv), np.empty(nf + 1, np.int64),
             np.empty(nfv, np.int32), np.empty(nf, np.int32), np.empty(nf, np.int32),
             np.empty(nc + 1, np.int64), np.empty(ncf, np.int32), err, dict(meta))
    lib.synth_copy(h, *[a.ctypes.data for a in (m.vx, m.vy, m.vz, m.face_vert_off, m.face_vert,
                                                  m.face_owner, m.face_neigh, m.cell_face_off, m.cell_face)])
    lib.synth_free(h)
    return m


def _box(lo, hi):
    lo = (ctypes.c_double * 3)(*lo)
    hi = (ctypes.c_double * 3)(*hi)
    return lo, hi


def hex_box(nx, ny=None, nz=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _take(_lib().synth_hex(nx, ny, nz, *_box(lo, hi)), "hex", n=(nx, ny, nz), lo=lo, hi=hi)


def tet_box(nx, ny=None, nz=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _take(_lib().synth_tet(nx, ny, nz, *_box(lo, hi)), "tet", n=(nx, ny, nz), lo=lo, hi=hi)


def prism_box(nx, ny=None, nz=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _take(_lib().synth_prism(nx, ny, nz, *_box(lo, hi)), "prism", n=(nx, ny, nz), lo=lo, hi=hi)


def voronoi_bcc(n, jitter=0.25, seed=1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    """Voronoi cells of a BCC lattice with cubic spacing h = 1/n (2 n^3 sites), each site
    jittered uniformly by +-jitter*h per axis (std::mt19937_64 seeded with `seed`), clipped to
    the box."""
    return _take(_lib().synth_voronoi_bcc(n, jitter, seed, *_box(lo, hi)), "voronoi", n=n, seed=seed,
                 jitter=jitter, lo=lo, hi=hi)


def voronoi_sites(sites: np.ndarray, h: float, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    s = np.ascontiguousarray(sites, dtype=np.float64)
    return _take(_lib().synth_voronoi_sites(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(s), h,
                                            *_box(lo, hi)), "voronoi", lo=lo, hi=hi)


def pipe(spacing=0.01537, layers=600, radius=1.0, length=6.0, jitter=0.25, seed=5) -> Mesh:
    """Extruded jittered 2D Voronoi disk: a pipe of the given radius and length."""
    return _take(_lib().synth_pipe(spacing, layers, radius, length, jitter, seed), "pipe", spacing=spacing,
                 layers=layers, radius=radius, length=length, seed=seed)


# ------------------------------------------------------------------------------------ fields
_REGION = {"plane": 0, "spheres": 1, "film": 2, "pipe": 3}


def region_params(region: dict) -> tuple[int, np.ndarray]:
    t = region["type"]
    if t == "plane":     # liquid where n.x < d
        p = list(region["n"]) + [region["d"]]
    elif t == "spheres":  # vapour inside every sphere (cx, cy, cz, R)
        p = [x for s in region["spheres"] for x in s]
    elif t == "film":    # liquid below z0 + a sin(2 pi x/lx) sin(2 pi y/ly)
        p = [region["z0"], region["a"], region.get("lx", 1.0), region.get("ly", 1.0)]
    elif t == "pipe":    # liquid at r > r0 - a sin(2 pi (z - t)/lam)
        p = [region["r0"], region["a"], region["lam"], region.get("t", 0.0)]
    else:
        raise ValueError(t)
    return _REGION[t], np.asarray(p, np.float64)


def alpha(mesh: Mesh, region: dict, mode: str = "subtet", level: int = 3) -> np.ndarray:
    """Liquid volume fraction per cell.

    mode 'subtet': each fan tetrahedron of the cell is refined `level` times (8**level sub-tets),
    the indicator is sampled at sub-tet centroids. mode 'hexgrid': (2**level)**3 midpoint samples
    of the cell's bounding box (axis-aligned hex cells)."""
    t, p = region_params(region)
    out = np.empty(mesh.n_cells)
    _lib().synth_alpha(*mesh._args(), t, p.ctypes.data, len(p), 0 if mode == "subtet" else 1, level,
                       out.ctypes.data)
    return out


def points(mesh: Mesh) -> tuple[np.ndarray, np.ndarray]:
    """(cell centroids [n_cells,3], face centroids [n_faces,3]) for evaluating profiles."""
    c = np.empty((mesh.n_cells, 3))
    f = np.empty((mesh.n_faces, 3))
    _lib().synth_points(*mesh._args(), c.ctypes.data, f.ctypes.data)
    return c, f


_CHUNK = 1 << 16


def _nearest_sphere(s: np.ndarray, x: np.ndarray):
    """(j, r_j, g) per point: the sphere j minimising |x - c_j| - R_j, the distance to its centre,
    and that minimum. Few spheres: brute force. Many: the 8 nearest centres from a k-d tree, which
    settle the minimum wherever the 8th centre is at least R_max beyond it; the other points fall
    back to brute force."""
    def brute(xs):
        r = np.linalg.norm(xs[:, None, :] - s[None, :, :3], axis=2)
        j = np.argmin(r - s[None, :, 3], axis=1)
        rr = r[np.arange(len(xs)), j]
        return j, rr, rr - s[j, 3]
    k = 8
    if len(s) <= 4 * k:
        return brute(x)
    from scipy.spatial import cKDTree
    d, idx = cKDTree(s[:, :3]).query(x, k=k, workers=-1)
    r = np.linalg.norm(x[:, None, :] - s[idx, :3], axis=2)
    gk = r - s[idx, 3]
    a = np.argmin(gk, axis=1)
    rows = np.arange(len(x))
    j, rr, g = idx[rows, a], r[rows, a], gk[rows, a]
    bad = np.nonzero(d[:, -1] - s[:, 3].max() < g)[0]
    if len(bad):
        j[bad], rr[bad], g[bad] = brute(x[bad])
    return j, rr, g


def region_g(region: dict, x: np.ndarray) -> np.ndarray:
    """Signed liquid indicator g(x) (> 0 in the liquid) of a region, vectorised."""
    if len(x) > _CHUNK:
        return np.concatenate([region_g(region, x[i:i + _CHUNK]) for i in range(0, len(x), _CHUNK)])
    t = region["type"]
    if t == "plane":
        return region["d"] - x @ np.asarray(region["n"], float)
    if t == "spheres":
        return _nearest_sphere(np.asarray(region["spheres"], float), x)[2]
    if t == "film":
        return (region["z0"] + region["a"] * np.sin(2 * np.pi * x[:, 0] / region.get("lx", 1.0))
                * np.sin(2 * np.pi * x[:, 1] / region.get("ly", 1.0)) - x[:, 2])
    if t == "pipe":
        r = np.hypot(x[:, 0], x[:, 1])
        return r - (region["r0"] - region["a"] * np.sin(2 * np.pi * (x[:, 2] - region.get("t", 0.0)) / region["lam"]))
    raise ValueError(t)


def temperature_at(region: dict, profile: dict, x: np.ndarray) -> np.ndarray:
    """Analytic temperature at points x [n,3].

    profile kinds:
      'radial'  liquid outside spheres: T_sat + dT (1 - R/r) from the nearest sphere; vapour T_sat
      'film'    liquid below the film: T_sat + dT (1 - z/eta); vapour T_sat
      'pipe'    liquid r > r_G: T_sat + dT (r - r_G)/(radius - r_G); vapour T_sat
      'linear'  T = T0 + g.x everywhere
      'stefan'  vapour x < x_g: T_sat + dT (1 - x/x_g); liquid T_sat
      'quadratic' T = T0 + g.x + 0.5 x^T H x
    """
    if len(x) > _CHUNK:  # bounded temporaries (sphere regions broadcast points x spheres)
        return np.concatenate([temperature_at(region, profile, x[i:i + _CHUNK]) for i in range(0, len(x), _CHUNK)])
    k = profile["kind"]
    Ts = profile.get("T_sat", T_SAT)
    if k == "linear":
        return profile["T0"] + x @ np.asarray(profile["g"], float)
    if k == "quadratic":
        H = np.asarray(profile["H"], float)
        return profile["T0"] + x @ np.asarray(profile["g"], float) + 0.5 * np.einsum("ni,ij,nj->n", x, H, x)
    if k == "stefan":
        xg = profile["x_g"]
        return np.where(x[:, 0] < xg, Ts + profile["dT"] * (1 - x[:, 0] / xg), Ts)
    liquid = region_g(region, x) > 0
    if k == "radial":
        s = np.asarray(region["spheres"], float)
        j, rr, _ = _nearest_sphere(s, x)
        RR = s[j, 3]
        T = Ts + profile["dT"] * (1 - RR / np.maximum(rr, 1e-300))
    elif k == "film":
        eta = region["z0"] + region["a"] * np.sin(2 * np.pi * x[:, 0] / region.get("lx", 1.0)) * np.sin(
            2 * np.pi * x[:, 1] / region.get("ly", 1.0))
        T = Ts + profile["dT"] * (1 - x[:, 2] / eta)
    elif k == "pipe":
        r = np.hypot(x[:, 0], x[:, 1])
        rg = region["r0"] - region["a"] * np.sin(2 * np.pi * (x[:, 2] - region.get("t", 0.0)) / region["lam"])
        T = Ts + profile["dT"] * (r - rg) / (profile.get("radius", 1.0) - rg)
    else:
        raise ValueError(k)
    return np.where(liquid, T, Ts)


def temperature(mesh: Mesh, region: dict, profile: dict, pts=None) -> tuple[np.ndarray, np.ndarray]:
    """(T at cell centroids [n_cells], T at face centroids [n_faces]; only boundary faces are
    read by the consumers)."""
    c, f = points(mesh) if pts is None else pts
    return temperature_at(region, profile, c), temperature_at(region, profile, f)
