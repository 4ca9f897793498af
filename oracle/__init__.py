"""FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of the sharp-interface VOF phase-change hot path (liboracle.so, from
oracle.cpp) plus an FP64 NumPy restatement of the isovalue-guess MLP (oracle.mlp). It exists to
check the CUDA library: only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import it. It shares no code with the library.

Pinned only in special cases (no independent reference exists for general inputs): the one-sweep
per-side gradient (closed forms when the neighbour gradients are equal; its upwind weights also
enter the pseudo-time solve, whose first step at a Courant number of 1 reproduces it). The
inverse-distance vertex field and the choice between two interface planes on one face are pinned
by cases worked by hand (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

ST_DEGENERATE = 1
ST_NOT_CONVERGED = 2
ST_SINGULAR_LSQ = 8
ST_NO_SIDE = 16

XF_RECON, XF_LINEAR, XF_AS_PRINTED = 0, 1, 2


def build(force: bool = False) -> str:
    so = os.path.join(_HERE, "liboracle.so")
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, so)
    return so


class _OrcMesh(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("n_verts", ctypes.c_int64),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
                ("face_vert_off", ctypes.c_void_p), ("face_vert", ctypes.c_void_p),
                ("face_owner", ctypes.c_void_p), ("face_neigh", ctypes.c_void_p),
                ("cell_face_off", ctypes.c_void_p), ("cell_face", ctypes.c_void_p)]


class _OrcExtrap(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("dtau", ctypes.c_double),
                ("iters", ctypes.c_int32 * 6)]


class _OrcProps(ctypes.Structure):
    _fields_ = [("k_l", ctypes.c_double), ("k_v", ctypes.c_double), ("h_lv", ctypes.c_double),
                ("T_sat", ctypes.c_double)]


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
        _LIB.orc_liquid_volume.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_void_p]
        _LIB.orc_reconstruct.argtypes = ([ctypes.c_void_p] * 4 + [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 7)
        _LIB.orc_reconstruct_m.argtypes = ([ctypes.c_void_p] * 4 + [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double]
                                          + [ctypes.c_void_p] * 7)
        _LIB.orc_phase_change.argtypes = ([ctypes.c_void_p] * 6 + [ctypes.c_double] + [ctypes.c_void_p] * 6
                                          + [ctypes.c_int] + [ctypes.c_void_p] * 16)
        _LIB.orc_extrap_dtau.argtypes = [ctypes.c_void_p] * 4
        _LIB.orc_lsq_study.argtypes = ([ctypes.c_void_p] * 6 + [ctypes.c_double] + [ctypes.c_void_p] * 3
                                       + [ctypes.c_int] + [ctypes.c_void_p] * 3)
        _LIB.orc_sym3_eigenvalues.argtypes = [ctypes.c_void_p] * 2
        _LIB.orc_extrapolate.argtypes = ([ctypes.c_void_p] * 7 + [ctypes.c_double, ctypes.c_int, ctypes.c_double]
                                         + [ctypes.c_void_p] * 3)
        _LIB.orc_vertex_field.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
        _LIB.orc_geometry.argtypes = [ctypes.c_void_p] * 5
        _LIB.orc_pairwise_sum.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _LIB.orc_interface_htc.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_double] * 2 + [ctypes.c_void_p] * 2
        _LIB.orc_htc_cell_sums.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_double] + [ctypes.c_void_p] * 2
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """Oracle bound to one mesh (any object with the synth.Mesh arrays)."""

    def __init__(self, mesh):
        self.mesh = mesh
        self._keep = [np.ascontiguousarray(a) for a in (mesh.vx, mesh.vy, mesh.vz, mesh.face_vert_off,
                                                          mesh.face_vert, mesh.face_owner, mesh.face_neigh,
                                                          mesh.cell_face_off, mesh.cell_face)]
        k = self._keep
        self.c = _OrcMesh(len(mesh.cell_face_off) - 1, len(mesh.face_owner), len(mesh.vx),
                          *[a.ctypes.data for a in k])
        self.ref = ctypes.byref(self.c)
        self._geo = None

    @property
    def n_cells(self):
        return self.c.n_cells

    def geometry(self) -> dict:
        """face_area (outward from owner) [nf,3], face_cen [nf,3], cell_vol [nc], cell_cen [nc,3]."""
        if self._geo is None:
            nf, nc = self.c.n_faces, self.c.n_cells
            g = dict(face_area=np.empty((nf, 3)), face_cen=np.empty((nf, 3)), cell_vol=np.empty(nc),
                     cell_cen=np.empty((nc, 3)))
            _lib().orc_geometry(self.ref, *[_p(g[k]) for k in ("face_area", "face_cen", "cell_vol", "cell_cen")])
            self._geo = g
        return self._geo

    def vertex_field(self, alpha: np.ndarray, mode: int = 0) -> np.ndarray:
        """R1: mode 0 inverse distance to cell centroids, mode 1 plain average."""
        phi = np.empty(self.c.n_verts)
        a = np.ascontiguousarray(alpha, np.float64)
        _lib().orc_vertex_field(self.ref, _p(self.geometry()["cell_cen"]), _p(a), mode, _p(phi))
        return phi

    def liquid_volume(self, cell: int, phi: np.ndarray, c: float, x0=None) -> dict:
        """R2 for one cell at isovalue c."""
        out = np.empty(9)
        x = None if x0 is None else np.ascontiguousarray(x0, np.float64)
        _lib().orc_liquid_volume(self.ref, int(cell), _p(phi), float(c), _p(x), _p(out))
        return dict(VL=out[0], area=out[1], vec_area=out[2:5].copy(), centroid=out[5:8].copy(), nloops=int(out[8]))

    def reconstruct(self, alpha, phi, eps=1e-12, tol=1e-12, max_iter=100, cells=None, method="bisect",
                    alpha_iso=0.5) -> dict:
        """R0 + R3 (+ geometry at the root). Arrays over all cells; untouched cells hold nan/0.
        method "bisect": bisection on V_L(c)/V - alpha; "cubic": bisection over the sorted vertex
        values, then the interval's cubic (interpolated from four evaluations) solved on its own;
        "fixed": the iso-surface at alpha_iso, no volume matching."""
        nc = self.c.n_cells
        a = np.ascontiguousarray(alpha, np.float64)
        r = dict(iso=np.full(nc, np.nan), status=np.zeros(nc, np.int32), evals=np.zeros(nc, np.int32),
                 A_int=np.zeros(nc), n_int=np.zeros((nc, 3)), x_gamma=np.zeros((nc, 3)),
                 nloops=np.zeros(nc, np.int32))
        cl = None if cells is None else np.ascontiguousarray(cells, np.int64)
        _lib().orc_reconstruct_m(self.ref, _p(a), _p(phi), _p(self.geometry()["cell_vol"]), eps, tol, max_iter,
                                 _p(cl), 0 if cl is None else len(cl), {"bisect": 0, "cubic": 1, "fixed": 2}[method],
                                 float(alpha_iso),
                                 *[_p(r[k]) for k in ("iso", "status", "evals", "A_int", "n_int", "x_gamma", "nloops")])
        return r

    def lsq_study(self, alpha, pc: dict, T, T_bnd, props: dict, variant: int) -> dict:
        """Appendix B's least squares on the band with the stencil-anisotropy study's variants (bits:
        1 standard stencil, 2 inverse-distance weights 1/|r|^2, 4 vertex neighbours), given a
        phase_change output `pc` (its crossing flags, x_f and band); returns grad, cond(G_P) and
        the singular flags (status)."""
        g = self.geometry()
        nc = self.c.n_cells
        o = dict(grad=np.zeros((nc, 3)), cond=np.zeros(nc), status=np.zeros(nc, np.int32))
        arr = lambda x: np.ascontiguousarray(x, np.float64)
        _lib().orc_lsq_study(self.ref, _p(g["face_cen"]), _p(g["cell_cen"]), _p(arr(alpha)), _p(arr(T)),
                             None if T_bnd is None else _p(arr(T_bnd)), float(props["T_sat"]),
                             _p(np.ascontiguousarray(pc["crossing"], np.uint8)), _p(arr(pc["x_f"])),
                             _p(np.ascontiguousarray(pc["in_band"], np.uint8)), int(variant),
                             _p(o["grad"]), _p(o["cond"]), _p(o["status"]))
        return o

    def extrap_dtau(self) -> float:
        """Pseudo-time step of Eq. (extrapolation): min over faces of |d_f|."""
        g = self.geometry()
        out = np.zeros(1)
        _lib().orc_extrap_dtau(self.ref, _p(g["cell_cen"]), _p(g["face_cen"]), _p(out))
        return float(out[0])

    def extrapolate(self, alpha, iface, n_int, grad, dtau=None, max_iter=120, tol=1e-3) -> dict:
        """The pseudo-time solve of Eq. (extrapolation) alone, on a given gradient field: the other
        side's gradient of every cell with iface != 0 (g_other), the six iteration counts (iters) and
        the no-side flags (status)."""
        g = self.geometry()
        nc = self.c.n_cells
        o = dict(g_other=np.zeros((nc, 3)), iters=np.zeros(6, np.int32), status=np.zeros(nc, np.int32))
        arr = lambda x: np.ascontiguousarray(x, np.float64)
        _lib().orc_extrapolate(self.ref, _p(g["face_area"]), _p(g["cell_vol"]), _p(arr(alpha)),
                               _p(np.ascontiguousarray(iface, np.uint8)), _p(arr(n_int)), _p(arr(grad)),
                               self.extrap_dtau() if dtau is None else float(dtau), int(max_iter), float(tol),
                               _p(o["g_other"]), _p(o["iters"]), _p(o["status"]))
        return o

    def phase_change(self, alpha, recon: dict, T, T_bnd, props: dict, eps=1e-12, xf_mode=XF_RECON,
                     extrap=None) -> dict:
        """R4-R8 given a reconstruction (oracle's own, or another one to be checked). `extrap`: None for
        R5's single upwind sweep, else a dict (max_iter, tol, dtau; dtau <= 0 or absent: the mesh's)
        for the pseudo-time solve of Eq. (extrapolation); its six iteration counts come back as
        `extrap_iters` (liquid x, y, z, vapour x, y, z)."""
        g = self.geometry()
        nc, nf = self.c.n_cells, self.c.n_faces
        o = dict(in_band=np.zeros(nc, np.uint8), grad=np.zeros((nc, 3)), grad_l=np.zeros((nc, 3)),
                 grad_v=np.zeros((nc, 3)), q_l=np.zeros(nc), q_v=np.zeros(nc), mdot=np.zeros(nc), Q=np.zeros(nc),
                 status=np.array(recon["status"], np.int32, copy=True), crossing=np.zeros(nf, np.uint8),
                 x_f=np.zeros((nf, 3)), d_own=np.zeros(nf), d_neigh=np.zeros(nf), A_int_f=np.zeros(nf),
                 totals=np.zeros(2))
        pr = _OrcProps(props["k_l"], props["k_v"], props["h_lv"], props["T_sat"])
        arr = lambda x: np.ascontiguousarray(x, np.float64)
        ex = None
        if extrap is not None:
            ex = _OrcExtrap(int(extrap.get("max_iter", 120)), float(extrap.get("tol", 1e-3)),
                            float(extrap.get("dtau", 0.0)))
        _lib().orc_phase_change(self.ref, _p(g["face_area"]), _p(g["face_cen"]), _p(g["cell_vol"]),
                                _p(g["cell_cen"]), _p(arr(alpha)), eps, _p(arr(recon["A_int"])),
                                _p(arr(recon["n_int"])), _p(arr(recon["x_gamma"])), _p(arr(T)),
                                None if T_bnd is None else _p(arr(T_bnd)), ctypes.byref(pr), xf_mode,
                                *[_p(o[k]) for k in ("in_band", "grad", "grad_l", "grad_v", "q_l", "q_v", "mdot", "Q",
                                                     "status", "crossing", "x_f", "d_own", "d_neigh", "A_int_f",
                                                     "totals")],
                                None if ex is None else ctypes.byref(ex))
        if ex is not None:
            o["extrap_iters"] = np.array(ex.iters[:], np.int32)
        o["a_own"], o["a_neigh"] = np.zeros(nf), np.zeros(nf)
        _lib().orc_interface_htc(self.ref, _p(arr(alpha)), _p(o["crossing"]), _p(o["A_int_f"]), _p(o["d_own"]),
                                 _p(o["d_neigh"]), props["k_l"], props["k_v"], _p(o["a_own"]), _p(o["a_neigh"]))
        # each cell's energy-matrix contributions of its detached faces: diagonal sum a_f, right-hand
        # side sum a_f T_sat
        o["htc_diag"], o["htc_rhs"] = np.zeros(nc), np.zeros(nc)
        _lib().orc_htc_cell_sums(self.ref, _p(o["crossing"]), _p(o["a_own"]), _p(o["a_neigh"]), float(props["T_sat"]),
                                 _p(o["htc_diag"]), _p(o["htc_rhs"]))
        return o

    def run(self, alpha, T, T_bnd, props, eps=1e-12, tol=1e-12, vertex_mode=0, xf_mode=XF_RECON) -> dict:
        """The whole path: R0-R8."""
        phi = self.vertex_field(alpha, vertex_mode)
        rec = self.reconstruct(alpha, phi, eps, tol)
        pc = self.phase_change(alpha, rec, T, T_bnd, props, eps, xf_mode)
        return dict(phi=phi, recon=rec, pc=pc)


def sym3_eigenvalues(A) -> np.ndarray:
    """Eigenvalues (ascending) of a symmetric 3x3 matrix by the oracle's Jacobi rotations."""
    out = np.zeros(3)
    _lib().orc_sym3_eigenvalues(_p(np.ascontiguousarray(A, np.float64).reshape(9)), _p(out))
    return out


def pairwise_sum(a: np.ndarray) -> float:
    out = np.zeros(1)
    x = np.ascontiguousarray(a, np.float64)
    _lib().orc_pairwise_sum(_p(x), len(x), _p(out))
    return float(out[0])
