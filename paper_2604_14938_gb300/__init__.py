"""GB300 (sm_103a) sharp-interface VOF phase-change hot path — Python binding.

Argument marshalling over the C ABI of ``libvof_gb300.so`` (include/vof.h): every step of the
path runs in the library's CUDA kernels; PyTorch supplies device memory and the stream. Each
tensor argument of the hot-path calls is checked before the call (float64, contiguous, on the
stated memory side, long enough for the mesh; ValueError otherwise). If the library is missing
this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvof_gb300.so")
_LIB = None

VOF_ST_DEGENERATE, VOF_ST_NOT_CONVERGED, VOF_ST_FALLBACK = 1, 2, 4
VOF_ST_SINGULAR_LSQ, VOF_ST_NO_SIDE, VOF_ST_MLP_SKIPPED = 8, 16, 32
XF_RECON, XF_LINEAR, XF_AS_PRINTED = 0, 1, 2
ROOT_BISECT, ROOT_LEARNED, ROOT_CUBIC, ROOT_FIXED = 0, 1, 2, 3

FIELDS = {
    "iface_idx": (0, np.int32, 1), "phi_v": (1, np.float64, 1), "iso": (2, np.float64, 1),
    "A_int": (3, np.float64, 1), "n_int": (4, np.float64, 3), "x_gamma": (5, np.float64, 3),
    "status": (6, np.int32, 1), "evals": (7, np.int32, 1), "grad": (8, np.float64, 3),
    "grad_l": (9, np.float64, 3), "grad_v": (10, np.float64, 3), "q_l": (11, np.float64, 1),
    "q_v": (12, np.float64, 1), "x_f": (13, np.float64, 3), "d_own": (14, np.float64, 1),
    "d_neigh": (15, np.float64, 1), "A_int_f": (16, np.float64, 1), "face_stamp": (17, np.int32, 1),
    "cell_vol": (18, np.float64, 1), "cell_cen": (19, np.float64, 3), "face_area": (20, np.float64, 3),
    "face_cen": (21, np.float64, 3), "iface_stamp": (22, np.int32, 1), "band_stamp": (23, np.int32, 1),
    "a_own": (24, np.float64, 1), "a_neigh": (25, np.float64, 1), "dtau": (26, np.float64, 1),
    "lsq_cond": (27, np.float64, 1), "htc_diag": (28, np.float64, 1), "htc_rhs": (29, np.float64, 1),
}


class VofError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("n_verts", ctypes.c_int64),
                ("cell_face_off", ctypes.c_void_p), ("cell_face", ctypes.c_void_p),
                ("face_vert_off", ctypes.c_void_p), ("face_vert", ctypes.c_void_p),
                ("face_owner", ctypes.c_void_p), ("face_neigh", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p)]


class Props(ctypes.Structure):
    _fields_ = [("k_l", ctypes.c_double), ("k_v", ctypes.c_double), ("h_lv", ctypes.c_double),
                ("T_sat", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("alpha_eps", ctypes.c_double), ("tol_alpha", ctypes.c_double), ("max_bisect", ctypes.c_int),
                ("root_mode", ctypes.c_int), ("max_secant", ctypes.c_int), ("xf_mode", ctypes.c_int),
                ("vertex_mode", ctypes.c_int), ("group_size", ctypes.c_int), ("htc", ctypes.c_int),
                ("alpha_iso", ctypes.c_double), ("extrap", ctypes.c_int), ("extrap_max_iter", ctypes.c_int),
                ("extrap_tol", ctypes.c_double), ("lsq_variant", ctypes.c_int), ("guess", ctypes.c_int),
                ("extrap_poll_limit", ctypes.c_int), ("root_narrow", ctypes.c_double)]


class Counts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("step", "n_iface", "n_band", "n_crossing", "n_degenerate",
                                               "n_not_converged", "n_fallback", "n_singular", "n_no_side",
                                               "n_mlp_skipped", "evals_total", "tet_evals", "tets_prepared",
                                               "tets_sectioned", "evals32_total")] + [
        ("extrap_iters", ctypes.c_int64 * 6)]


def lib():
    """The loaded library; raises VofError when it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise VofError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, st = ctypes.c_void_p, ctypes.c_int
        sig = {
            "vof_mesh_create": [vp, vp, vp], "vof_mesh_destroy": [vp], "vof_reconstruct": [vp, vp, vp, vp],
            "vof_phase_change_source": [vp] * 10, "vof_step": [vp] * 10, "vof_step_host": [vp] * 9,
            "vof_field_size": [vp, ctypes.c_int, vp, vp], "vof_copy_field": [vp, ctypes.c_int, vp, ctypes.c_int64, vp],
            "vof_get_counts": [vp, vp, vp], "vof_mesh_info": [vp, vp], "vof_mesh_bins": [vp, vp],
            "vof_timing_enable": [vp, ctypes.c_int], "vof_timing_read": [vp, vp, vp, ctypes.c_int, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = st
        L.vof_last_error.restype = ctypes.c_char_p
        L.vof_default_options.argtypes = [vp]
        L.vof_default_options.restype = None
        _LIB = L
    return _LIB


def _check(status: int, what: str):
    if status != 0:
        raise VofError(f"{what} failed with status {status}: {lib().vof_last_error().decode()}")


def default_options(**kw) -> Options:
    o = Options()
    lib().vof_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def props_of(d: dict) -> Props:
    return Props(d["k_l"], d["k_v"], d["h_lv"], d["T_sat"])


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _arg(t, n: int, name: str, what: str, cuda: bool = True, optional: bool = False):
    """The address of a float64 tensor argument, after the checks the C ABI cannot make on a bare
    pointer: a contiguous torch tensor of dtype float64 with at least n elements, in CUDA device
    memory (cuda=True) or in host memory (cuda=False). None passes as NULL where the argument is
    optional. A wrong argument raises ValueError before any call into the library, where it would
    otherwise be read or written out of bounds."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{what}: {name} is required")
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{what}: {name} must be a torch tensor, not {type(t).__name__}")
    if t.dtype != torch.float64:
        raise ValueError(f"{what}: {name} must be float64, not {t.dtype}")
    if bool(t.is_cuda) != cuda:
        raise ValueError(f"{what}: {name} must be in {'CUDA device' if cuda else 'host'} memory")
    if not t.is_contiguous():
        raise ValueError(f"{what}: {name} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{what}: {name} holds {t.numel()} values, {n} needed")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """A mesh uploaded to the GPU (library-owned). `m` is any object with the primitive arrays
    of the mesh format (vx, vy, vz, face_vert_off, face_vert, face_owner, face_neigh,
    cell_face_off, cell_face)."""

    def __init__(self, m, stream=None):
        keep = [np.ascontiguousarray(a, dt) for a, dt in (
            (m.cell_face_off, np.int64), (m.cell_face, np.int32), (m.face_vert_off, np.int64),
            (m.face_vert, np.int32), (m.face_owner, np.int32), (m.face_neigh, np.int32),
            (m.vx, np.float64), (m.vy, np.float64), (m.vz, np.float64))]
        d = _Desc(len(keep[0]) - 1, len(keep[4]), len(keep[6]), *[a.ctypes.data for a in keep])
        h = ctypes.c_void_p()
        _check(lib().vof_mesh_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)), "vof_mesh_create")
        self.h = h
        info = (ctypes.c_int64 * 5)()
        _check(lib().vof_mesh_info(h, info), "vof_mesh_info")
        self.n_cells, self.n_faces, self.n_verts, self.max_cell_verts, self.max_cell_tets = list(info)
        bins = (ctypes.c_int64 * 5)()
        _check(lib().vof_mesh_bins(h, bins), "vof_mesh_bins")
        self.bin_cells = list(bins)

    def close(self):
        if getattr(self, "h", None) and not getattr(self, "_owned_by_batch", False):
            lib().vof_mesh_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the hot path
    def reconstruct(self, alpha, opt: Options | None = None, stream=None):
        """vof_reconstruct: alpha is a CUDA float64 tensor [n_cells]."""
        o = opt or default_options()
        pa = _arg(alpha, self.n_cells, "alpha", "vof_reconstruct")
        _check(lib().vof_reconstruct(self.h, pa, ctypes.byref(o), _stream(stream)), "vof_reconstruct")

    def phase_change_source(self, alpha, T, T_bnd, props: dict, mdot, Q, totals, opt: Options | None = None,
                            stream=None):
        """vof_phase_change_source: all tensors CUDA float64 (T_bnd may be None)."""
        o = opt or default_options()
        p = props_of(props)
        a = self._step_args("vof_phase_change_source", alpha, T, T_bnd, mdot, Q, totals)
        _check(lib().vof_phase_change_source(self.h, a[0], a[1], a[2], ctypes.byref(p), ctypes.byref(o), a[3], a[4],
                                             a[5], _stream(stream)), "vof_phase_change_source")

    def step(self, alpha, T, T_bnd, props: dict, mdot, Q, totals, opt: Options | None = None, stream=None):
        """vof_step: reconstruct + phase-change source in one call."""
        o = opt or default_options()
        p = props_of(props)
        a = self._step_args("vof_step", alpha, T, T_bnd, mdot, Q, totals)
        _check(lib().vof_step(self.h, a[0], a[1], a[2], ctypes.byref(p), ctypes.byref(o), a[3], a[4], a[5],
                              _stream(stream)), "vof_step")

    def step_host(self, h_alpha, h_T, h_T_bnd, props: dict, h_mdot, h_totals, opt: Options | None = None,
                  stream=None):
        """vof_step_host: host tensors (pinned for asynchronous copies); synchronises."""
        o = opt or default_options()
        p = props_of(props)
        w = "vof_step_host"
        nc, nf = self.n_cells, self.n_faces
        a = (_arg(h_alpha, nc, "h_alpha", w, cuda=False), _arg(h_T, nc, "h_T", w, cuda=False),
             _arg(h_T_bnd, nf, "h_T_bnd", w, cuda=False, optional=True), _arg(h_mdot, nc, "h_mdot", w, cuda=False),
             _arg(h_totals, 2, "h_totals", w, cuda=False))
        _check(lib().vof_step_host(self.h, a[0], a[1], a[2], ctypes.byref(p), ctypes.byref(o), a[3], a[4],
                                   _stream(stream)), w)

    def _step_args(self, what, alpha, T, T_bnd, mdot, Q, totals):
        """Checked device addresses of a step's tensors: alpha, T, mdot, Q [n_cells], T_bnd
        [n_faces] or None, totals [2]."""
        nc, nf = self.n_cells, self.n_faces
        return (_arg(alpha, nc, "alpha", what), _arg(T, nc, "T", what), _arg(T_bnd, nf, "T_bnd", what, optional=True),
                _arg(mdot, nc, "mdot", what), _arg(Q, nc, "Q", what), _arg(totals, 2, "totals", what))

    # ---- results
    def field(self, name: str, stream=None):
        """A copy of a workspace field as a CUDA tensor."""
        import torch
        fid, dt, width = FIELDS[name]
        cnt, eb = ctypes.c_int64(), ctypes.c_int()
        _check(lib().vof_field_size(self.h, fid, ctypes.byref(cnt), ctypes.byref(eb)), "vof_field_size")
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dt]
        out = torch.empty(cnt.value, dtype=tdt, device="cuda")
        _check(lib().vof_copy_field(self.h, fid, _ptr(out), cnt.value, _stream(stream)), "vof_copy_field")
        return out.view(-1, width) if width > 1 else out

    KERNEL_CLASSES = ("select", "mlp_features", "root", "xmark", "xface", "lsq", "mlp_forward", "geom", "extrap",
                      "source", "htc")

    def timing_enable(self, on: bool = True):
        _check(lib().vof_timing_enable(self.h, int(on)), "vof_timing_enable")

    def timing_read(self, stream=None) -> dict:
        """{kernel class: (milliseconds summed, launches)} since the last read (synchronises)."""
        n = len(self.KERNEL_CLASSES)
        ms, nl = (ctypes.c_double * n)(), (ctypes.c_int64 * n)()
        _check(lib().vof_timing_read(self.h, ms, nl, n, _stream(stream)), "vof_timing_read")
        return {k: (ms[i], nl[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    # FP64 flops per unit of the root search's algorithmic work (see the kernel header):
    # one tetrahedron evaluation = x = ref - c, three FMAs, one add (8 flops); preparing one
    # tetrahedron = 6 differences, 12 products, 3 divisions, 3 sums (24); cutting one in the
    # final geometry = 3-4 edge cuts, cross products, norms and moments (60); 2 per evaluation.
    FLOPS_TET_EVAL, FLOPS_TET_PREP, FLOPS_TET_SECTION, FLOPS_EVAL = 8, 24, 60, 2

    def root_flops(self, counts: dict) -> int:
        """Algorithmic FP64 flops of the root-search launches summed in `counts`: rows prepared,
        tetrahedron evaluations and per-evaluation scaling."""
        return (self.FLOPS_TET_EVAL * counts["tet_evals"] + self.FLOPS_TET_PREP * counts["tets_prepared"]
                + self.FLOPS_EVAL * counts["evals_total"])

    def geom_flops(self, counts: dict) -> int:
        """Algorithmic flops of the interface-geometry launches in `counts` (the sections of the cut
        tetrahedra; the kernel runs them in FP32 pair arithmetic)."""
        return self.FLOPS_TET_SECTION * counts["tets_sectioned"]

    def counts(self, stream=None) -> dict:
        c = Counts()
        _check(lib().vof_get_counts(self.h, ctypes.byref(c), _stream(stream)), "vof_get_counts")
        out = {n: getattr(c, n) for n, _ in Counts._fields_}
        out["extrap_iters"] = list(c.extrap_iters)
        return out


def fp64_peak(iters: int = 20000, reps: int = 3, stream=None) -> dict:
    """vof_probe_fp64_fma: the FP64 FMA rate of the current device (TFLOP/s), the best of `reps`
    timed launches of independent FMA chains at full occupancy."""
    L = lib()
    f = L.vof_probe_fp64_fma
    f.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    ms, fl = ctypes.c_double(), ctypes.c_double()
    _check(f(iters, reps, ctypes.byref(ms), ctypes.byref(fl), _stream(stream)), "vof_probe_fp64_fma")
    return {"tflops": fl.value / (ms.value * 1e-3) / 1e12, "ms": ms.value, "flops": fl.value}


# ---------------------------------------------------------------------------------- learned guess
N_MLP_PARAMS = 11009
N_MLP_FEATURES = 40
MLP_PATH = os.path.join(_HERE, "mlp_iso.npy")


def _mlp_sig():
    L = lib()
    if getattr(L, "_mlp_sig", False):
        return L
    vp, st = ctypes.c_void_p, ctypes.c_int
    for name, args in {"vof_mlp_create": [vp, vp], "vof_mlp_destroy": [vp], "vof_mlp_get_params": [vp, vp],
                       "vof_mlp_forward": [vp, vp, ctypes.c_int64, vp, vp],
                       "vof_mlp_train_step": [vp, vp, vp, ctypes.c_int64, ctypes.c_float, vp, vp],
                       "vof_mlp_grad": [vp, vp, vp, ctypes.c_int64, vp, vp, vp],
                       "vof_mesh_set_mlp": [vp, vp], "vof_mlp_features": [vp, vp, vp, vp, vp]}.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L._mlp_sig = True
    return L


class Mlp:
    """The isovalue-guess MLP on the device (vof_mlp_*). Parameters: float32 [N_MLP_PARAMS]."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, np.float32)
        if p.shape != (N_MLP_PARAMS,):
            raise ValueError(f"expected {N_MLP_PARAMS} parameters")
        h = ctypes.c_void_p()
        _check(_mlp_sig().vof_mlp_create(p.ctypes.data, ctypes.byref(h)), "vof_mlp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _mlp_sig().vof_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(N_MLP_PARAMS, np.float32)
        _check(_mlp_sig().vof_mlp_get_params(self.h, out.ctypes.data), "vof_mlp_get_params")
        return out

    def forward(self, X, y=None, stream=None):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device) if y is None else y
        _check(_mlp_sig().vof_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(y), _stream(stream)), "vof_mlp_forward")
        return y

    def train_step(self, X, t, lr: float, loss=None, stream=None):
        _check(_mlp_sig().vof_mlp_train_step(self.h, _ptr(X), _ptr(t), X.shape[0], ctypes.c_float(lr), _ptr(loss),
                                             _stream(stream)), "vof_mlp_train_step")

    def grad(self, X, t, stream=None):
        import torch
        g = torch.empty(N_MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(_mlp_sig().vof_mlp_grad(self.h, _ptr(X), _ptr(t), X.shape[0], _ptr(g), _ptr(loss), _stream(stream)),
               "vof_mlp_grad")
        return g, loss


def _mesh_set_mlp(self, mlp):
    """Attaches an Mlp (kept alive by the mesh) for ROOT_LEARNED; None detaches."""
    _check(_mlp_sig().vof_mesh_set_mlp(self.h, None if mlp is None else mlp.h), "vof_mesh_set_mlp")
    self._mlp = mlp


def _mesh_mlp_features(self, alpha, stream=None):
    """(features [n_iface, 40] float32, ok [n_iface] int32) of the last reconstruction, which was
    made with the CUDA float64 tensor `alpha`."""
    import torch
    pa = _arg(alpha, self.n_cells, "alpha", "vof_mlp_features")
    n = self.counts()["n_iface"]
    X = torch.empty((max(n, 1), N_MLP_FEATURES), dtype=torch.float32, device="cuda")
    ok = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    _check(_mlp_sig().vof_mlp_features(self.h, pa, _ptr(X), _ptr(ok), _stream(stream)), "vof_mlp_features")
    return X[:n], ok[:n]


Mesh.set_mlp = _mesh_set_mlp
Mesh.mlp_features = _mesh_mlp_features


def load_default_mlp(mesh: Mesh) -> bool:
    """Attaches the trained weights shipped with the package (mlp_iso.npy) to `mesh`; False if
    there are none."""
    if not os.path.exists(MLP_PATH):
        return False
    mesh.set_mlp(Mlp(np.load(MLP_PATH)))
    return True


# ------------------------------------------------------------------- graphs, autotuning, batches
def _ext_sig():
    L = lib()
    if getattr(L, "_ext_sig", False):
        return L
    vp, st = ctypes.c_void_p, ctypes.c_int
    for name, args in {"vof_step_graph": [vp] * 10, "vof_autotune": [vp, vp, vp, ctypes.c_int, vp, vp],
                       "vof_set_group_sizes": [vp, vp], "vof_batch_create": [vp, ctypes.c_int, vp, vp],
                       "vof_batch_destroy": [vp], "vof_batch_mesh": [vp, vp], "vof_batch_offsets": [vp, vp, vp, vp],
                       "vof_batch_totals": [vp, vp, vp]}.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L._ext_sig = True
    return L


def _mesh_step_graph(self, alpha, T, T_bnd, props: dict, mdot, Q, totals, opt: Options | None = None, stream=None):
    """vof_step_graph: the step captured once into a CUDA graph and replayed (non-default stream)."""
    o = opt or default_options()
    p = props_of(props)
    a = self._step_args("vof_step_graph", alpha, T, T_bnd, mdot, Q, totals)
    _check(_ext_sig().vof_step_graph(self.h, a[0], a[1], a[2], ctypes.byref(p), ctypes.byref(o), a[3], a[4], a[5],
                                     _stream(stream)), "vof_step_graph")


def _mesh_autotune(self, alpha, opt: Options | None = None, reps: int = 5, stream=None) -> list:
    """vof_autotune: lanes per cell of every tetrahedron-count bin, timed on `alpha`."""
    o = opt or default_options()
    G = (ctypes.c_int * 5)()
    pa = _arg(alpha, self.n_cells, "alpha", "vof_autotune")
    _check(_ext_sig().vof_autotune(self.h, pa, ctypes.byref(o), reps, G, _stream(stream)), "vof_autotune")
    return list(G)


def _mesh_set_group_sizes(self, G):
    arr = (ctypes.c_int * 5)(*G)
    _check(_ext_sig().vof_set_group_sizes(self.h, arr), "vof_set_group_sizes")


Mesh.step_graph = _mesh_step_graph
Mesh.autotune = _mesh_autotune
Mesh.set_group_sizes = _mesh_set_group_sizes


class Batch:
    """Disjoint union of meshes stepped as one mesh (vof_batch_*); `mesh` is the union Mesh."""

    def __init__(self, meshes, stream=None):
        keeps, descs = [], (_Desc * len(meshes))()
        for i, m in enumerate(meshes):
            keep = [np.ascontiguousarray(a, dt) for a, dt in (
                (m.cell_face_off, np.int64), (m.cell_face, np.int32), (m.face_vert_off, np.int64),
                (m.face_vert, np.int32), (m.face_owner, np.int32), (m.face_neigh, np.int32),
                (m.vx, np.float64), (m.vy, np.float64), (m.vz, np.float64))]
            keeps.append(keep)
            descs[i] = _Desc(len(keep[0]) - 1, len(keep[4]), len(keep[6]), *[a.ctypes.data for a in keep])
        h = ctypes.c_void_p()
        _check(_ext_sig().vof_batch_create(descs, len(meshes), _stream(stream), ctypes.byref(h)), "vof_batch_create")
        self.h = h
        self.n = len(meshes)
        mh = ctypes.c_void_p()
        _check(_ext_sig().vof_batch_mesh(h, ctypes.byref(mh)), "vof_batch_mesh")
        self.mesh = Mesh.__new__(Mesh)
        self.mesh.h = mh
        self.mesh._owned_by_batch = True
        info = (ctypes.c_int64 * 5)()
        _check(lib().vof_mesh_info(mh, info), "vof_mesh_info")
        (self.mesh.n_cells, self.mesh.n_faces, self.mesh.n_verts, self.mesh.max_cell_verts,
         self.mesh.max_cell_tets) = list(info)
        bins = (ctypes.c_int64 * 5)()
        _check(lib().vof_mesh_bins(mh, bins), "vof_mesh_bins")
        self.mesh.bin_cells = list(bins)
        self.cell_off = np.zeros(self.n + 1, np.int64)
        self.face_off = np.zeros(self.n + 1, np.int64)
        self.vert_off = np.zeros(self.n + 1, np.int64)
        _check(_ext_sig().vof_batch_offsets(h, self.cell_off.ctypes.data, self.face_off.ctypes.data,
                                            self.vert_off.ctypes.data), "vof_batch_offsets")

    def totals(self, out=None, stream=None):
        """Per-mesh totals [n, 2] of the last step."""
        import torch
        out = torch.empty((self.n, 2), dtype=torch.float64, device="cuda") if out is None else out
        _check(_ext_sig().vof_batch_totals(self.h, _ptr(out), _stream(stream)), "vof_batch_totals")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.mesh.h = None
            _ext_sig().vof_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
