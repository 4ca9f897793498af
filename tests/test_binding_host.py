"""The binding's argument checks, which need no GPU: a tensor of the wrong dtype, memory side
(host or CUDA device), layout or length raises ValueError before any call into the library,
where the kernels would read or write it out of bounds; valid tensors reach the library."""
import types

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vof():
    from paper_2604_14938_gb300 import build as b
    b.build()
    import paper_2604_14938_gb300 as p
    return p


def _mesh(vof, nc=10, nf=30):
    """A Mesh object with sizes but no device mesh (handle NULL): enough for the checks."""
    M = vof.Mesh.__new__(vof.Mesh)
    M.h = None
    M.n_cells, M.n_faces = nc, nf
    return M


def _f64(n):
    return torch.zeros(n, dtype=torch.float64)


def test_arg_passes_a_contiguous_float64_tensor_of_enough_length(vof):
    t = _f64(12)
    assert vof._arg(t, 10, "alpha", "call", cuda=False).value == t.data_ptr()
    v = _f64(20)[4:14]  # a contiguous view: its own address, offset included
    assert vof._arg(v, 10, "alpha", "call", cuda=False).value == v.data_ptr()
    assert vof._arg(None, 10, "T_bnd", "call", optional=True) is None


@pytest.mark.parametrize("bad, n, cuda, optional, msg", [
    (None, 10, True, False, "is required"),
    ([0.0] * 10, 10, False, False, "torch tensor"),
    (torch.zeros(10, dtype=torch.float32), 10, False, False, "float64"),
    (torch.zeros(9, dtype=torch.float64), 10, False, False, "9 values, 10 needed"),
    (torch.zeros(20, dtype=torch.float64)[::2], 10, False, False, "contiguous"),
    (torch.zeros(10, dtype=torch.float64), 10, True, False, "CUDA device"),
])
def test_arg_rejects(vof, bad, n, cuda, optional, msg):
    with pytest.raises(ValueError, match=msg):
        vof._arg(bad, n, "x", "call", cuda=cuda, optional=optional)


def test_device_calls_reject_host_tensors_before_the_library(vof):
    M = _mesh(vof)
    nc, nf = M.n_cells, M.n_faces
    a, T, Tb, mdot, Q, tot = _f64(nc), _f64(nc), _f64(nf), _f64(nc), _f64(nc), _f64(2)
    props = dict(T_sat=373.15, k_l=0.68, k_v=0.025, h_lv=2.26e6)
    calls = {
        "vof_reconstruct": lambda: M.reconstruct(a),
        "vof_step": lambda: M.step(a, T, Tb, props, mdot, Q, tot),
        "vof_phase_change_source": lambda: M.phase_change_source(a, T, Tb, props, mdot, Q, tot),
        "vof_step_graph": lambda: M.step_graph(a, T, Tb, props, mdot, Q, tot),
        "vof_autotune": lambda: M.autotune(a),
        "vof_mlp_features": lambda: M.mlp_features(a),
    }
    for what, call in calls.items():
        with pytest.raises(ValueError, match=f"{what}: alpha must be in CUDA device memory"):
            call()


def test_host_step_checks_each_buffer(vof):
    M = _mesh(vof)
    nc, nf = M.n_cells, M.n_faces
    props = dict(T_sat=373.15, k_l=0.68, k_v=0.025, h_lv=2.26e6)
    good = dict(h_alpha=_f64(nc), h_T=_f64(nc), h_T_bnd=_f64(nf), h_mdot=_f64(nc), h_totals=_f64(2))
    for name, bad in (("h_alpha", _f64(nc - 1)), ("h_T", torch.zeros(nc, dtype=torch.float32)),
                      ("h_T_bnd", _f64(nf - 1)), ("h_mdot", _f64(2 * nc)[::2]), ("h_totals", _f64(1))):
        args = dict(good, **{name: bad})
        with pytest.raises(ValueError, match=f"vof_step_host: {name}"):
            M.step_host(args["h_alpha"], args["h_T"], args["h_T_bnd"], props, args["h_mdot"], args["h_totals"])
    # valid buffers pass the checks and reach the library, which refuses the missing device mesh
    # (a stand-in stream object: the default stream's handle, no CUDA call)
    s0 = types.SimpleNamespace(cuda_stream=0)
    for tb in (good["h_T_bnd"], None):
        with pytest.raises(vof.VofError, match="null argument"):
            M.step_host(good["h_alpha"], good["h_T"], tb, props, good["h_mdot"], good["h_totals"], stream=s0)
