"""The allocation-free totals entry point (vof_totals_static) against the totals of the regular
step, through the C ABI, on two calls in a row. Callers that cannot allocate device memory (stream
capture, real-time loops, hosts with their own pool) use it; it keeps its scratch in a file-scope
device array. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from gpu_helpers import case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _lib():
    import paper_2604_14938_gb300 as vof
    L = vof.lib()
    L.vof_totals_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    L.vof_totals_static.restype = ctypes.c_int
    return vof, L


def _step_products(name):
    import synth
    vof, _ = _lib()
    m, a, T, Tb = case(name)
    M = vof.Mesh(m)
    d = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    mdot = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(mdot)
    tot = torch.empty(2, dtype=torch.float64, device="cuda")
    M.step(d(a), d(T), d(Tb), synth.PROPS, mdot, Q, tot)
    idx = M.field("iface_idx").long()
    vol = M.field("cell_vol")
    return (mdot[idx] * vol[idx]).contiguous(), (Q[idx] * vol[idx]).contiguous(), tot


def test_static_totals_match_step_totals_twice():
    """Both entry points sum the same pairwise tree (zero-padded to a power of two), so the totals
    agree bit for bit; two calls in a row with different sizes."""
    vof, L = _lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for name in ("voronoi_film", "hex_sphere"):  # two calls in a row, different sizes
        mv, qv, tot = _step_products(name)
        out.fill_(float("nan"))
        st = L.vof_totals_static(mv.data_ptr(), qv.data_ptr(), mv.numel(), out.data_ptr(), stream)
        assert st == 0, L.vof_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), tot.cpu().numpy())


@pytest.mark.parametrize("n", [0, 1, 2049, 3_141_593, 4_194_304])
def test_static_totals_sizes_against_the_tree(n):
    """Seeded values at the edges of the size range (empty, one value, one past a chunk, many
    chunks over the grid-stride loop, the maximum) against the pairwise tree summed on the host
    (the oracle's), bit for bit, on two calls in a row."""
    import oracle
    vof, L = _lib()
    rng = np.random.default_rng(n)
    a = rng.normal(size=n) * np.exp(rng.uniform(-20, 20, size=n))
    b = rng.uniform(-1, 1, size=n)
    da = torch.as_tensor(a, device="cuda") if n else torch.zeros(1, dtype=torch.float64, device="cuda")
    db = torch.as_tensor(b, device="cuda") if n else torch.zeros(1, dtype=torch.float64, device="cuda")
    want = np.array([oracle.pairwise_sum(a), oracle.pairwise_sum(b)])
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(float("nan"))
        assert L.vof_totals_static(da.data_ptr(), db.data_ptr(), n, out.data_ptr(), stream) == 0, L.vof_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)


def test_static_totals_reject_oversize():
    vof, L = _lib()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = L.vof_totals_static(x.data_ptr(), x.data_ptr(), 4194304 + 1, out.data_ptr(), None)
    assert st == 1
    assert b"VOF_TOTALS_STATIC_MAX_N" in L.vof_last_error()
