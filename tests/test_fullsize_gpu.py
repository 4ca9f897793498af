"""Parity at the full sizes of the benchmark workloads, in the launch configuration that bench.py
times: lanes per cell autotuned on the live field, the learned root search, CUDA graph replay
(eager steps with a new input every step for the moving pipe film, the 64-mesh union for the
batch).

The oracle runs over the whole mesh where that is cheap (vertex field, cell geometry, and the
downstream steps given the GPU reconstruction) and one cell at a time on a seeded sample of the
interface cells (cut volume and interface geometry at the GPU isovalue). Bars as in the small
parity tests: |V_L/V - alpha| <= 1e-10, index outputs bit-exact, totals to 1e-10; with the
oracle starting from the GPU reconstruction, relative 1e-8 on gradients (in the Euclidean norm),
heat rates, mdot and Q, except where the oracle's own answer moves by more than 1e-10 under
one-ulp rounding of the cell centroids: there the allowance is 100 times that movement."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import EPS, ulp_spread, within
from synth.workloads import workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14938_gb300 as vof  # noqa: E402

SAMPLE = 300
KEYS = ("iface_idx", "phi_v", "iso", "A_int", "n_int", "x_gamma", "status", "evals", "grad", "grad_l",
        "grad_v", "q_l", "q_v", "band_stamp", "face_stamp")


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _run(M, a, T, Tb, n_cells, mode, graph, batch=None, tune=True, **kw):
    """Autotune for `mode` (unless tune is False), then one step as the benchmark takes it; numpy
    outputs."""
    opt = vof.default_options(root_mode=mode, **kw)
    s = torch.cuda.Stream()  # graph capture needs a stream of its own
    with torch.cuda.stream(s):
        ta, tT = _dev(a), _dev(T)
        tTb = None if Tb is None else _dev(Tb)
        if tune:
            M.autotune(ta, opt, reps=3, stream=s)
        mdot = torch.empty(n_cells, dtype=torch.float64, device="cuda")
        Q = torch.empty_like(mdot)
        tot = torch.empty(2, dtype=torch.float64, device="cuda")
        if graph:
            M.step_graph(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt, stream=s)
        else:
            M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt, stream=s)
        s.synchronize()
        g = {k: M.field(k, stream=s).cpu().numpy() for k in KEYS}
        g.update(mdot=mdot.cpu().numpy(), Q=Q.cpu().numpy(), totals=tot.cpu().numpy(), counts=M.counts(stream=s))
        if batch is not None:
            g["batch_totals"] = batch.totals(stream=s).cpu().numpy()
    torch.cuda.synchronize()
    return g


def cell_vertices(m, cells):
    """Unique vertices of the given cells (vectorised CSR walk)."""
    def expand(off, vals, rows):
        lo, hi = off[rows], off[rows + 1]
        n = hi - lo
        start = np.repeat(lo - np.concatenate(([0], np.cumsum(n)[:-1])), n)
        return vals[start + np.arange(n.sum())]
    faces = expand(np.asarray(m.cell_face_off), np.asarray(m.cell_face), np.asarray(cells)) & 0x7FFFFFFF
    return np.unique(expand(np.asarray(m.face_vert_off), np.asarray(m.face_vert), faces))


def sample_cells(m, a, I, rng):
    """A seeded sample of interface cells, with the most-faceted cells and the alpha extremes."""
    nf = np.diff(np.asarray(m.cell_face_off))[I]
    pick = [rng.choice(I, min(SAMPLE, len(I)), replace=False), I[np.argsort(-nf, kind="stable")[:20]],
            I[np.argsort(a[I], kind="stable")[:10]], I[np.argsort(-a[I], kind="stable")[:10]]]
    return np.unique(np.concatenate(pick))


def check_mesh(m, a, T, Tb, g, rng, cells=None):
    """Every check on one mesh; `g` holds that mesh's slice of the GPU outputs."""
    I = np.where((a > EPS) & (a < 1 - EPS))[0]
    assert np.array_equal(g["iface_idx"], I)
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    # a1 vertex field on every vertex of the interface cells. Its conditioning sets the bar: the
    # two sides round the cell centroids independently (an ulp of a unit coordinate is 1.1e-16),
    # and over a vertex-centroid distance of h/2 that moves an inverse-distance weight by about
    # 2e-16/h relative, 2e-14 at h = 0.01; 1e-12 leaves room for cells ten times closer.
    vs = cell_vertices(m, I)
    np.testing.assert_allclose(g["phi_v"][vs], O.vertex_field(a)[vs], rtol=0, atol=1e-12)
    # a2/a3 on the sample, one cell at a time
    worst = 0.0
    for c in sample_cells(m, a, I, rng) if cells is None else cells:
        assert not g["status"][c] & 1, c
        geo = O.liquid_volume(int(c), g["phi_v"], g["iso"][c])
        worst = max(worst, abs(geo["VL"] / V[c] - a[c]))
        h = V[c] ** (1 / 3)
        assert geo["area"] == pytest.approx(g["A_int"][c], rel=1e-9, abs=1e-13 * h * h)
        vn = np.linalg.norm(geo["vec_area"])
        if vn > 1e-9 * geo["area"]:
            np.testing.assert_allclose(g["n_int"][c], -geo["vec_area"] / vn, atol=1e-8)
        if geo["area"] > 0:
            np.testing.assert_allclose(g["x_gamma"][c], geo["centroid"], atol=1e-9 * h)
    assert worst <= 1e-10, worst
    # a4-a7 over the whole mesh, the oracle starting from the GPU reconstruction. Bar: relative
    # 1e-8 (vectors in the Euclidean norm), widened to 100 times the oracle's own change under
    # one-ulp centroid rounding where the modified stencil is ill-conditioned (crossing points
    # within a fraction of a percent of h of the centroid on several faces).
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    keys = ("grad", "grad_l", "grad_v", "q_l", "q_v", "mdot", "Q")
    pc, spread = ulp_spread(O, a, rec, T, Tb, synth.PROPS, keys)
    band = pc["in_band"].astype(bool)
    assert np.array_equal(g["band_stamp"] == g["step"], band)
    for k in keys:
        sel = band if k == "grad" else I
        ok, worst = within(g[k][sel], pc[k][sel], spread[k][sel])
        assert ok, (k, worst)
    outside = np.ones(len(a), bool)
    outside[I] = False
    assert not np.any(g["mdot"][outside])
    return pc["totals"]


@pytest.fixture(scope="module", params=["film250k", "voronoi2m", "pipe8m"])
def full(request):
    m, a, T, Tb, _, extra = workload(request.param)
    M = vof.Mesh(m)
    assert vof.load_default_mlp(M)
    if request.param == "pipe8m":
        # the benchmark's second step: the film moved by one layer, T_bnd not passed
        n2d = m.n_cells // extra["layers"]
        _run(M, a, T, None, m.n_cells, vof.ROOT_LEARNED, graph=False)
        a, T, Tb = np.roll(a, n2d), np.roll(T, n2d), None
        g = _run(M, a, T, Tb, m.n_cells, vof.ROOT_LEARNED, graph=False)
    else:
        g = _run(M, a, T, Tb, m.n_cells, vof.ROOT_LEARNED, graph=True)
    g["step"] = g["counts"]["step"]
    return request.param, m, a, T, Tb, g, M


def test_full_size_parity(full):
    name, m, a, T, Tb, g, M = full
    tot = check_mesh(m, a, T, Tb, g, np.random.default_rng(7))
    np.testing.assert_allclose(g["totals"], tot, rtol=1e-10)
    c = g["counts"]
    assert c["n_not_converged"] == 0
    assert c["n_iface"] == len(g["iface_idx"])


@pytest.mark.parametrize("mode", ["bisect", "cubic"])
def test_full_size_other_root_modes(full, mode):
    """The FP64 bisection path and the interval-cubic path on the same mesh meet every bar; on
    these Voronoi workloads the learned guess cuts bisection's FP64 evaluations per cell several
    fold, and the interval cubic needs about one FP64 pass per cell."""
    name, m, a, T, Tb, g, M = full
    if name == "pipe8m":
        pytest.skip("the moving film is timed with the learned path only")
    gb = _run(M, a, T, Tb, m.n_cells, vof.ROOT_BISECT if mode == "bisect" else vof.ROOT_CUBIC, graph=True)
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    I = gb["iface_idx"]
    for c in sample_cells(m, a, I, np.random.default_rng(11)):
        assert abs(O.liquid_volume(int(c), gb["phi_v"], gb["iso"][c])["VL"] / V[c] - a[c]) <= 1e-10
    assert gb["counts"]["n_not_converged"] == 0
    gb["step"] = gb["counts"]["step"]
    check_mesh(m, a, T, Tb, gb, np.random.default_rng(13))
    per_cell = lambda x: x["counts"]["evals_total"] / len(I)
    if mode == "bisect":
        assert per_cell(g) * 5 < per_cell(gb), (per_cell(g), per_cell(gb))
    else:
        assert per_cell(gb) <= 1.5, per_cell(gb)


@pytest.mark.parametrize("G", [1, 2])
def test_full_size_lanes_that_do_not_fit_the_mode(full, G):
    """Lanes per cell chosen for one root mode can be too few for another: plain bisection keeps FP64
    rows, twice the shared memory of the learned path's FP32 rows, and the 2M case's largest cells
    (the 65-192 tetrahedra bin) do not fit one or two lanes per cell in a block. The step then
    takes the next lane count that fits, instead of failing the launch, and meets the bar."""
    name, m, a, T, Tb, g, M = full
    if name != "voronoi2m":
        pytest.skip("the 2M case holds the largest cells")
    M.set_group_sizes([G] * 5)
    gb = _run(M, a, T, Tb, m.n_cells, vof.ROOT_BISECT, graph=False, tune=False)
    O = oracle.Oracle(m)
    V = O.geometry()["cell_vol"]
    I = gb["iface_idx"]
    assert len(I) == len(g["iface_idx"])
    for c in sample_cells(m, a, I, np.random.default_rng(17)):
        assert abs(O.liquid_volume(int(c), gb["phi_v"], gb["iso"][c])["VL"] / V[c] - a[c]) <= 1e-10
    assert gb["counts"]["n_not_converged"] == 0


def test_full_size_extrapolation(full):
    """The pseudo-time solve of Eq. (extrapolation) at full size, learned path, graph replay: the six
    iteration counts exact, the per-side gradients and the sources within the bars, against the
    oracle's solve starting from the GPU reconstruction and least-squares inputs."""
    name, m, a, T, Tb, g, M = full
    if name == "pipe8m":
        pytest.skip("the moving film is timed with the single sweep")
    ge = _run(M, a, T, Tb, m.n_cells, vof.ROOT_LEARNED, graph=True, extrap=1)
    O = oracle.Oracle(m)
    rec = dict(status=ge["status"], A_int=ge["A_int"], n_int=ge["n_int"], x_gamma=ge["x_gamma"])
    keys = ("grad_l", "grad_v", "q_l", "q_v", "mdot", "Q")
    pc, spread = ulp_spread(O, a, rec, T, Tb, synth.PROPS, keys, extrap={})
    assert list(ge["counts"]["extrap_iters"]) == list(pc["extrap_iters"])
    I = ge["iface_idx"]
    assert np.array_equal(ge["status"][I] & 16, pc["status"][I] & 16)
    for k in keys:
        ok, worst = within(ge[k][I], pc[k][I], spread[k][I])
        assert ok, (k, worst)
    np.testing.assert_allclose(ge["totals"], pc["totals"], rtol=1e-10)


def test_full_size_batch64():
    """The 64-mesh union in one graph: eight meshes (every kind, the largest) checked in full
    against the oracle, and every mesh's totals against the oracle's downstream totals on the
    checked meshes."""
    meshes, a, T, Tb, _, _ = workload("batch64")
    B = vof.Batch(meshes)
    assert vof.load_default_mlp(B.mesh)
    g = _run(B.mesh, a, T, Tb, B.mesh.n_cells, vof.ROOT_LEARNED, graph=True, batch=B)
    step = g["counts"]["step"]
    kinds = {}
    for i, m in enumerate(meshes):
        kinds.setdefault(m.kind, []).append(i)
    pick = sorted({ks[0] for ks in kinds.values()} | {ks[-1] for ks in kinds.values()}
                  | {int(np.argmax([m.n_cells for m in meshes]))})
    rng = np.random.default_rng(5)
    for i in pick:
        m = meshes[i]
        c0, c1 = B.cell_off[i], B.cell_off[i + 1]
        v0, v1 = B.vert_off[i], B.vert_off[i + 1]
        gi = {k: g[k][c0:c1] for k in KEYS if k not in ("iface_idx", "phi_v", "face_stamp")}
        gi.update(mdot=g["mdot"][c0:c1], Q=g["Q"][c0:c1], phi_v=g["phi_v"][v0:v1], step=step)
        I = g["iface_idx"]
        gi["iface_idx"] = I[(I >= c0) & (I < c1)] - c0
        tot = check_mesh(m, a[c0:c1], T[c0:c1], Tb[B.face_off[i]:B.face_off[i + 1]], gi, rng)
        np.testing.assert_allclose(g["batch_totals"][i], tot, rtol=1e-10)
    assert g["counts"]["n_not_converged"] == 0
