"""GPU parity of the pseudo-time extrapolation (options.extrap = 1, Eq. extrapolation solved in
full): the CUDA path through the C ABI against the oracle starting from the GPU reconstruction.

Steps with at most ten interface cells per warp of the launch keep each lane's constants in
registers; larger ones loop over groups of ten; both are covered. Bars: iteration counts of the six solves and the no-side flags exact; the pseudo-time step to one
ulp; the per-side gradients, heat rates, mdot and Q to relative 1e-8 (vectors in the Euclidean
norm), widened to 100 times the oracle's own movement under one-ulp centroid rounding where the
least-squares stencil is ill-conditioned; totals to 1e-10. A solve whose largest change lands
within rounding of the tolerance could stop one iteration apart on the two sides; none of these
seeded cases does."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import EPS, case, gpu_step, ulp_spread, within

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14938_gb300 as vof  # noqa: E402

CASES = ["hex_sphere", "voronoi_film", "voronoi_spheres", "tet_sphere", "prism_sphere", "pipe_film"]
KEYS = ("grad_l", "grad_v", "q_l", "q_v", "mdot", "Q")


def check(m, a, T, Tb, g, ex):
    O = oracle.Oracle(m)
    rec = dict(status=g["status"], A_int=g["A_int"], n_int=g["n_int"], x_gamma=g["x_gamma"])
    pc, spread = ulp_spread(O, a, rec, T, Tb, synth.PROPS, KEYS, extrap=ex)
    assert list(g["counts"]["extrap_iters"]) == list(pc["extrap_iters"])
    I = g["iface_idx"]
    assert np.array_equal(g["status"][I] & 16, pc["status"][I] & 16)
    assert g["counts"]["n_no_side"] == int(np.count_nonzero(pc["status"][I] & 16))
    for k in KEYS:
        ok, worst = within(g[k][I], pc[k][I], spread[k][I])
        assert ok, (k, worst)
    np.testing.assert_allclose(g["totals"], pc["totals"], rtol=1e-10, atol=1e-300)
    return O, pc


@pytest.mark.parametrize("name", CASES)
def test_extrap_parity(name):
    m, a, T, Tb = case(name)
    M, g = gpu_step(m, a, T, Tb, extrap=1)
    O, pc = check(m, a, T, Tb, g, {})
    assert g["dtau"][0] == pytest.approx(O.extrap_dtau(), rel=5e-16)
    assert g["counts"]["n_not_converged"] == 0


def test_extrap_many_slots_per_lane():
    """More interface cells than the launch has lane triples (a 256-thread block per SM, ten cells
    per warp): each lane loops over several cells per iteration."""
    m, a, T, Tb = case("voronoi_many_spheres")
    M, g = gpu_step(m, a, T, Tb, extrap=1)
    assert g["counts"]["n_iface"] > torch.cuda.get_device_properties(0).multi_processor_count * 8 * 10
    check(m, a, T, Tb, g, {})


@pytest.mark.parametrize("max_iter,tol", [(1, 1e-3), (3, 1e-3), (40, 1e-6)])
def test_extrap_caps_and_tolerances(max_iter, tol):
    m, a, T, Tb = case("voronoi_film")
    M, g = gpu_step(m, a, T, Tb, extrap=1, extrap_max_iter=max_iter, extrap_tol=tol)
    check(m, a, T, Tb, g, dict(max_iter=max_iter, tol=tol))
    assert max(g["counts"]["extrap_iters"]) <= max_iter


def test_extrap_learned_graph_replay_matches_eager():
    """The benchmark's configuration: learned root search, graph replay; the replayed step gives
    the eager step's outputs bit for bit, and the single-sweep step after it is unchanged."""
    m, a, T, Tb = case("voronoi_spheres")
    M = vof.Mesh(m)
    assert vof.load_default_mlp(M)
    d = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        ta, tT, tTb = d(a), d(T), d(Tb)
        for graph, ex in ((False, 1), (True, 1), (True, 1), (False, 0)):
            opt = vof.default_options(root_mode=vof.ROOT_LEARNED, extrap=ex)
            mdot = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
            Q, tot = torch.empty_like(mdot), torch.empty(2, dtype=torch.float64, device="cuda")
            (M.step_graph if graph else M.step)(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt, stream=s)
            s.synchronize()
            outs.append(dict(mdot=mdot.cpu().numpy(), totals=tot.cpu().numpy(), counts=M.counts(stream=s),
                             grad_v=M.field("grad_v", stream=s).cpu().numpy()))
    torch.cuda.synchronize()
    for o in outs[1:3]:
        assert np.array_equal(o["mdot"], outs[0]["mdot"]) and np.array_equal(o["totals"], outs[0]["totals"])
        assert o["counts"]["extrap_iters"] == outs[0]["counts"]["extrap_iters"]
    assert outs[3]["counts"]["extrap_iters"] == [0] * 6
    _, g0 = gpu_step(m, a, T, Tb, root_mode=vof.ROOT_LEARNED, dev_mesh=M)
    assert np.array_equal(outs[3]["mdot"], g0["mdot"])


@pytest.mark.parametrize("bad", [dict(extrap=2), dict(extrap=1, extrap_max_iter=0),
                                 dict(extrap=1, extrap_max_iter=1001), dict(extrap=1, extrap_tol=0.0),
                                 dict(extrap=1, extrap_tol=float("nan"))])
def test_extrap_options_rejected(bad):
    m, a, T, Tb = case("hex_sphere")
    with pytest.raises(RuntimeError):
        gpu_step(m, a, T, Tb, **bad)


def test_extrap_without_interface():
    """No interface cell: every solve stops after its first iteration, no source anywhere."""
    m, a, T, Tb = case("hex_sphere")
    a = np.ones(m.n_cells)
    M, g = gpu_step(m, a, T, Tb, extrap=1)
    assert g["counts"]["n_iface"] == 0
    assert list(g["counts"]["extrap_iters"]) == [1] * 6
    assert not np.any(g["mdot"]) and not np.any(g["totals"])


def test_barrier_poll_limit_reports_and_recovers():
    """The extrapolation's per-iteration barrier is a bounded poll: with a limit of one read per
    block (options.extrap_poll_limit = 1), a block that finds the barrier not yet full stops
    waiting, the kernel returns, and the step reports -1 iterations for all six solves; the next
    step with the default limit is exact again (same counts and outputs as before)."""
    m, a, T, Tb = case("voronoi_spheres")
    M, g1 = gpu_step(m, a, T, Tb, extrap=1)
    assert min(g1["counts"]["extrap_iters"]) > 0
    gave_up = None
    for _ in range(20):  # a launch in which every block found every barrier full is possible, not likely
        _, gf = gpu_step(m, a, T, Tb, dev_mesh=M, extrap=1, extrap_poll_limit=1)
        if list(gf["counts"]["extrap_iters"]) == [-1] * 6:
            gave_up = gf
            break
    assert gave_up is not None
    _, g2 = gpu_step(m, a, T, Tb, dev_mesh=M, extrap=1)
    assert list(g2["counts"]["extrap_iters"]) == list(g1["counts"]["extrap_iters"])
    for k in ("grad_l", "grad_v", "mdot", "Q", "totals"):
        assert np.array_equal(g2[k], g1[k]), k
