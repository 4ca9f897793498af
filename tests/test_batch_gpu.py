"""Batches, graph replay and the autotuner on the GPU: a union of meshes of every kind gives, per
mesh, bit-for-bit the outputs and totals of stepping that mesh alone; a replayed graph gives the
eager step's outputs; tuned lanes-per-cell choices keep the parity bar."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import case, gpu_step

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14938_gb300 as vof  # noqa: E402

d = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _run(M, a, T, Tb, n_cells, graph=False, stream=None, **opt):
    mdot = torch.empty(n_cells, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(mdot)
    tot = torch.empty(2, dtype=torch.float64, device="cuda")
    o = vof.default_options(**opt)
    if graph:
        M.step_graph(d(a), d(T), d(Tb), synth.PROPS, mdot, Q, tot, o, stream=stream)
    else:
        M.step(d(a), d(T), d(Tb), synth.PROPS, mdot, Q, tot, o)
    torch.cuda.synchronize()
    return mdot.cpu().numpy(), tot.cpu().numpy()


def test_batch_equals_separate_runs():
    names = ["hex_sphere", "tet_sphere", "prism_sphere", "voronoi_spheres", "pipe_film"]
    cases = [case(n) for n in names]
    B = vof.Batch([c[0] for c in cases])
    B.mesh.set_group_sizes([1, 2, 4, 16, 32])
    a = np.concatenate([c[1] for c in cases])
    T = np.concatenate([c[2] for c in cases])
    Tb = np.concatenate([c[3] for c in cases])
    mdot, _ = _run(B.mesh, a, T, Tb, B.mesh.n_cells)
    tot = B.totals().cpu().numpy()
    for i, (m, ai, Ti, Tbi) in enumerate(cases):
        M = vof.Mesh(m)
        M.set_group_sizes([1, 2, 4, 16, 32])
        md, t1 = _run(M, ai, Ti, Tbi, m.n_cells)
        assert np.array_equal(mdot[B.cell_off[i]:B.cell_off[i + 1]], md), names[i]
        assert np.array_equal(tot[i], t1), names[i]


def test_graph_replay_matches_eager_and_follows_inputs():
    m, a, T, Tb = case("voronoi_film")
    M = vof.Mesh(m)
    s = torch.cuda.Stream()
    ta, tT, tTb = d(a), d(T), d(Tb)
    mdot = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(mdot)
    tot = torch.empty(2, dtype=torch.float64, device="cuda")
    o = vof.default_options()
    M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, o)
    torch.cuda.synchronize()
    ref = mdot.clone()
    with torch.cuda.stream(s):
        for _ in range(3):
            M.step_graph(ta, tT, tTb, synth.PROPS, mdot, Q, tot, o, stream=s)
    s.synchronize()
    assert torch.equal(mdot, ref)
    # new data in the same buffers: the replayed graph follows it
    a2 = np.clip(a * 0.9 + 0.05, 0, 1)
    ta.copy_(d(a2))
    with torch.cuda.stream(s):
        M.step_graph(ta, tT, tTb, synth.PROPS, mdot, Q, tot, o, stream=s)
    s.synchronize()
    r = oracle.Oracle(m).run(a2, T, Tb, synth.PROPS)
    ref2 = r["pc"]["mdot"]
    err = np.abs(mdot.cpu().numpy() - ref2) / np.maximum(np.abs(ref2), 1e-3 * np.abs(ref2).max())
    assert err.max() <= 1e-8


def test_autotune_choices_keep_parity():
    cases = [case(n) for n in ("hex_sphere", "voronoi_spheres")]
    B = vof.Batch([c[0] for c in cases])
    a = np.concatenate([c[1] for c in cases])
    G = B.mesh.autotune(d(a))
    assert all(g in (0, 1, 2, 4, 8, 16, 32) for g in G)
    assert any(G)
    T = np.concatenate([c[2] for c in cases])
    Tb = np.concatenate([c[3] for c in cases])
    _, g = gpu_step(None, a, T, Tb, dev_mesh=B.mesh, n_cells=B.mesh.n_cells)
    for i, (m, ai, Ti, Tbi) in enumerate(cases):
        O = oracle.Oracle(m)
        V = O.geometry()["cell_vol"]
        off, voff = B.cell_off[i], B.vert_off[i]
        phi = g["phi_v"][voff:B.vert_off[i + 1]]
        for c in np.where((ai > 1e-12) & (ai < 1 - 1e-12))[0]:
            assert abs(O.liquid_volume(c, phi, g["iso"][off + c])["VL"] / V[c] - ai[c]) <= 1e-10


def test_batch_extrapolation_shares_step_and_stop():
    """The pseudo-time extrapolation in a batch: one mesh to the step, so dtau is the smallest over
    the meshes and each solve stops when no mesh moves by tol or more. The step's homogeneous
    iteration matrix is non-negative with row sums <= 1, so a mesh's largest change never grows:
    the batch's count of a solve is the largest of the meshes' counts at the batch's dtau, and each
    mesh's values are the oracle's after exactly that many iterations."""
    names = ["voronoi_spheres", "hex_sphere", "prism_sphere"]
    cases = [case(n) for n in names]
    B = vof.Batch([c[0] for c in cases])
    a = np.concatenate([c[1] for c in cases])
    T = np.concatenate([c[2] for c in cases])
    Tb = np.concatenate([c[3] for c in cases])
    _run(B.mesh, a, T, Tb, B.mesh.n_cells, extrap=1)
    K = B.mesh.counts()["extrap_iters"]
    dtau = float(B.mesh.field("dtau").cpu().numpy()[0])
    f = {k: B.mesh.field(k).cpu().numpy() for k in ("status", "A_int", "n_int", "x_gamma", "grad_l", "grad_v")}
    own_K = []
    for i, (m, ai, Ti, Tbi) in enumerate(cases):
        O = oracle.Oracle(m)
        assert O.extrap_dtau() >= dtau
        c0, c1 = B.cell_off[i], B.cell_off[i + 1]
        I = np.where((ai > 1e-12) & (ai < 1 - 1e-12))[0]  # the fields hold values on interface cells
        rec = {k: f[k][c0:c1] for k in ("status", "A_int", "n_int", "x_gamma")}
        own_K.append(O.phase_change(ai, rec, Ti, Tbi, synth.PROPS, extrap=dict(dtau=dtau))["extrap_iters"])
        for k_it in sorted(set(K)):
            pc = O.phase_change(ai, rec, Ti, Tbi, synth.PROPS, extrap=dict(dtau=dtau, max_iter=k_it, tol=0.0))
            for j in range(6):
                if K[j] != k_it:
                    continue
                side, comp = ("grad_l", "grad_v")[j // 3], j % 3
                g, o = f[side][c0:c1, comp][I], pc[side][I, comp]
                scale = max(np.abs(o).max(), 1e-300)
                assert np.abs(g - o).max() <= 1e-8 * scale, (names[i], j)
    assert list(K) == list(np.max(np.array(own_K), axis=0))
