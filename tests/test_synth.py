"""The seeded input generators: closed, conforming meshes of every kind; fields in range."""
import numpy as np
import pytest

import synth


def _closure(m):
    P = np.stack([m.vx, m.vy, m.vz], 1)
    fa = np.zeros((m.n_faces, 3))
    for f in range(m.n_faces):
        L = P[m.face_loop(f)]
        fa[f] = 0.5 * np.cross(L, np.roll(L, -1, 0)).sum(0)
    res = 0.0
    for c in range(m.n_cells):
        s = np.zeros(3)
        for f, r in m.cell_faces(c):
            s += -fa[f] if r else fa[f]
        res = max(res, np.abs(s).max())
    return res


@pytest.mark.parametrize("mk", [lambda: synth.hex_box(3), lambda: synth.tet_box(2), lambda: synth.prism_box(2),
                                lambda: synth.voronoi_bcc(4, seed=1), lambda: synth.pipe(0.2, 2, 1.0, 0.5, seed=2)])
def test_meshes_closed_and_conforming(mk):
    m = mk()
    assert m.conform_errors == 0
    assert _closure(m) < 1e-14
    # every interior face is listed by both cells, every boundary face by one
    cnt = np.bincount(m.cell_face & 0x7FFFFFFF, minlength=m.n_faces)
    assert np.all(cnt == np.where(m.face_neigh >= 0, 2, 1))


def test_voronoi_is_deterministic_and_sized():
    a = synth.voronoi_bcc(6, seed=1)
    b = synth.voronoi_bcc(6, seed=1)
    c = synth.voronoi_bcc(6, seed=2)
    assert a.n_cells == 2 * 6 ** 3
    assert np.array_equal(a.vx, b.vx) and np.array_equal(a.face_vert, b.face_vert)
    assert not np.array_equal(a.vx, c.vx)


def test_alpha_in_range_and_volume():
    m = synth.hex_box(16)
    reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.3)])
    a = synth.alpha(m, reg, mode="hexgrid", level=3)
    assert a.min() >= 0 and a.max() <= 1
    vapour = (1 - a).sum() / 16 ** 3
    assert vapour == pytest.approx(4 / 3 * np.pi * 0.3 ** 3, rel=2e-3)
    mv = synth.voronoi_bcc(8, seed=1)
    av = synth.alpha(mv, dict(type="film", z0=0.3, a=0.03), mode="subtet", level=2)
    assert 0.0 <= av.min() and av.max() <= 1.0
    assert ((av > 0) & (av < 1)).sum() > 50
