"""Oracle triangulation pins (reading of Sec. 4.3, Listing 7, Fig. 25b)."""
import numpy as np
import pytest

import oracle
import _pins


@pytest.mark.parametrize("N", [1, 2, 16, 32, 48])
def test_euler_and_orientation(N):
    m = oracle.build_mesh(N)
    ok, msg = _pins.pin_euler(m)
    assert ok, msg
    ok, msg = _pins.pin_orientation(m)
    assert ok, msg


@pytest.mark.parametrize("N", [16, 32])
def test_every_edge_shared_by_two_opposite_triangles(N, mesh_factory):
    m = mesh_factory(N)
    for e in range(0, m.E, 7):
        a, b = m.edge[e]
        L, R = m.etri[e]
        tl, tr = list(m.tri[L]), list(m.tri[R])
        # left triangle holds a->b, right triangle holds b->a
        assert any(tl[c] == a and tl[(c + 1) % 3] == b for c in range(3))
        assert any(tr[c] == b and tr[(c + 1) % 3] == a for c in range(3))
    # every triangle has 3 distinct nodes
    t = m.tri
    assert np.all((t[:, 0] != t[:, 1]) & (t[:, 1] != t[:, 2]) & (t[:, 0] != t[:, 2]))


def _row_of(N):
    nx = oracle.row_nx(N)
    off = np.concatenate([[0], np.cumsum(nx)])
    row = np.repeat(np.arange(2 * N), nx)
    col = np.arange(off[-1]) - off[row]
    return nx, off, row, col


@pytest.mark.parametrize("N", [8, 16])
def test_strips_are_four_fold_symmetric_in_longitude(N):
    m = oracle.build_mesh(N)
    nx, off, row, col = _row_of(N)
    rot = off[row] + (col + nx[row] // 4) % nx[row]
    strip = (row[m.tri].min(1) != row[m.tri].max(1))
    tris = m.tri[strip]
    key = lambda t: tuple(np.roll(t, -int(np.argmin(t))))
    S = {key(t) for t in tris}
    assert {key(rot[t]) for t in tris} == S


@pytest.mark.parametrize("N", [8, 16])
def test_mirror_symmetry_about_equator_off_the_equator_strip(N):
    m = oracle.build_mesh(N)
    nx, off, row, col = _row_of(N)
    mirror = off[2 * N - 1 - row] + col
    rmin, rmax = row[m.tri].min(1), row[m.tri].max(1)
    keep = ~((rmin == N - 1) & (rmax == N))
    tris = m.tri[keep]
    # mirroring reverses orientation: compare unoriented triangles
    S = {tuple(sorted(t)) for t in tris}
    assert {tuple(sorted(mirror[t])) for t in tris} == S


def test_strip_and_cap_counts():
    N = 6
    m = oracle.build_mesh(N)
    nx, off, row, col = _row_of(N)
    rmin, rmax = row[m.tri].min(1), row[m.tri].max(1)
    assert ((rmin == 0) & (rmax == 0)).sum() == nx[0] - 2
    assert ((rmin == 2 * N - 1) & (rmax == 2 * N - 1)).sum() == nx[-1] - 2
    for j in range(2 * N - 1):
        assert ((rmin == j) & (rmax == j + 1)).sum() == nx[j] + nx[j + 1]
