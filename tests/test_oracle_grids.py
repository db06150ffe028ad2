"""Oracle pins on the other reduced Gaussian grid families: the regular F<N>
grid (4N points on each of 2N parallels, Sec. 4.2.3.6) and grids given by an
arbitrary PL array (points per parallel, Sec. 4.2.3.7), including odd ring
lengths at the poles."""
import numpy as np
import pytest

import oracle
import _pins


def _pl_grid(N):
    """A classic-like reduced grid: octahedral lengths stretched by 1.1 and
    rounded to multiples of 5, every third parallel one longer (odd lengths
    at both poles), mirrored about the equator."""
    o = oracle.row_nx(N)
    pl = (np.round(o * 1.1 / 5) * 5 + (np.arange(2 * N) % 3 == 0)).astype(np.int32)
    pl[N:] = pl[:N][::-1]
    return pl


def _mesh(kind, N):
    return oracle.build_mesh(N, pl=oracle.regular_nx(N) if kind == "F" else _pl_grid(N))


@pytest.mark.parametrize("N", [1, 2, 8, 80, 640])
def test_regular_grid_has_8_n_squared_points(N):
    lat, lon = oracle.grid_lonlat(N, oracle.regular_nx(N))
    assert lat.size == 8 * N * N  # nx = 4N, ny = 2N
    rows = np.unique(lat)
    assert rows.size == 2 * N
    assert np.allclose(rows, np.sort(np.arcsin(oracle.gaussian_rows(N)[0])), rtol=0, atol=1e-15)


def test_explicit_octahedral_pl_array_gives_the_octahedral_mesh():
    N = 16
    m0 = oracle.build_mesh(N)
    m1 = oracle.build_mesh(N, pl=oracle.row_nx(N))
    assert np.array_equal(m0.tri, m1.tri) and np.array_equal(m0.vol, m1.vol)


@pytest.mark.parametrize("kind,N", [("F", 8), ("F", 16), ("P", 6), ("P", 16)])
def test_closed_oriented_mesh_and_exact_invariants(kind, N):
    m = _mesh(kind, N)
    if kind == "P":
        assert m.lat.size == int(_pl_grid(N).sum()) and _pl_grid(N)[0] % 2 == 1
    for pin in (_pins.pin_euler, _pins.pin_orientation, _pins.pin_total_volume, _pins.pin_closed_tangent,
                _pins.pin_grad_constant, _pins.pin_conservation):
        ok, detail = pin(m)
        assert ok, (pin.__name__, detail)


@pytest.mark.parametrize("kind,N", [("F", 6), ("P", 6)])
def test_edge_assembly_equals_direct_dual_cell_walk(kind, N):
    ok, detail = _pins.pin_bruteforce(_mesh(kind, N))
    assert ok, detail


def test_regular_grid_is_four_fold_symmetric():
    """Rotating F<N> by a quarter turn (N points on every parallel) maps the
    strips onto themselves: off the pole rows (whose caps are closed by a
    zig-zag of chords, which no rotation preserves) the dual volumes repeat
    with period N along each row."""
    N = 16
    m = _mesh("F", N)
    vol = m.vol.reshape(2 * N, 4 * N)[1:-1]
    assert np.abs(vol - np.roll(vol, N, axis=1)).max() <= 1e-12 * vol.max()


def _orders(errs, Ns):
    return [np.log(errs[i] / errs[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(len(errs) - 1)]


NS = [16, 32, 64]


def test_regular_grid_operators_converge_at_second_order():
    from paper_1908_06091_b300 import synth
    a, b = synth.sh_coeffs(8, 7)
    ms = [_mesh("F", N) for N in NS]
    eg = [_pins.grad_error(m, a, b) for m in ms]
    ed, ez = zip(*[_pins.wind_errors(m) for m in ms])
    el = [_pins.lap_eigen_error(m, 5) for m in ms]
    for errs in (eg, ed, ez, el):
        assert min(_orders(errs, NS)) > 1.8, errs
    assert eg[-1] < 6e-3 and el[-1] < 7e-3


def test_irregular_pl_grid_operators_converge():
    from paper_1908_06091_b300 import synth
    a, b = synth.sh_coeffs(8, 7)
    ms = [_mesh("P", N) for N in NS]
    eg = [_pins.grad_error(m, a, b) for m in ms]
    el = [_pins.lap_eigen_error(m, 5) for m in ms]
    assert min(_orders(eg, NS)) > 1.0 and eg[-1] < 1.5e-2, eg
    assert min(_orders(el, NS)) > 1.7 and el[-1] < 8e-3, el


@pytest.mark.parametrize("pl", [[20, 24, 20], [20, 2, 2, 20], [], [20]])
def test_pl_arrays_need_an_even_number_of_parallels_of_three_points_or_more(pl):
    with pytest.raises(ValueError):
        oracle.build_mesh(len(pl) // 2 or 1, pl=pl)
