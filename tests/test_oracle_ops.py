"""Oracle operator pins: exact identities, conservation, and convergence to
the continuous operators on analytic spherical-harmonic fields."""
import numpy as np
import pytest

import oracle
import _pins


@pytest.mark.parametrize("N", [16, 32])
def test_gradient_of_constant_is_exactly_zero(N, mesh_factory):
    ok, msg = _pins.pin_grad_constant(mesh_factory(N))
    assert ok, msg


@pytest.mark.parametrize("N", [16, 32])
def test_discrete_conservation(N, mesh_factory):
    ok, msg = _pins.pin_conservation(mesh_factory(N))
    assert ok, msg


def test_laplacian_sums_to_zero(mesh_factory):
    m = mesh_factory(32)
    f = np.random.default_rng(3).standard_normal((m.V, 3))
    L = oracle.lap(m, f)
    r = np.abs((m.vol[:, None] * L).sum(0)) / (m.vol[:, None] * np.abs(L)).sum(0)
    assert r.max() < 1e-13


def test_levels_are_independent(mesh_factory):
    m = mesh_factory(16)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((m.V, 5))
    uv = rng.standard_normal((m.V, 5, 2))
    g = oracle.grad(m, f)
    d = oracle.div(m, uv)
    for k in (0, 3):
        assert np.array_equal(g[:, k], oracle.grad(m, f[:, k])[:, 0])
        assert np.array_equal(d[:, k], oracle.div(m, uv[:, k])[:, 0])


def _orders(errs, Ns):
    return [np.log(errs[i] / errs[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(len(errs) - 1)]


NS = [16, 32, 64]


def test_gradient_converges_to_analytic(mesh_factory):
    from paper_1908_06091_b300 import synth
    a, b = synth.sh_coeffs(8, 7)
    errs = [_pins.grad_error(mesh_factory(N), a, b) for N in NS]
    assert errs[-1] < 1e-2
    assert min(_orders(errs, NS)) > 1.5, errs


def test_div_and_curl_converge_to_analytic_laplacians(mesh_factory):
    ed, ez = zip(*[_pins.wind_errors(mesh_factory(N)) for N in NS])
    assert ed[-1] < 1.2e-2 and ez[-1] < 1.2e-2
    assert min(_orders(ed, NS)) > 1.5 and min(_orders(ez, NS)) > 1.5, (ed, ez)


def test_solid_body_rotation(mesh_factory):
    dn, ez = zip(*[_pins.solid_body_errors(mesh_factory(N)) for N in NS])
    # analytic: divergence 0, vorticity 2 U sin(lat) / R
    assert dn[-1] < 3e-4 and ez[-1] < 1.5e-3
    assert min(_orders(dn, NS)) > 1.2 and min(_orders(ez, NS)) > 1.2, (dn, ez)


def test_curl_of_grad_vanishes_under_refinement(mesh_factory):
    from paper_1908_06091_b300 import synth
    a, b = synth.sh_coeffs(8, 9)
    rs = []
    for N in NS:
        m = mesh_factory(N)
        f = synth.sh_eval(m.lat, m.lon, a, b).numpy()
        g = oracle.grad(m, f)
        z = oracle.curl(m, g)[:, 0]
        L = oracle.lap(m, f)[:, 0]
        rs.append(np.sqrt((m.vol * z ** 2).sum() / (m.vol * L ** 2).sum()))
    assert rs[-1] < 2e-2 and rs[0] > rs[1] > rs[2], rs


@pytest.mark.parametrize("l", [1, 2, 5, 10])
def test_laplacian_eigenvalues_of_spherical_harmonics(l, mesh_factory):
    errs = [_pins.lap_eigen_error(mesh_factory(N), l) for N in NS]
    assert errs[-1] < 0.025, errs
    assert min(_orders(errs, NS)) > 1.6, errs
