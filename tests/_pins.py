"""Checks that tie the oracle to facts other than itself.

Each pin returns (ok, detail).  They are used by the oracle's own tests and by
the planted-mistake tests, which switch a known mistake on inside the oracle
and require at least one pin to fail.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1908_06091_b300 import synth

R = oracle.EARTH_RADIUS_M


def _wl2(w, err, ref):
    return float(np.sqrt((w * err ** 2).sum() / (w * ref ** 2).sum()))


def pin_euler(m):
    """Closed triangulated sphere: E = 3V - 6, F = 2V - 4."""
    ok = m.E == 3 * m.V - 6 and m.F == 2 * m.V - 4
    return ok, f"V={m.V} E={m.E} F={m.F}"


def pin_orientation(m):
    """Every triangle is counter-clockwise seen from outside."""
    xyz = np.stack([np.cos(m.lat) * np.cos(m.lon), np.cos(m.lat) * np.sin(m.lon), np.sin(m.lat)], 1)
    a, b, c = xyz[m.tri[:, 0]], xyz[m.tri[:, 1]], xyz[m.tri[:, 2]]
    det = np.einsum("ij,ij->i", np.cross(b - a, c - a), a)
    return bool((det > 0).all()), f"min det {det.min():.3e}"


def _row_starts(m):
    nx = np.asarray(oracle.row_nx(m.N))
    return nx, np.concatenate([[0], np.cumsum(nx)])


def pin_gaussian_rows(m, tol=1e-14):
    """Row latitudes are the Gauss-Legendre nodes of degree 2N, north to
    south (numpy's leggauss)."""
    nx, off = _row_starts(m)
    x, _ = np.polynomial.legendre.leggauss(2 * m.N)
    err = np.abs(np.sin(m.lat[off[:-1]]) - x[::-1]).max()
    same = all(np.all(m.lat[off[j]:off[j + 1]] == m.lat[off[j]]) for j in range(len(nx)))
    return bool(err <= tol and same), f"max |sin(lat) - x| {err:.3e}"


def pin_longitudes(m, tol=1e-15):
    """Each row starts at longitude 0 and its points are equispaced."""
    nx, off = _row_starts(m)
    err = max(np.abs(m.lon[off[j]:off[j + 1]] - 2 * np.pi * np.arange(n) / n).max()
              for j, n in enumerate(nx))
    return bool(err <= tol), f"max lon error {err:.3e}"


def pin_total_volume(m, tol=1e-13):
    """Dual cells tile the sphere: sum V_i = 4 pi R^2."""
    rel = abs(m.vol.sum() / (4 * np.pi * m.R ** 2) - 1.0)
    return rel <= tol, f"rel {rel:.3e}"


def pin_closed_tangent(m, tol=1e-14):
    """The dual boundary of every node is closed: sum_e T_e^(i) = 0."""
    acc = np.zeros((m.V, 3))
    sgn = np.ones(m.E)
    np.add.at(acc, m.edge[:, 0], m.T * sgn[:, None])
    np.add.at(acc, m.edge[:, 1], -m.T * sgn[:, None])
    scale = np.abs(m.T).max()
    rel = np.abs(acc).max() / scale
    return rel <= tol, f"rel {rel:.3e}"


def pin_grad_constant(m):
    """Difference-form gradient of a constant is exactly zero."""
    g = oracle.grad(m, np.full((m.V, 2), 3.25))
    return bool(np.all(g == 0.0)), f"max {np.abs(g).max():.3e}"


def pin_bruteforce(m, nodes=None, tol=1e-12, seed=5):
    """Edge-assembled grad/div/curl and volumes equal a direct walk of each
    node's dual cell (arc integrals per incident triangle, no edge list)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(m.V)
    uv = rng.standard_normal((m.V, 2))
    g = oracle.grad(m, f)[:, 0, :]
    d = oracle.div(m, uv)[:, 0]
    z = oracle.curl(m, uv)[:, 0]
    if nodes is None:
        nodes = range(m.V)
    nodes = list(nodes)
    gb = np.zeros((len(nodes), 2))
    db = np.zeros(len(nodes))
    zb = np.zeros(len(nodes))
    vb = np.zeros(len(nodes))
    for r, i in enumerate(nodes):
        gb[r], vb[r] = oracle.bruteforce_node(m, i, "grad", f)
        db[r], _ = oracle.bruteforce_node(m, i, "div", uv)
        zb[r], _ = oracle.bruteforce_node(m, i, "curl", uv)
    # errors relative to the largest value of each operator over the nodes
    worst = max(np.abs(g[nodes] - gb).max() / np.abs(gb).max(),
                np.abs(d[nodes] - db).max() / np.abs(db).max(),
                np.abs(z[nodes] - zb).max() / np.abs(zb).max(),
                (np.abs(m.vol[nodes] - vb) / vb).max())
    return worst <= tol, f"worst rel {worst:.3e}"


def pin_conservation(m, tol=1e-13, seed=6):
    """Flux form on a closed sphere: sum_i V_i D_i = 0 and sum_i V_i Z_i = 0
    to rounding, relative to sum_i V_i |D_i|."""
    rng = np.random.default_rng(seed)
    uv = rng.standard_normal((m.V, 2))
    d = oracle.div(m, uv)[:, 0]
    z = oracle.curl(m, uv)[:, 0]
    rd = abs((m.vol * d).sum()) / (m.vol * np.abs(d)).sum()
    rz = abs((m.vol * z).sum()) / (m.vol * np.abs(z)).sum()
    return max(rd, rz) <= tol, f"div {rd:.3e} curl {rz:.3e}"


def analytic_grad(m, a, b):
    gy = synth.sh_eval(m.lat, m.lon, a, b, deriv="lat").numpy() / m.R
    gx = synth.sh_eval(m.lat, m.lon, a, b, deriv="lon").numpy() / (m.R * np.cos(m.lat))
    return gx, gy


def grad_error(m, a, b):
    """Area-weighted relative L2 error of the gradient of a harmonic sum
    against its analytic gradient (complex-step in latitude)."""
    f = synth.sh_eval(m.lat, m.lon, a, b).numpy()
    gx, gy = analytic_grad(m, a, b)
    g = oracle.grad(m, f)[:, 0, :]
    return float(np.sqrt((m.vol * ((g[:, 0] - gx) ** 2 + (g[:, 1] - gy) ** 2)).sum()
                         / (m.vol * (gx ** 2 + gy ** 2)).sum()))


def pin_grad_analytic(m, bound):
    a, b = synth.sh_coeffs(8, 7)
    e = grad_error(m, a, b)
    return e <= bound, f"rel L2 {e:.3e} (bound {bound:.1e})"


def solid_body_errors(m, U=20.0):
    """(|div| / (U/R), rel L2 error of curl against 2 U sin(lat) / R)."""
    sb = synth.solid_body_wind(m.lat, U)
    d = oracle.div(m, sb)[:, 0]
    z = oracle.curl(m, sb)[:, 0]
    zr = 2 * U * np.sin(m.lat) / m.R
    dn = float(np.sqrt((m.vol * d ** 2).sum() / m.vol.sum()) / (U / m.R))
    return dn, _wl2(m.vol, z - zr, zr)


def pin_solid_body(m, div_bound, curl_bound):
    dn, ez = solid_body_errors(m)
    return dn <= div_bound and ez <= curl_bound, f"div {dn:.3e} curl {ez:.3e}"


def lap_eigen_error(m, l, mm=1):
    """Rayleigh quotient of the discrete Laplacian on Y_lm vs -l(l+1)/R^2."""
    a = np.zeros((l + 1, l + 1))
    b = np.zeros((l + 1, l + 1))
    a[l, min(mm, l)] = 1.0
    if l >= 1:
        b[l, 1] = 0.5
    Y = synth.sh_eval(m.lat, m.lon, a, b).numpy()
    L = oracle.lap(m, Y)[:, 0]
    lam = (m.vol * L * Y).sum() / (m.vol * Y * Y).sum()
    return abs(lam / (-l * (l + 1) / m.R ** 2) - 1.0)


def pin_lap_eigen(m, l, bound):
    e = lap_eigen_error(m, l)
    return e <= bound, f"l={l} rel {e:.3e} (bound {bound:.1e})"


def wind_errors(m, lmax=8, seed=11):
    """Rel. L2 errors of div(grad chi) vs lap(chi) and curl(k x grad psi)
    vs lap(psi), analytic Laplacian -l(l+1)/R^2 per degree."""
    a, b = synth.sh_coeffs(lmax, seed)
    gx, gy = analytic_grad(m, a, b)
    ls = np.array([-l * (l + 1) / m.R ** 2 for l in range(lmax + 1)])
    lapa = synth.sh_eval(m.lat, m.lon, a, b, scale_l=ls).numpy()
    d = oracle.div(m, np.stack([gx, gy], 1))[:, 0]
    z = oracle.curl(m, np.stack([-gy, gx], 1))[:, 0]
    return _wl2(m.vol, d - lapa, lapa), _wl2(m.vol, z - lapa, lapa)


def pin_wind(m, bound):
    ed, ez = wind_errors(m)
    return max(ed, ez) <= bound, f"div {ed:.3e} curl {ez:.3e}"
