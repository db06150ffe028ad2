"""Oracle grid pins: the paper's printed sizes and row formula, and the
Gauss-Legendre facts that define the Gaussian latitudes (Sec. 4.2.3.5)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("row", _rows("grid_sizes.txt"), ids=lambda r: r[0])
def test_node_counts_printed_in_paper(row):
    N = int(row[0][1:])
    nodes, tol = float(row[1]), float(row[2])
    V = oracle.num_nodes(N)
    assert abs(V - nodes) <= tol * nodes, (V, nodes)


@pytest.mark.parametrize("row", _rows("octahedral_nx.txt"), ids=lambda r: r[0])
def test_row_lengths_listing6(row):
    N = int(row[0][1:])
    assert list(oracle.row_nx(N)) == [int(x) for x in row[1:]]


def test_node_count_closed_form():
    # sum of 2 * (20 + 4j), j < N  =  4 N^2 + 36 N
    for N in (1, 2, 16, 80, 640, 1280):
        assert oracle.num_nodes(N) == 4 * N * N + 36 * N


@pytest.mark.parametrize("N", [1, 2, 16, 32, 80, 400])
def test_gaussian_latitudes_match_library_gauss_legendre(N):
    mu, w = oracle.gaussian_rows(N)
    x, wx = np.polynomial.legendre.leggauss(2 * N)
    order = np.argsort(mu)
    assert np.abs(mu[order] - x).max() < 1e-14
    # numpy's weights lose ~1e-9 relative near the poles for large N
    assert (np.abs(w[order] - wx) / wx).max() < 1e-8


def test_gauss_rows_are_correctly_rounded_50_digit_newton():
    import mpmath
    mpmath.mp.dps = 50
    N = 400
    n = 2 * N
    mu, w = oracle.gaussian_rows(N)

    def P(t):
        p0, p1 = mpmath.mpf(1), t
        for k in range(1, n):
            p0, p1 = p1, ((2 * k + 1) * t * p1 - k * p0) / (k + 1)
        return p1, n * (t * p1 - p0) / (t * t - 1)

    for i in (0, 1, N - 1):
        t = mpmath.mpf(mu[i])
        for _ in range(5):
            p, dp = P(t)
            t = t - p / dp
        p, dp = P(t)
        wr = 2 / ((1 - t * t) * dp * dp)
        assert float(t) == mu[i]                    # correctly rounded root
        assert abs(float(wr / w[i]) - 1) < 1e-14


@pytest.mark.parametrize("N", [16, 48])
def test_gauss_weights_and_exactness(N):
    mu, w = oracle.gaussian_rows(N)
    assert np.all(np.diff(mu) < 0), "rows must run north to south"
    assert np.allclose(mu, -mu[::-1], atol=0, rtol=0)
    assert abs(w.sum() - 2.0) < 1e-14
    # Gauss-Legendre with 2N nodes integrates polynomials of degree < 4N
    # exactly: int P_l P_k = 2/(2l+1) delta_lk
    from numpy.polynomial import legendre as Lg
    for l in (0, 3, 2 * N - 1, 2 * N):
        for k in (l, l + 1, 4 * N - 1 - l):
            if k < 0 or l + k >= 4 * N:
                continue
            pl = Lg.legval(mu, np.eye(l + 1)[l])
            pk = Lg.legval(mu, np.eye(k + 1)[k])
            exact = 2.0 / (2 * l + 1) if l == k else 0.0
            assert abs((w * pl * pk).sum() - exact) < 1e-13


def test_lonlat_first_point_at_greenwich_and_equispaced():
    N = 8
    lat, lon = oracle.grid_lonlat(N)
    nx = oracle.row_nx(N)
    mu, _ = oracle.gaussian_rows(N)
    off = 0
    for j, n in enumerate(nx):
        assert lon[off] == 0.0
        assert np.allclose(lon[off:off + n], 2 * np.pi * np.arange(n) / n, rtol=0, atol=1e-15)
        assert np.allclose(np.sin(lat[off:off + n]), mu[j], rtol=0, atol=1e-15)
        off += n
    assert off == lat.shape[0]
