"""Seeded synthetic inputs: spherical-harmonic fields on grid nodes.

This module draws and evaluates test/benchmark inputs only; it holds none of
the finite-volume method's arithmetic and imports nothing from the CUDA path
or from the oracle, so both sides can be fed the same values.

Fields are sums of real, 4-pi normalised spherical harmonics
    f(lat, lon) = sum_{l<=lmax} sum_{m<=l} (a_lm cos(m lon) + b_lm sin(m lon)) Pbar_lm(sin lat)
with a_lm, b_lm ~ N(0, 1) / (l + 1) and b_l0 = 0, drawn from
numpy.random.Generator(PCG64(seed)).  Pbar_lm uses the standard stable
column recurrences (Holmes and Featherstone, J. Geodesy 76, 2002):
    Pbar_00 = 1,  Pbar_11 = sqrt(3) cos,  Pbar_mm = sqrt((2m+1)/(2m)) cos Pbar_{m-1,m-1},
    Pbar_{m+1,m} = sqrt(2m+3) sin Pbar_mm,
    Pbar_lm = a sin Pbar_{l-1,m} - b Pbar_{l-2,m},
        a = sqrt((2l-1)(2l+1) / ((l-m)(l+m))),
        b = sqrt((2l+1)(l+m-1)(l-m-1) / ((l-m)(l+m)(2l-3))).
Latitude derivatives use the complex-step method (Squire and Trapp, SIAM
Rev. 40, 1998): d/dlat f = Im f(lat + i h) / h, exact to rounding.

Multi-level fields mix 8 seeded basis fields per level with weights that grow
with the level: f_k = (1 + k / L) * sum_b w_kb F_b, w_kb ~ N(0, 1/8).
Vector winds are W = k x grad(psi) + grad(chi) from two harmonic sums (their
divergence is lap(chi), their curl lap(psi)), in local (east, north)
components, plus the solid-body wind u = U cos(lat), v = 0.

Everything is torch float64.  The Legendre part runs on the CPU over the
distinct latitudes of the grid; the per-node sums run on any device (CPU for
the oracle's inputs, CUDA for large benchmark inputs), all basis fields of a
kind in one pass.
"""
from __future__ import annotations

import math

import numpy as np
import torch

BASE_SEED = 20261203
N_BASIS = 8
WIND_SCALE = 1.0e7  # m^2/s for psi and chi: winds of order 10 m/s


def sh_coeffs(lmax: int, seed: int):
    """(a, b) coefficient arrays [lmax+1][lmax+1] (l, m); zero for m > l."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.zeros((lmax + 1, lmax + 1))
    b = np.zeros((lmax + 1, lmax + 1))
    for l in range(lmax + 1):
        for m in range(l + 1):
            a[l, m] = rng.standard_normal() / (l + 1)
            b[l, m] = 0.0 if m == 0 else rng.standard_normal() / (l + 1)
    return a, b


def legendre_bar(lmax: int, lat: torch.Tensor) -> torch.Tensor:
    """Pbar_lm(sin lat) for all l, m <= lmax: shape [lmax+1, lmax+1, n].

    ``lat`` may be complex (for complex-step derivatives)."""
    s = torch.sin(lat)
    c = torch.cos(lat)
    P = torch.zeros((lmax + 1, lmax + 1) + tuple(lat.shape), dtype=lat.dtype, device=lat.device)
    P[0, 0] = 1.0
    for m in range(1, lmax + 1):
        fac = math.sqrt(3.0) if m == 1 else math.sqrt((2.0 * m + 1.0) / (2.0 * m))
        P[m, m] = fac * c * P[m - 1, m - 1]
    for m in range(0, lmax):
        P[m + 1, m] = math.sqrt(2.0 * m + 3.0) * s * P[m, m]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((2.0 * l - 1.0) * (2.0 * l + 1.0) / ((l - m) * (l + m)))
            b = math.sqrt((2.0 * l + 1.0) * (l + m - 1.0) * (l - m - 1.0)
                          / ((l - m) * (l + m) * (2.0 * l - 3.0)))
            P[l, m] = a * s * P[l - 1, m] - b * P[l - 2, m]
    return P


def _as_t(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64)
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=device)


def sh_eval_many(lat, lon, coeffs, *, deriv: str | None = None, scale_l=None,
                 device=None) -> torch.Tensor:
    """Evaluate K harmonic sums at V nodes: float64 tensor [V, K].

    coeffs: list of (a, b) coefficient arrays of one common lmax.
    deriv: None (value), 'lat' (d/dlat, complex step) or 'lon' (d/dlon).
    scale_l: optional per-degree multipliers (e.g. -l(l+1)/R^2 for the
    continuous Laplacian).  The Legendre part runs on the CPU over the
    distinct latitudes; the per-node sum over orders m runs on `device`."""
    device = device or (lat.device if isinstance(lat, torch.Tensor) else "cpu")
    lat_c = _as_t(lat, "cpu")
    lon_d = _as_t(lon, device)
    lmax = coeffs[0][0].shape[0] - 1
    A = torch.as_tensor(np.stack([c[0] for c in coeffs]), dtype=torch.float64)  # [K, l, m]
    B = torch.as_tensor(np.stack([c[1] for c in coeffs]), dtype=torch.float64)
    if scale_l is not None:
        sl = torch.as_tensor(np.asarray(scale_l, dtype=np.float64))[None, :, None]
        A = A * sl
        B = B * sl
    ulat, inv = torch.unique(lat_c, return_inverse=True)
    h = 1e-30
    if deriv == "lat":
        P = legendre_bar(lmax, ulat.to(torch.complex128) + 1j * h).imag / h
    else:
        P = legendre_bar(lmax, ulat)
    Am = torch.einsum("klm,lmr->mrk", A, P).to(device)  # [m, rows, K]
    Bm = torch.einsum("klm,lmr->mrk", B, P).to(device)
    inv = inv.to(device)
    out = torch.zeros((lon_d.shape[0], len(coeffs)), dtype=torch.float64, device=device)
    c1, s1 = torch.cos(lon_d), torch.sin(lon_d)
    cm, sm = torch.ones_like(lon_d), torch.zeros_like(lon_d)
    for m in range(lmax + 1):
        if deriv == "lon":
            out += m * (Bm[m][inv] * cm[:, None] - Am[m][inv] * sm[:, None])
        else:
            out += Am[m][inv] * cm[:, None] + Bm[m][inv] * sm[:, None]
        cm, sm = cm * c1 - sm * s1, sm * c1 + cm * s1
    return out


def sh_eval(lat, lon, a, b, *, deriv: str | None = None, scale_l=None,
            device=None) -> torch.Tensor:
    """Evaluate one harmonic sum at the nodes (float64 tensor of shape [V])."""
    return sh_eval_many(lat, lon, [(a, b)], deriv=deriv, scale_l=scale_l, device=device)[:, 0]


def level_weights(nlev: int, seed: int) -> np.ndarray:
    """[nlev][N_BASIS] mixing weights, amplitude growing as 1 + k/nlev."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((nlev, N_BASIS)) / math.sqrt(N_BASIS)
    return w * (1.0 + np.arange(nlev) / max(nlev, 1))[:, None]


def scalar_basis(lat, lon, lmax: int, seed: int, device=None) -> torch.Tensor:
    """[V][N_BASIS] float64 harmonic basis fields."""
    coeffs = [sh_coeffs(lmax, seed * 1000 + bidx) for bidx in range(N_BASIS)]
    return sh_eval_many(lat, lon, coeffs, device=device)


def scalar_field(lat, lon, nlev: int, lmax: int, seed: int = BASE_SEED, device=None) -> torch.Tensor:
    """[V][nlev] float64: per-level mixture of the harmonic basis."""
    basis = scalar_basis(lat, lon, lmax, seed, device=device)
    w = torch.as_tensor(level_weights(nlev, seed + 1), device=basis.device)
    return basis @ w.T


def wind_basis(lat, lon, lmax: int, seed: int, R: float, device=None) -> torch.Tensor:
    """[V][N_BASIS][2] float64 winds W_b = k x grad(psi_b) + grad(chi_b)."""
    device = device or (lat.device if isinstance(lat, torch.Tensor) else "cpu")
    coslat = torch.cos(_as_t(lat, device))[:, None]
    scale = lambda c: (c[0] * WIND_SCALE, c[1] * WIND_SCALE)
    psi = [scale(sh_coeffs(lmax, seed * 1000 + 100 + b)) for b in range(N_BASIS)]
    chi = [scale(sh_coeffs(lmax, seed * 1000 + 200 + b)) for b in range(N_BASIS)]
    psi_lat = sh_eval_many(lat, lon, psi, deriv="lat", device=device)
    psi_lon = sh_eval_many(lat, lon, psi, deriv="lon", device=device)
    chi_lat = sh_eval_many(lat, lon, chi, deriv="lat", device=device)
    chi_lon = sh_eval_many(lat, lon, chi, deriv="lon", device=device)
    u = (-psi_lat + chi_lon / coslat) / R
    v = (psi_lon / coslat + chi_lat) / R
    return torch.stack([u, v], dim=2)


def wind_field(lat, lon, nlev: int, lmax: int, R: float, seed: int = BASE_SEED,
               device=None) -> torch.Tensor:
    """[V][nlev][2] float64 per-level mixture of the wind basis."""
    basis = wind_basis(lat, lon, lmax, seed, R, device=device)
    w = torch.as_tensor(level_weights(nlev, seed + 2), device=basis.device)
    return torch.einsum("vbc,kb->vkc", basis, w)


def solid_body_wind(lat, U: float = 20.0) -> np.ndarray:
    """[V][2]: u = U cos(lat), v = 0."""
    lat = np.asarray(lat, dtype=np.float64)
    return np.stack([U * np.cos(lat), np.zeros_like(lat)], axis=1)
