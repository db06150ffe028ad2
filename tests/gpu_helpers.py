"""Shared helpers of the GPU parity tests: build both sides, feed them the
same seeded inputs, compare element by element in grid order."""
from __future__ import annotations

import functools

import numpy as np
import torch

import oracle
from paper_1908_06091_b300 import nabla, synth

R = oracle.EARTH_RADIUS_M
NP_DT = {torch.float32: np.float32, torch.float64: np.float64}


@functools.lru_cache(maxsize=8)
def product(N: int, reorder: int = 1):
    g = nabla.Grid(N)
    m = nabla.Mesh(g, reorder)
    meth = nabla.Method(m, R)
    return g, m, meth


@functools.lru_cache(maxsize=6)
def oracle_mesh(N: int):
    return oracle.build_mesh(N, R)


def inputs(om, nlev: int, lmax: int, dtype, seed: int = synth.BASE_SEED):
    """Seeded scalar [V][L] and wind [V][L][2] in grid order, rounded to
    dtype (the exact values both sides receive)."""
    f = synth.scalar_field(om.lat, om.lon, nlev, lmax, seed).numpy()
    uv = synth.wind_field(om.lat, om.lon, nlev, lmax, R, seed).numpy()
    dt = NP_DT[dtype]
    return f.astype(dt), uv.astype(dt)


def to_device(fs: "nabla.NodeColumns", x_grid: np.ndarray, perm: np.ndarray, nvar: int,
              stride_pad: bool = True) -> torch.Tensor:
    """Grid-order host array -> functionspace-order device field view."""
    x = torch.as_tensor(np.ascontiguousarray(x_grid[perm]))
    if stride_pad:
        t = fs.create_field(nvar=nvar, fill=float("nan"))
    else:
        shape = (x.shape[0], fs.nlev) if nvar == 1 else (x.shape[0], fs.nlev, 2)
        t = torch.full(shape, float("nan"), dtype=fs.dtype, device="cuda")
    t.copy_(x.to("cuda"))
    return t


def to_grid(t: torch.Tensor, perm: np.ndarray) -> np.ndarray:
    x = t.detach().cpu().numpy().astype(np.float64)
    out = np.empty_like(x)
    out[perm] = x
    return out


def rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref|| / ||ref||, component-wise maximum for vector fields."""
    if x.ndim == 3:
        return max(rel_l2(x[..., c], ref[..., c]) for c in range(x.shape[-1]))
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def pole_mask(om) -> np.ndarray:
    """Grid-order mask of the first and last grid rows (the pole-row nodes,
    evaluated by the kernels' FP64 pole tiles)."""
    V = om.V
    # rows are north to south; a row is the run of nodes sharing its latitude
    first = int(np.argmax(om.lat != om.lat[0]))
    last = int(np.argmax(om.lat[::-1] != om.lat[-1]))
    m = np.zeros(V, dtype=bool)
    m[:first] = True
    m[V - last:] = True
    return m


def error_stats(x: np.ndarray, ref: np.ndarray, pole: np.ndarray) -> dict:
    """Per-op error figures against the oracle, component-wise maximum for
    vector fields:
      rel_l2      ||x - ref||_2 / ||ref||_2 over all node-levels;
      max_rel     max |x - ref| / max |ref| (the per-node maximum error,
                  scaled by the field's largest value);
      max_abs     max |x - ref|;
      pole_rel_l2 relative L2 over the pole-row nodes alone."""
    if x.ndim == 3:
        parts = [error_stats(x[..., c], ref[..., c], pole) for c in range(x.shape[-1])]
        return {k: max(p[k] for p in parts) for k in parts[0]}
    d = x - ref
    return {"rel_l2": float(np.linalg.norm(d.ravel()) / np.linalg.norm(ref.ravel())),
            "max_rel": float(np.abs(d).max() / np.abs(ref).max()),
            "max_abs": float(np.abs(d).max()),
            "pole_rel_l2": float(np.linalg.norm(d[pole].ravel()) / np.linalg.norm(ref[pole].ravel()))}


def oracle_op(om, op: str, x: np.ndarray) -> np.ndarray:
    return {"grad": oracle.grad, "div": oracle.div, "curl": oracle.curl, "lap": oracle.lap}[op](om, x)


def run_op(meth, fs, op: str, xin: torch.Tensor, scratch=None) -> torch.Tensor:
    nout = 2 if op == "grad" else 1
    out = fs.create_field(nvar=nout, fill=float("nan"))
    nabla.apply(meth, op, xin, out, scratch=scratch)
    torch.cuda.synchronize()
    assert nabla.device_status() == 0, "a kernel recorded a device error"
    return out
