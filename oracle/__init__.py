"""Plain FP64 CPU oracle for the median-dual nabla operators.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA path; the C source it wraps (``nabla_oracle.c``) is
compiled with gcc into ``oracle/_build/libnabla_oracle.so``.

Everything here is in the original grid order (rows north to south, points
west to east, Sec. 4.2.3 / Listing 5) and uses the layout of the paper's
NodeColumns function space (a vertical column contiguous, Sec. 4.5 Fig. 31):
scalar fields ``[node][level]``, vector fields ``[node][level][2]`` with the
local (east, north) components innermost.

Pins: see ``tests/test_oracle_*.py``.  Each function below names the passage
of the paper it follows; the operator formulas are readings (the paper names
the operators and the edge-based finite-volume method, Sec. 4.7, Fig. 33, but
prints no formula).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nabla_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libnabla_oracle.so")

EARTH_RADIUS_M = 6.37122e6


def build(force: bool = False) -> str:
    """Compile the oracle's C source with gcc (plain -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_L = ctypes.c_long


def _declare(L: ctypes.CDLL) -> None:
    L.or_num_nodes.restype = _L
    L.or_num_nodes.argtypes = [ctypes.c_int]
    L.or_num_triangles.restype = _L
    L.or_num_triangles.argtypes = [ctypes.c_int]
    L.or_row_nx.argtypes = [ctypes.c_int, _P]
    L.or_gaussian_rows.argtypes = [ctypes.c_int, _P, _P]
    L.or_grid_lonlat.argtypes = [ctypes.c_int, _P, _P]
    L.or_triangulate.argtypes = [ctypes.c_int, _P]
    L.or_num_nodes_pl.restype = _L
    L.or_num_nodes_pl.argtypes = [ctypes.c_int, _P]
    L.or_grid_lonlat_pl.argtypes = [ctypes.c_int, _P, _P, _P]
    L.or_triangulate_pl.argtypes = [ctypes.c_int, _P, _P]
    L.or_edges.restype = _L
    L.or_edges.argtypes = [_L, _L, _P, _P, _P]
    L.or_node_edges.argtypes = [_L, _L, _P, _P, _P]
    L.or_frames.argtypes = [_L, _P, _P, _P, _P]
    L.or_geometry.argtypes = [_L, _L, _L, _P, _P, _P, _P, _P, ctypes.c_double, _P, _P, _P]
    for name in ("or_grad", "or_div", "or_curl"):
        getattr(L, name).argtypes = [_L, _P, _P, _P, _P, _P, _P, _P, _L, _P, _P]
    L.or_lap.argtypes = [_L, _P, _P, _P, _P, _P, _P, _P, _L, _P, _P, _P]
    L.or_bruteforce_node.argtypes = [_L, _L, _P, _P, _P, ctypes.c_double, _L, ctypes.c_int,
                                     _P, _P, _P, _P]
    L.or_set_mutation.argtypes = [ctypes.c_int]
    L.or_get_mutation.restype = ctypes.c_int


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def set_mutation(m: int) -> None:
    """Plant mistake number ``m`` in the oracle (0 = none).  Tests only."""
    lib().or_set_mutation(int(m))


# ------------------------------------------------------------------- grid

def num_nodes(N: int) -> int:
    """V = sum over the 2N rows of 20 + 4j (Listing 6, Sec. 4.2.3.7)."""
    return int(lib().or_num_nodes(N))


def row_nx(N: int) -> np.ndarray:
    nx = np.zeros(2 * N, dtype=np.int32)
    lib().or_row_nx(N, _ptr(nx))
    return nx


def regular_nx(N: int) -> np.ndarray:
    """Points per parallel of the regular Gaussian grid F<N>: 4N on each of
    the 2N parallels (Sec. 4.2.3.6)."""
    return np.full(2 * N, 4 * N, dtype=np.int32)


def _pl_array(pl) -> np.ndarray:
    """A reduced Gaussian grid's PL array (points per parallel, north to
    south, Sec. 4.2.3.7): an even number of rows, at least 3 points each."""
    nx = np.ascontiguousarray(pl, dtype=np.int32)
    if nx.ndim != 1 or nx.size < 2 or nx.size % 2 or (nx < 3).any():
        raise ValueError("PL array: an even number of parallels, each with at least 3 points")
    return nx


def gaussian_rows(N: int):
    """Roots of P_2N north to south and Gauss weights (Sec. 4.2.3.5)."""
    mu = np.zeros(2 * N)
    w = np.zeros(2 * N)
    lib().or_gaussian_rows(N, _ptr(mu), _ptr(w))
    return mu, w


def grid_lonlat(N: int, pl=None):
    """(lat, lon) in radians per node, original order (Sec. 4.2, 4.2.3.5);
    pl: the PL array of another reduced Gaussian grid with 2N parallels
    (default: the octahedral O<N>)."""
    if pl is None:
        V = num_nodes(N)
        lat = np.zeros(V)
        lon = np.zeros(V)
        lib().or_grid_lonlat(N, _ptr(lat), _ptr(lon))
        return lat, lon
    nx = _pl_array(pl)
    V = int(lib().or_num_nodes_pl(nx.size, _ptr(nx)))
    lat = np.zeros(V)
    lon = np.zeros(V)
    lib().or_grid_lonlat_pl(nx.size, _ptr(nx), _ptr(lat), _ptr(lon))
    return lat, lon


# ------------------------------------------------------------------- mesh

def triangulate(N: int, pl=None) -> np.ndarray:
    """[F][3] counter-clockwise triangles (reading of Sec. 4.3, Fig. 25b);
    pl as for grid_lonlat."""
    if pl is None:
        F = int(lib().or_num_triangles(N))
        tri = np.zeros((F, 3), dtype=np.int32)
        lib().or_triangulate(N, _ptr(tri))
        return tri
    nx = _pl_array(pl)
    F = 2 * int(nx.sum()) - 4
    tri = np.zeros((F, 3), dtype=np.int32)
    lib().or_triangulate_pl(nx.size, _ptr(nx), _ptr(tri))
    return tri


def edges(V: int, tri: np.ndarray):
    """Unique edges (a<b) with their (left, right) triangles."""
    F = tri.shape[0]
    E = 3 * F // 2
    edge = np.zeros((E, 2), dtype=np.int32)
    etri = np.zeros((E, 2), dtype=np.int32)
    got = lib().or_edges(V, F, _ptr(tri), _ptr(edge), _ptr(etri))
    if got != E:
        raise ValueError(f"mesh is not a closed oriented surface (edges {got} != {E})")
    return edge, etri


def node_edges(V: int, edge: np.ndarray):
    E = edge.shape[0]
    ptr = np.zeros(V + 1, dtype=np.int64)
    lst = np.zeros(2 * E, dtype=np.int32)
    lib().or_node_edges(V, E, _ptr(edge), _ptr(ptr), _ptr(lst))
    return ptr, lst


@dataclass
class Mesh:
    """Oracle mesh + median-dual geometry of O<N> (original node order)."""
    N: int
    R: float
    lat: np.ndarray
    lon: np.ndarray
    tri: np.ndarray
    edge: np.ndarray
    etri: np.ndarray
    nptr: np.ndarray
    nlist: np.ndarray
    east: np.ndarray
    north: np.ndarray
    vol: np.ndarray
    S: np.ndarray
    T: np.ndarray

    @property
    def V(self) -> int:
        return self.lat.shape[0]

    @property
    def E(self) -> int:
        return self.edge.shape[0]

    @property
    def F(self) -> int:
        return self.tri.shape[0]


def build_mesh(N: int, R: float = EARTH_RADIUS_M, pl=None) -> Mesh:
    """Grid -> mesh -> median-dual geometry (Sec. 4.2, 4.3, 4.7).  pl: the
    PL array of a reduced Gaussian grid with 2N parallels (Sec. 4.2.3.7;
    default: octahedral O<N>)."""
    L = lib()
    lat, lon = grid_lonlat(N, pl)
    V = lat.shape[0]
    tri = triangulate(N, pl)
    edge, etri = edges(V, tri)
    nptr, nlist = node_edges(V, edge)
    east = np.zeros((V, 3))
    north = np.zeros((V, 3))
    L.or_frames(V, _ptr(lat), _ptr(lon), _ptr(east), _ptr(north))
    E = edge.shape[0]
    vol = np.zeros(V)
    S = np.zeros((E, 3))
    T = np.zeros((E, 3))
    L.or_geometry(V, tri.shape[0], E, _ptr(lat), _ptr(lon), _ptr(tri), _ptr(edge), _ptr(etri),
                  float(R), _ptr(vol), _ptr(S), _ptr(T))
    return Mesh(N, float(R), lat, lon, tri, edge, etri, nptr, nlist, east, north, vol, S, T)


# -------------------------------------------------------------- operators

def _levels(f: np.ndarray, vector: bool):
    f = np.ascontiguousarray(f, dtype=np.float64)
    if vector:
        if f.ndim == 2:
            f = f.reshape(f.shape[0], 1, 2)
        assert f.ndim == 3 and f.shape[2] == 2
    else:
        if f.ndim == 1:
            f = f.reshape(-1, 1)
        assert f.ndim == 2
    return f, f.shape[1]


def grad(m: Mesh, f: np.ndarray) -> np.ndarray:
    """Gradient, horizontal components (Sec. 4.7, Listing 12): [V][L] -> [V][L][2]."""
    f, L = _levels(f, False)
    out = np.zeros((m.V, L, 2))
    lib().or_grad(m.V, _ptr(m.nptr), _ptr(m.nlist), _ptr(m.edge), _ptr(m.S), _ptr(m.vol),
                  _ptr(m.east), _ptr(m.north), L, _ptr(f), _ptr(out))
    return out


def div(m: Mesh, uv: np.ndarray) -> np.ndarray:
    """Divergence (Sec. 4.7, Fig. 33): [V][L][2] -> [V][L]."""
    uv, L = _levels(uv, True)
    out = np.zeros((m.V, L))
    lib().or_div(m.V, _ptr(m.nptr), _ptr(m.nlist), _ptr(m.edge), _ptr(m.S), _ptr(m.vol),
                 _ptr(m.east), _ptr(m.north), L, _ptr(uv), _ptr(out))
    return out


def curl(m: Mesh, uv: np.ndarray) -> np.ndarray:
    """Vertical curl (Sec. 4.7, Fig. 33): [V][L][2] -> [V][L]."""
    uv, L = _levels(uv, True)
    out = np.zeros((m.V, L))
    lib().or_curl(m.V, _ptr(m.nptr), _ptr(m.nlist), _ptr(m.edge), _ptr(m.T), _ptr(m.vol),
                  _ptr(m.east), _ptr(m.north), L, _ptr(uv), _ptr(out))
    return out


def lap(m: Mesh, f: np.ndarray) -> np.ndarray:
    """Laplacian = div(grad) (Sec. 4.7, Fig. 33): [V][L] -> [V][L]."""
    f, L = _levels(f, False)
    tmp = np.zeros((m.V, L, 2))
    out = np.zeros((m.V, L))
    lib().or_lap(m.V, _ptr(m.nptr), _ptr(m.nlist), _ptr(m.edge), _ptr(m.S), _ptr(m.vol),
                 _ptr(m.east), _ptr(m.north), L, _ptr(f), _ptr(tmp), _ptr(out))
    return out


def bruteforce_node(m: Mesh, i: int, op: str, field: np.ndarray):
    """Direct walk of node i's dual cell (no edge list): returns (value, volume).

    op 'grad' takes a scalar per node; 'div' and 'curl' take [V][2]."""
    code = {"grad": 0, "div": 1, "curl": 2}[op]
    out = np.zeros(2)
    vol = np.zeros(1)
    f = np.ascontiguousarray(field, dtype=np.float64)
    dummy = np.zeros(1)
    lib().or_bruteforce_node(m.V, m.F, _ptr(m.lat), _ptr(m.lon), _ptr(m.tri), m.R, int(i), code,
                             _ptr(f) if code == 0 else _ptr(dummy),
                             _ptr(f) if code != 0 else _ptr(dummy), _ptr(out), _ptr(vol))
    return (out if code == 0 else out[0]), float(vol[0])
