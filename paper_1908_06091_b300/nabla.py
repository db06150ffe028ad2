"""Thin ctypes binding of the C ABI in ``include/nabla_b300.h``.

Argument marshalling only: every step of the operators runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.  Loading fails
loudly if the shared object has not been built (``build.py``); there is no
CPU fallback.

Concept chain (Sec. 4.7, Listing 12):

    grid = Grid(1280)                  # O1280 (Sec. 4.2.3.7)
    mesh = Mesh(grid)                  # structured triangulation (Sec. 4.3)
    method = Method(mesh)              # fvm::Method: median-dual geometry
    fs = NodeColumns(method, 137, torch.float32)   # Sec. 4.5
    f = fs.create_field()              # [V, 137] view of a [V, Lp] tensor
    g = fs.create_field(nvar=2)        # [V, 137, 2]
    gradient(method, f, g)             # fvm::Nabla::gradient
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# NB_LIBRARY=debug loads the bounds-checked build (build.py, variant "debug")
LIB_PATH = os.path.join(_HERE, "_lib", "libnabla_b300_debug.so" if os.environ.get("NB_LIBRARY") == "debug"
                        else "libnabla_b300.so")

NB_OK, NB_EINVAL, NB_ESHAPE, NB_EDTYPE, NB_EOOM, NB_ECUDA, NB_ETIMEOUT, NB_EBUDGET = range(8)
NB_F32, NB_F64 = 0, 1
OP_GRAD, OP_DIV, OP_CURL, OP_LAP = 0, 1, 2, 3
OPS = {"grad": OP_GRAD, "div": OP_DIV, "curl": OP_CURL, "lap": OP_LAP}
KERNEL_AUTO, KERNEL_DIRECT, KERNEL_TILED, KERNEL_EDGE = 0, 1, 2, 3
LAP_TWO_PASS, LAP_FUSED = 0, 1
EARTH_RADIUS_M = 6.37122e6


class NablaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[nabla status {code}] {msg}")
        self.code = code


class nb_field(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("nvar", ctypes.c_int32),
                ("nnodes", ctypes.c_int64), ("nlev", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("node_stride", ctypes.c_int64), ("lev_stride", ctypes.c_int64)]


class nb_batch_item(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("reserved", ctypes.c_int32), ("method", ctypes.c_void_p),
                ("inp", nb_field), ("out", nb_field)]


class nb_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("N", ctypes.c_int32), ("nlev", ctypes.c_int32),
                ("nfields", ctypes.c_int32), ("dtype", ctypes.c_int32), ("keep_output", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


class nb_allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("release", _RELEASE_FN)]


class nb_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("node_levels", ctypes.c_int64), ("bytes", ctypes.c_int64)]


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64P = ctypes.POINTER(ctypes.c_int64)
_FP = ctypes.POINTER(nb_field)

# name -> argtypes; every function returns int except the two string getters
SIGNATURES = {
    "nb_grid_create_octahedral": [_I, ctypes.POINTER(_P)],
    "nb_grid_create_regular": [_I, ctypes.POINTER(_P)],
    "nb_grid_create_reduced": [_I, _P, ctypes.POINTER(_P)],
    "nb_grid_create_named": [ctypes.c_char_p, ctypes.POINTER(_P)],
    "nb_grid_pl": [_P, _P],
    "nb_grid_release": [_P],
    "nb_grid_size": [_P, _I64P],
    "nb_grid_gaussian_number": [_P, ctypes.POINTER(_I)],
    "nb_grid_lonlat": [_P, _P],
    "nb_mesh_create": [_P, _I, ctypes.POINTER(_P)],
    "nb_partition_equal_regions": [_P, _I, _P, _P, ctypes.POINTER(ctypes.c_int32)],
    "nb_partition_halo": [_P, _P, _I, _I64P, _P, _I64P, _P],
    "nb_mesh_release": [_P],
    "nb_mesh_sizes": [_P, _I64P, _I64P, _I64P],
    "nb_mesh_permutation": [_P, _P],
    "nb_mesh_triangles": [_P, _P],
    "nb_mesh_edges": [_P, _P],
    "nb_mesh_cap_begin": [_P, _I64P],
    "nb_mesh_lap_plan": [_P, _I] + [ctypes.POINTER(ctypes.c_int32)] * 4,
    "nb_check_tile_plan": [_P, ctypes.c_int32, _P, _P, _P, _P],
    "nb_check_slot_lists": [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int64],
    "nb_mesh_csr": [_P, _P, _P],
    "nb_mesh_node_pairs": [_P, _P],
    "nb_mesh_tile_plan": [_P, _I, _I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                          _I64P, _P, _P, _P, _P],
    "nb_method_create": [_P, ctypes.c_double, ctypes.POINTER(_P)],
    "nb_method_release": [_P],
    "nb_method_dual_volumes": [_P, _P],
    "nb_method_device_bytes": [_P, _I64P],
    "nb_method_set_kernel": [_P, _I, _I],
    "nb_method_set_compensated": [_P, _I],
    "nb_method_set_staging": [_P, _I, _I],
    "nb_method_set_wait_limit": [_P, ctypes.c_int64],
    "nb_method_set_item_shape": [_P, _I, _I],
    "nb_method_set_node_pairs": [_P, _I],
    "nb_method_set_laplacian_route": [_P, _I],
    "nb_fs_nodecolumns": [_P, _I, _I, ctypes.POINTER(_P)],
    "nb_fs_release": [_P],
    "nb_fs_level_stride": [_P, _I64P],
    "nb_field_view": [_P, _P, _I, ctypes.c_int64, ctypes.c_int64, _FP],
    "nb_nabla_gradient": [_P, _FP, _FP, _P],
    "nb_nabla_divergence": [_P, _FP, _FP, _P],
    "nb_nabla_curl": [_P, _FP, _FP, _P],
    "nb_nabla_laplacian": [_P, _FP, _FP, _FP, _P],
    "nb_nabla_divcurl": [_P, _FP, _FP, _FP, _P],
    "nb_nabla_gradlap": [_P, _FP, _FP, _FP, _P],
    "nb_field_upload": [_FP, _P, _P],
    "nb_field_reduce": [_P, _FP, _I, _P, _P],
    "nb_field_download": [_P, _FP, _P],
    "nb_nabla_apply": [_P, _I, _FP, _FP, _FP, _P],
    "nb_nabla_laplacian_noalloc": [_P, _FP, _FP, _P],
    "nb_nabla_apply_host": [_P, _I, _P, _P, _FP, _FP, _FP, _P],
    "nb_set_allocator": [ctypes.POINTER(nb_allocator)],
    "nb_launch_count": [_I64P],
    "nb_probe_fp64_rate": [ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "nb_device_status": [_I, ctypes.POINTER(ctypes.c_int32)],
    "nb_batch_create": [_P, _I, ctypes.POINTER(_P)],
    "nb_batch_release": [_P],
    "nb_batch_tune": [_P, _P],
    "nb_batch_run": [_P, _P],
    "nb_batch_set_compensated": [_P, _I],
    "nb_batch_info": [_P, _I64P, _I64P, _P, _P],
    "nb_batch_graph_nodes": [_P, _P, _P],
    "nb_server_create": [ctypes.c_int64, _I, _I, ctypes.POINTER(_P)],
    "nb_server_release": [_P],
    "nb_server_add_grid": [_P, _P, _P, _P],
    "nb_server_submit": [_P, ctypes.POINTER(nb_request), ctypes.POINTER(ctypes.c_uint64)],
    "nb_server_wait": [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(nb_result)],
    "nb_server_poll": [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(nb_result)],
    "nb_server_output": [_P, ctypes.c_uint64, _P, ctypes.c_int64],
    "nb_server_input": [_P, ctypes.c_uint64, _P, ctypes.c_int64],
    "nb_server_inject_failure": [_P, ctypes.c_uint64, ctypes.c_int32],
    "nb_server_stats": [_P, _I64P, _I64P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "nb_server_run_trace": [_P, ctypes.POINTER(nb_request), _P, _I, ctypes.POINTER(nb_result)],
}


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"nabla_b300 CUDA library missing: {LIB_PATH} "
                               "(run `python -m paper_1908_06091_b300.build`)")
        L = ctypes.CDLL(LIB_PATH)
        L.nb_version.restype = ctypes.c_char_p
        L.nb_last_error.restype = ctypes.c_char_p
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != NB_OK:
        raise NablaError(rc, lib().nb_last_error().decode())


def version() -> str:
    return lib().nb_version().decode()


def launch_count() -> int:
    c = ctypes.c_int64()
    check(lib().nb_launch_count(ctypes.byref(c)))
    return c.value


def probe_fp64_rate(iters: int = 40000, stream=None):
    """(TFLOP/s, ms) of the device's FP64 FMA-chain probe (nb_probe_fp64_rate)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    check(lib().nb_probe_fp64_rate(int(iters), ctypes.c_void_p(_stream(stream)), ctypes.byref(tf),
                                   ctypes.byref(ms)))
    return tf.value, ms.value


def device_status(clear: bool = False) -> int:
    """0 if every kernel ran normally, else the NB_* code a kernel recorded."""
    c = ctypes.c_int32()
    check(lib().nb_device_status(1 if clear else 0, ctypes.byref(c)))
    return c.value


# callbacks of the installed allocator, kept alive while the library may call them
_allocator_keep = []


def _torch_alloc(ctx, nbytes, stream):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # out of memory: the library call fails with NB_EOOM
        return None


def _torch_release(ctx, ptr, nbytes, stream):
    torch.cuda.caching_allocator_delete(ptr)


def use_torch_allocator(on: bool = True) -> None:
    """Serve the library's own device buffers (method geometry, tile plans,
    batch tables, Laplacian scratch) from torch's caching allocator, or, with
    on=False, from the CUDA runtime again.  Objects keep the allocator that
    was current when they were created."""
    if on:
        a = nb_allocator(None, _ALLOC_FN(_torch_alloc), _RELEASE_FN(_torch_release))
        check(lib().nb_set_allocator(ctypes.byref(a)))
        _allocator_keep.append(a)
    else:
        check(lib().nb_set_allocator(None))


class _Handle:
    _release = ""

    def __init__(self):
        self._h = ctypes.c_void_p()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            getattr(_lib, self._release)(h)
            self._h = ctypes.c_void_p()

    @property
    def handle(self):
        return self._h


class Grid(_Handle):
    """Reduced Gaussian grid (Sec. 4.2.3): Grid(N) is the octahedral O<N>;
    Grid.regular(N) the regular F<N>; Grid.reduced(pl) any PL array;
    Grid.named("O1280") / Grid.named("F640") by name."""
    _release = "nb_grid_release"

    def __init__(self, N: int = 0, *, _make=None):
        super().__init__()
        if _make is None:
            check(lib().nb_grid_create_octahedral(int(N), ctypes.byref(self._h)))
        else:
            check(_make(ctypes.byref(self._h)))
        n = ctypes.c_int()
        check(lib().nb_grid_gaussian_number(self._h, ctypes.byref(n)))
        self.N = n.value

    @classmethod
    def regular(cls, N: int) -> "Grid":
        return cls(_make=lambda out: lib().nb_grid_create_regular(int(N), out))

    @classmethod
    def reduced(cls, pl) -> "Grid":
        arr = np.ascontiguousarray(pl, dtype=np.int32)
        return cls(_make=lambda out: lib().nb_grid_create_reduced(int(arr.size), arr.ctypes.data, out))

    @classmethod
    def named(cls, name: str) -> "Grid":
        return cls(_make=lambda out: lib().nb_grid_create_named(name.encode(), out))

    def pl(self) -> np.ndarray:
        """Points per row, north to south."""
        out = np.zeros(2 * self.N, dtype=np.int32)
        check(lib().nb_grid_pl(self._h, out.ctypes.data))
        return out

    @property
    def size(self) -> int:
        v = ctypes.c_int64()
        check(lib().nb_grid_size(self._h, ctypes.byref(v)))
        return v.value

    def lonlat(self) -> np.ndarray:
        out = np.zeros((self.size, 2))
        check(lib().nb_grid_lonlat(self._h, out.ctypes.data))
        return out


def equal_regions(grid: "Grid", nparts: int):
    """EqualRegions partition (Sec. 4.2.4.2): part id per grid point (grid
    order) and the regions per band, north to south."""
    nz = ctypes.c_int32()
    check(lib().nb_partition_equal_regions(grid.handle, int(nparts), None, None, ctypes.byref(nz)))
    zones = np.zeros(nz.value, dtype=np.int32)
    part = np.zeros(grid.size, dtype=np.int32)
    check(lib().nb_partition_equal_regions(grid.handle, int(nparts), part.ctypes.data, zones.ctypes.data,
                                           ctypes.byref(nz)))
    return part, zones


def partition_halo(mesh: "Mesh", part_mesh_order: np.ndarray, p: int):
    """Owned nodes and one-ring halo of partition p (Sec. 4.4), both in
    functionspace order, from a part id per node in functionspace order."""
    part = np.ascontiguousarray(part_mesh_order, dtype=np.int32)
    no, nh = ctypes.c_int64(), ctypes.c_int64()
    check(lib().nb_partition_halo(mesh.handle, part.ctypes.data, int(p), ctypes.byref(no), None,
                                  ctypes.byref(nh), None))
    owned = np.zeros(no.value, dtype=np.int32)
    halo = np.zeros(nh.value, dtype=np.int32)
    check(lib().nb_partition_halo(mesh.handle, part.ctypes.data, int(p), ctypes.byref(no), owned.ctypes.data,
                                  ctypes.byref(nh), halo.ctypes.data))
    return owned, halo


class Mesh(_Handle):
    """Structured triangulation of a grid (Sec. 4.3), Hilbert-ordered by default."""
    _release = "nb_mesh_release"

    def __init__(self, grid: Grid, reorder: int = 1):
        super().__init__()
        self.grid = grid
        check(lib().nb_mesh_create(grid.handle, int(reorder), ctypes.byref(self._h)))
        v, e, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().nb_mesh_sizes(self._h, ctypes.byref(v), ctypes.byref(e), ctypes.byref(t)))
        self.V, self.E, self.F = v.value, e.value, t.value
        c = ctypes.c_int64()
        check(lib().nb_mesh_cap_begin(self._h, ctypes.byref(c)))
        self.cap_begin = c.value

    def permutation(self) -> np.ndarray:
        out = np.zeros(self.V, dtype=np.int32)
        check(lib().nb_mesh_permutation(self._h, out.ctypes.data))
        return out

    def triangles(self) -> np.ndarray:
        out = np.zeros((self.F, 3), dtype=np.int32)
        check(lib().nb_mesh_triangles(self._h, out.ctypes.data))
        return out

    def edges(self) -> np.ndarray:
        out = np.zeros((self.E, 2), dtype=np.int32)
        check(lib().nb_mesh_edges(self._h, out.ctypes.data))
        return out

    def csr(self):
        rp = np.zeros(self.V + 1, dtype=np.int64)
        nb = np.zeros(2 * self.E, dtype=np.int32)
        check(lib().nb_mesh_csr(self._h, rp.ctypes.data, nb.ctypes.data))
        return rp, nb

    def node_pairs(self) -> np.ndarray:
        """Partner of every paired node (-1: unpaired), functionspace order."""
        mate = np.zeros(self.V, dtype=np.int32)
        check(lib().nb_mesh_node_pairs(self._h, mate.ctypes.data))
        return mate

    def lap_plan(self, nlev: int):
        """(tiles, main tiles, max g-nodes, fits) of the single-pass
        Laplacian's plan for FP32 columns of nlev levels (host only)."""
        v = [ctypes.c_int32() for _ in range(4)]
        check(lib().nb_mesh_lap_plan(self._h, int(nlev), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def tile_plan(self, rcap: int, nmax: int = 256):
        """(node0, halo_ptr, halo, lnbr, ntiles_main) of the staged kernels' plan."""
        nt, nm, nh = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(lib().nb_mesh_tile_plan(self._h, rcap, nmax, ctypes.byref(nt), ctypes.byref(nm),
                                      ctypes.byref(nh), None, None, None, None))
        node0 = np.zeros(nt.value + 1, dtype=np.int32)
        hptr = np.zeros(nt.value + 1, dtype=np.int32)
        halo = np.zeros(max(nh.value, 1), dtype=np.int32)
        lnbr = np.zeros(2 * self.E, dtype=np.uint16)
        check(lib().nb_mesh_tile_plan(self._h, rcap, nmax, ctypes.byref(nt), ctypes.byref(nm),
                                      ctypes.byref(nh), node0.ctypes.data, hptr.ctypes.data,
                                      halo.ctypes.data, lnbr.ctypes.data))
        return node0, hptr, halo[:nh.value], lnbr, nm.value

    def check_tile_plan(self, node0, halo_ptr, halo, lnbr) -> None:
        """Raise NablaError unless the plan (format of tile_plan) is valid
        (nb_check_tile_plan)."""
        n0 = np.ascontiguousarray(node0, dtype=np.int32)
        hp = np.ascontiguousarray(halo_ptr, dtype=np.int32)
        h = np.ascontiguousarray(halo if len(halo) else np.zeros(1), dtype=np.int32)
        ln = np.ascontiguousarray(lnbr, dtype=np.uint16)
        check(lib().nb_check_tile_plan(self._h, len(n0) - 1, n0.ctypes.data, hp.ctypes.data, h.ctypes.data,
                                       ln.ctypes.data))

    def check_slot_lists(self, node0, slot_ptr, npairs, slots) -> None:
        """Raise NablaError unless the slot lists of a staged plan are valid
        (nb_check_slot_lists)."""
        n0 = np.ascontiguousarray(node0, dtype=np.int32)
        sp = np.ascontiguousarray(slot_ptr, dtype=np.int32)
        npr = np.ascontiguousarray(npairs, dtype=np.int32)
        sl = np.ascontiguousarray(slots, dtype=np.uint32)
        n = len(sl)
        if n == 0:
            sl = np.zeros(4, dtype=np.uint32)
        check(lib().nb_check_slot_lists(self._h, len(n0) - 1, n0.ctypes.data, sp.ctypes.data, npr.ctypes.data,
                                        sl.ctypes.data, n))


class Method(_Handle):
    """fvm::Method (Sec. 4.7): median-dual geometry resident on the current device."""
    _release = "nb_method_release"

    def __init__(self, mesh: Mesh, radius: float = EARTH_RADIUS_M):
        super().__init__()
        self.mesh = mesh
        self.radius = float(radius)
        check(lib().nb_method_create(mesh.handle, self.radius, ctypes.byref(self._h)))

    def dual_volumes(self) -> np.ndarray:
        out = np.zeros(self.mesh.V)
        check(lib().nb_method_dual_volumes(self._h, out.ctypes.data))
        return out

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        check(lib().nb_method_device_bytes(self._h, ctypes.byref(b)))
        return b.value

    def set_kernel(self, variant: int, tile_nodes: int = 0) -> None:
        check(lib().nb_method_set_kernel(self._h, int(variant), int(tile_nodes)))

    def set_staging(self, nstages: int, stage_kb: int) -> None:
        check(lib().nb_method_set_staging(self._h, int(nstages), int(stage_kb)))

    def set_compensated(self, on: bool) -> None:
        check(lib().nb_method_set_compensated(self._h, 1 if on else 0))

    def set_laplacian_route(self, route: int) -> None:
        """LAP_TWO_PASS (default) or LAP_FUSED (single-pass Laplacian for
        the FP32 staged path); see nb_method_set_laplacian_route."""
        check(lib().nb_method_set_laplacian_route(self._h, int(route)))

    def set_item_shape(self, units: int = 0, aligned: int = -1) -> None:
        """Item shape of the staged div / curl kernels (0 / -1: chosen by
        the library); see nb_method_set_item_shape."""
        check(lib().nb_method_set_item_shape(self._h, int(units), int(aligned)))

    def set_node_pairs(self, mode: int = -1) -> None:
        """Node pairs in the staged kernels: 1 in every pass, 0 in none, -1
        (the default) in all but the fused div+curl pass; see
        nb_method_set_node_pairs."""
        check(lib().nb_method_set_node_pairs(self._h, int(mode)))

    def set_wait_limit(self, limit_ns: int = -1) -> None:
        """Limit of the staged kernels' pipeline waits in ns (-1 = default
        2 s; 0 = test once).  A wait that runs out records NB_ETIMEOUT in the
        device status word."""
        check(lib().nb_method_set_wait_limit(self._h, int(limit_ns)))


_DT = {torch.float32: NB_F32, torch.float64: NB_F64}


class NodeColumns(_Handle):
    """NodeColumns function space (Sec. 4.5): nlev levels, padded stride Lp."""
    _release = "nb_fs_release"

    def __init__(self, method: Method, nlev: int, dtype=torch.float32):
        super().__init__()
        self.method = method
        self.nlev = int(nlev)
        self.dtype = dtype
        check(lib().nb_fs_nodecolumns(method.handle, self.nlev, _DT[dtype], ctypes.byref(self._h)))
        lp = ctypes.c_int64()
        check(lib().nb_fs_level_stride(self._h, ctypes.byref(lp)))
        self.lp = lp.value

    def create_field(self, nvar: int = 1, device="cuda", fill=None) -> torch.Tensor:
        """[V, nlev] (nvar 1) or [V, nlev, 2] view of a padded [V, Lp(, 2)] tensor."""
        V = self.method.mesh.V
        shape = (V, self.lp) if nvar == 1 else (V, self.lp, 2)
        t = torch.empty(shape, dtype=self.dtype, device=device) if fill is None else \
            torch.full(shape, float(fill), dtype=self.dtype, device=device)
        return t[:, :self.nlev]


def field_view(t: torch.Tensor, nvar: int) -> nb_field:
    """nb_field describing a [V, L] or [V, L, 2] tensor (levels contiguous)."""
    if t.dtype not in _DT:
        raise TypeError(f"unsupported dtype {t.dtype}")
    f = nb_field()
    f.data = t.data_ptr()
    f.dtype = _DT[t.dtype]
    f.nvar = nvar
    f.nnodes = t.shape[0]
    f.nlev = t.shape[1]
    f.reserved = 0
    f.node_stride = t.stride(0)
    f.lev_stride = t.stride(1)
    if nvar == 1 and t.dim() != 2:
        raise ValueError("scalar field must be [V, L]")
    if nvar == 2 and (t.dim() != 3 or t.shape[2] != 2 or t.stride(2) != 1):
        raise ValueError("vector field must be [V, L, 2] with components innermost")
    return f


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def apply(method: Method, op, inp: torch.Tensor, out: torch.Tensor, scratch=None, stream=None):
    """fvm::Nabla operator `op` ('grad', 'div', 'curl', 'lap' or an OP_* code)."""
    code = OPS[op] if isinstance(op, str) else int(op)
    nin = 2 if code in (OP_DIV, OP_CURL) else 1
    nout = 2 if code == OP_GRAD else 1
    fi, fo = field_view(inp, nin), field_view(out, nout)
    fs = ctypes.byref(field_view(scratch, 2)) if scratch is not None else None
    check(lib().nb_nabla_apply(method.handle, code, ctypes.byref(fi), ctypes.byref(fo), fs,
                               ctypes.c_void_p(_stream(stream))))
    return out


def gradient(method, f, g, stream=None):
    return apply(method, OP_GRAD, f, g, stream=stream)


def divergence(method, uv, d, stream=None):
    return apply(method, OP_DIV, uv, d, stream=stream)


def curl(method, uv, z, stream=None):
    return apply(method, OP_CURL, uv, z, stream=stream)


def laplacian(method, f, lap, scratch=None, stream=None):
    return apply(method, OP_LAP, f, lap, scratch=scratch, stream=stream)


REDUCE = {"min": 0, "max": 1, "sum": 2, "area_mean": 3, "area_rms": 4}


def reduce(method, field: torch.Tensor, kind: str, nvar: int = 1, stream=None) -> np.ndarray:
    """Per-level (and per-component) reduction over the nodes, in FP64:
    min, max, sum, area_mean or area_rms (dual-volume weighted)."""
    fv = field_view(field, nvar)
    out = np.zeros((fv.nlev, nvar))
    check(lib().nb_field_reduce(method.handle, ctypes.byref(fv), REDUCE[kind], out.ctypes.data,
                                ctypes.c_void_p(_stream(stream))))
    return out if nvar == 2 else out[:, 0]


def upload(field: torch.Tensor, host: torch.Tensor, nvar: int, stream=None):
    """Enqueue the copy of a whole host field (laid out like `field`'s base
    storage, node stride included) into the device field; returns at once."""
    fv = field_view(field, nvar)
    check(lib().nb_field_upload(ctypes.byref(fv), ctypes.c_void_p(host.data_ptr()),
                                ctypes.c_void_p(_stream(stream))))


def download(host: torch.Tensor, field: torch.Tensor, nvar: int, stream=None):
    """Enqueue the copy of a whole device field to host memory; returns at once."""
    fv = field_view(field, nvar)
    check(lib().nb_field_download(ctypes.c_void_p(host.data_ptr()), ctypes.byref(fv),
                                  ctypes.c_void_p(_stream(stream))))


def gradlap(method, f, g, lap, stream=None):
    """Gradient into g and Laplacian into lap of one field; the Laplacian's
    divergence pass reads g."""
    fi, fg, fl = field_view(f, 1), field_view(g, 2), field_view(lap, 1)
    check(lib().nb_nabla_gradlap(method.handle, ctypes.byref(fi), ctypes.byref(fg), ctypes.byref(fl),
                                 ctypes.c_void_p(_stream(stream))))


def divcurl(method, uv, d, z, stream=None):
    """Divergence into d and curl into z of one wind, in one pass."""
    fi, fd, fz = field_view(uv, 2), field_view(d, 1), field_view(z, 1)
    check(lib().nb_nabla_divcurl(method.handle, ctypes.byref(fi), ctypes.byref(fd), ctypes.byref(fz),
                                 ctypes.c_void_p(_stream(stream))))


class Batch(_Handle):
    """Many nabla operations in one persistent launch replayed from a CUDA graph.

    items: list of (op, method, in_tensor, out_tensor)."""
    _release = "nb_batch_release"

    def __init__(self, items):
        super().__init__()
        self._keep = items  # the tensors must outlive the batch
        arr = (nb_batch_item * len(items))()
        for k, (op, meth, xin, xout) in enumerate(items):
            code = OPS[op] if isinstance(op, str) else int(op)
            nin = 2 if code in (OP_DIV, OP_CURL) else 1
            nout = 2 if code == OP_GRAD else 1
            arr[k].op = code
            arr[k].reserved = 0
            arr[k].method = meth.handle.value
            arr[k].inp = field_view(xin, nin)
            arr[k].out = field_view(xout, nout)
        check(lib().nb_batch_create(arr, len(items), ctypes.byref(self._h)))
        self.n = len(items)

    def tune(self, stream=None):
        check(lib().nb_batch_tune(self._h, ctypes.c_void_p(_stream(stream))))

    def run(self, stream=None):
        check(lib().nb_batch_run(self._h, ctypes.c_void_p(_stream(stream))))

    def set_compensated(self, on: bool):
        check(lib().nb_batch_set_compensated(self._h, 1 if on else 0))

    def info(self):
        u, nl = ctypes.c_int64(), ctypes.c_int64()
        npw = np.zeros(self.n, dtype=np.int32)
        lpb = np.zeros(self.n, dtype=np.int32)
        check(lib().nb_batch_info(self._h, ctypes.byref(u), ctypes.byref(nl), npw.ctypes.data,
                                  lpb.ctypes.data))
        gn, gk = ctypes.c_int64(), ctypes.c_int64()
        check(lib().nb_batch_graph_nodes(self._h, ctypes.byref(gn), ctypes.byref(gk)))
        return {"units": u.value, "node_levels": nl.value, "nodes_per_warp": npw.tolist(),
                "levels_per_block": lpb.tolist(), "graph_nodes": gn.value, "graph_kernels": gk.value}


class Server(_Handle):
    """Continuous-batching request server (see nb_server_* in the header)."""
    _release = "nb_server_release"

    def __init__(self, budget_bytes: int, nstreams: int = 4, max_inflight: int = 16):
        super().__init__()
        self.grids = {}
        check(lib().nb_server_create(int(budget_bytes), int(nstreams), int(max_inflight),
                                     ctypes.byref(self._h)))

    def add_grid(self, method, scalar_basis: np.ndarray, wind_basis: np.ndarray):
        sb = np.ascontiguousarray(scalar_basis, dtype=np.float64)
        wb = np.ascontiguousarray(wind_basis, dtype=np.float64)
        assert sb.shape == (method.mesh.V, 8) and wb.shape == (method.mesh.V, 8, 2)
        check(lib().nb_server_add_grid(self._h, method.handle, sb.ctypes.data, wb.ctypes.data))
        self.grids[method.mesh.grid.N] = method

    @staticmethod
    def request(op, N, nlev, nfields=1, dtype=NB_F32, seed=0, keep_output=False, keep_input=False):
        r = nb_request()
        r.op = OPS[op] if isinstance(op, str) else int(op)
        r.N, r.nlev, r.nfields, r.dtype = int(N), int(nlev), int(nfields), int(dtype)
        r.keep_output = 2 if keep_input else (1 if keep_output else 0)
        r.seed = int(seed)
        return r

    def submit(self, req) -> int:
        t = ctypes.c_uint64()
        check(lib().nb_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: float = 60000.0):
        res = nb_result()
        check(lib().nb_server_wait(self._h, ticket, float(timeout_ms), ctypes.byref(res)))
        return res

    def poll(self, ticket: int):
        """The request's result if it has finished, else None (never blocks)."""
        res, done = nb_result(), ctypes.c_int32()
        check(lib().nb_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(res)))
        return res if done.value else None

    def output(self, ticket: int, req) -> np.ndarray:
        meth = self.grids[req.N]
        q = 2 if req.dtype == NB_F64 else 4
        lp = (req.nlev + q - 1) // q * q
        nvar = 2 if req.op == OP_GRAD else 1
        dt = np.float64 if req.dtype == NB_F64 else np.float32
        out = np.zeros((req.nfields, meth.mesh.V, lp, nvar), dtype=dt)
        check(lib().nb_server_output(self._h, ticket, out.ctypes.data, out.nbytes))
        return out[:, :, :req.nlev, :] if nvar == 2 else out[:, :, :req.nlev, 0]

    def input(self, ticket: int, req) -> np.ndarray:
        meth = self.grids[req.N]
        q = 2 if req.dtype == NB_F64 else 4
        lp = (req.nlev + q - 1) // q * q
        nvar = 2 if req.op in (OP_DIV, OP_CURL) else 1
        dt = np.float64 if req.dtype == NB_F64 else np.float32
        x = np.zeros((req.nfields, meth.mesh.V, lp, nvar), dtype=dt)
        check(lib().nb_server_input(self._h, ticket, x.ctypes.data, x.nbytes))
        return x[:, :, :req.nlev, :] if nvar == 2 else x[:, :, :req.nlev, 0]

    def inject_failure(self, seed: int, alloc_index: int) -> None:
        """Refuse the alloc_index-th device allocation of every request
        submitted afterwards with this seed (-1 removes it); such a request
        ends with NB_EOOM (see nb_server_inject_failure)."""
        check(lib().nb_server_inject_failure(self._h, int(seed), int(alloc_index)))

    def stats(self):
        u, p = ctypes.c_int64(), ctypes.c_int64()
        q, f = ctypes.c_int32(), ctypes.c_int32()
        check(lib().nb_server_stats(self._h, ctypes.byref(u), ctypes.byref(p), ctypes.byref(q),
                                    ctypes.byref(f)))
        return {"used": u.value, "peak_used": p.value, "pending": q.value, "inflight": f.value}

    def run_trace(self, reqs, arrivals):
        n = len(reqs)
        arr = (nb_request * n)(*reqs)
        times = np.ascontiguousarray(arrivals, dtype=np.float64)
        res = (nb_result * n)()
        check(lib().nb_server_run_trace(self._h, arr, times.ctypes.data, n, res))
        return res


NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024


def laplacian_noalloc(method, f, lap, stream=None):
    """Laplacian whose intermediate gradient lives in the library's fixed
    scratch array (no device allocation; see nb_nabla_laplacian_noalloc)."""
    fi, fo = field_view(f, 1), field_view(lap, 1)
    check(lib().nb_nabla_laplacian_noalloc(method.handle, ctypes.byref(fi), ctypes.byref(fo),
                                           ctypes.c_void_p(_stream(stream))))
    return lap


def apply_host(method: Method, op, host_in: torch.Tensor, host_out: torch.Tensor,
               dev_in: torch.Tensor, dev_out: torch.Tensor, scratch=None, stream=None):
    """End-to-end call on host buffers laid out like dev_in / dev_out (their
    padded storage: pass the base tensors, e.g. ``t._base`` of a view)."""
    code = OPS[op] if isinstance(op, str) else int(op)
    nin = 2 if code in (OP_DIV, OP_CURL) else 1
    nout = 2 if code == OP_GRAD else 1
    fi, fo = field_view(dev_in, nin), field_view(dev_out, nout)
    fs = ctypes.byref(field_view(scratch, 2)) if scratch is not None else None
    check(lib().nb_nabla_apply_host(method.handle, code, ctypes.c_void_p(host_in.data_ptr()),
                                    ctypes.c_void_p(host_out.data_ptr()), ctypes.byref(fi),
                                    ctypes.byref(fo), fs, ctypes.c_void_p(_stream(stream))))
    return host_out
