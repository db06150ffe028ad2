"""Host-side C-ABI checks (no GPU): the library loads, exports every symbol
its header declares, and its host mesh builder reproduces the oracle's grid
and triangulation (two independent implementations)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_1908_06091_b300 import nabla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nb_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = nabla.lib()
    names = _declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares each of them
    assert set(names) <= set(nabla.SIGNATURES) | {"nb_version", "nb_last_error"}


def test_version_and_error_reporting():
    assert "sm_103a" in nabla.version()
    with pytest.raises(nabla.NablaError) as ei:
        nabla.Grid(0)
    assert ei.value.code == nabla.NB_EINVAL and "N must be" in str(ei.value)


@pytest.mark.parametrize("N", [1, 16, 32, 80, 640, 1280])
def test_grid_matches_oracle_bit_for_bit(N):
    """Both sides compute correctly rounded Legendre roots, so the node
    positions agree exactly (the dual geometry reacts to the last bit)."""
    g = nabla.Grid(N)
    assert g.size == oracle.num_nodes(N)
    ll = g.lonlat()
    lat, lon = oracle.grid_lonlat(N)
    assert np.array_equal(ll[:, 0], lon)
    assert np.array_equal(ll[:, 1], lat)


@pytest.mark.parametrize("N,reorder", [(1, 0), (16, 0), (16, 1), (48, 1)])
def test_mesh_matches_oracle_triangulation(N, reorder):
    g = nabla.Grid(N)
    m = nabla.Mesh(g, reorder)
    assert (m.V, m.E, m.F) == (g.size, 3 * g.size - 6, 2 * g.size - 4)
    perm = m.permutation()
    assert np.array_equal(np.sort(perm), np.arange(m.V))
    tri = perm[m.triangles()]                       # back to grid numbering
    ot = oracle.triangulate(N)
    canon = lambda t: {tuple(np.roll(r, -int(np.argmin(r)))) for r in t}
    assert canon(tri) == canon(ot)                  # same oriented triangles
    e = perm[m.edges()]
    oe, _ = oracle.edges(g.size, ot)
    assert {tuple(sorted(x)) for x in e} == {tuple(sorted(x)) for x in oe}


def test_pole_rows_come_last():
    N = 24
    m = nabla.Mesh(nabla.Grid(N), 1)
    perm = m.permutation()
    nx = oracle.row_nx(N)
    assert m.cap_begin == m.V - nx[0] - nx[-1]
    tail = set(perm[m.cap_begin:].tolist())
    assert tail == set(range(nx[0])) | set(range(m.V - nx[-1], m.V))


def test_hilbert_order_is_local():
    """Consecutive nodes in the reordered mesh are close on the sphere."""
    N = 64
    g = nabla.Grid(N)
    m = nabla.Mesh(g, 1)
    ll = g.lonlat()[m.permutation()]
    xyz = np.stack([np.cos(ll[:, 1]) * np.cos(ll[:, 0]), np.cos(ll[:, 1]) * np.sin(ll[:, 0]),
                    np.sin(ll[:, 1])], 1)
    step = np.linalg.norm(np.diff(xyz[:m.cap_begin], axis=0), axis=1)
    h = np.pi / (2 * N)
    assert np.median(step) < 1.5 * h
    m0 = nabla.Mesh(g, 0)
    ll0 = g.lonlat()[m0.permutation()]
    # tiles of 64 consecutive nodes: Hilbert tiles are much more compact
    def spread(llx):
        x = np.stack([np.cos(llx[:, 1]) * np.cos(llx[:, 0]), np.cos(llx[:, 1]) * np.sin(llx[:, 0]),
                      np.sin(llx[:, 1])], 1)[: (m.cap_begin // 64) * 64].reshape(-1, 64, 3)
        return np.linalg.norm(x - x.mean(1, keepdims=True), axis=2).max(1).mean()
    assert spread(ll) < 0.5 * spread(ll0)


def test_method_requires_a_device_and_reports_it():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the GPU tests")
    m = nabla.Mesh(nabla.Grid(4), 1)
    with pytest.raises(nabla.NablaError) as ei:
        nabla.Method(m)
    assert ei.value.code == nabla.NB_ECUDA


@pytest.mark.parametrize("N,rcap,nmax", [(16, 12, 256), (48, 87, 256), (64, 175, 256), (64, 40, 8)])
def test_tile_plan_fits_stage_and_maps_every_neighbour(N, rcap, nmax):
    """Host check of the staged kernels' plan: every tile's own nodes plus
    halo fit the stage, tiles cover the nodes in order with the pole block
    separate, and each staged-row index resolves to the CSR neighbour."""
    m = nabla.Mesh(nabla.Grid(N), 1)
    rp, nbr = m.csr()
    node0, hptr, halo, lnbr, ntm = m.tile_plan(rcap, nmax)
    assert node0[0] == 0 and node0[-1] == m.V and np.all(np.diff(node0) > 0)
    assert node0[ntm] == m.cap_begin
    n = np.diff(node0)
    H = np.diff(hptr)
    assert np.all(n <= nmax)
    assert np.all(n + H <= np.maximum(rcap, 1 + np.diff(rp)[node0[:-1]]))
    for t in range(len(n)):
        a, b = node0[t], node0[t + 1]
        h = halo[hptr[t]:hptr[t + 1]]
        assert np.all(np.diff(h) > 0) and not np.any((h >= a) & (h < b))
        p = np.arange(rp[a], rp[b])
        loc = lnbr[p].astype(np.int64)
        hi = np.clip(loc - (b - a), 0, max(len(h) - 1, 0))
        res = np.where(loc < b - a, a + loc, h[hi] if len(h) else a + loc)
        assert np.array_equal(res, nbr[p])
    # the pole rows (nodes from cap_begin on) are one node per tile, so the
    # staged kernels can spread their slower FP64 path over many CTAs
    assert np.all(n[ntm:] == 1) and len(n) - ntm == m.V - m.cap_begin
    # neighbour lists agree with the edge list
    e = m.edges()
    deg = np.bincount(e.ravel(), minlength=m.V)
    assert np.array_equal(np.diff(rp), deg)


def test_allocator_and_server_poll_argument_checks():
    """nb_set_allocator wants both callbacks (NULL restores the CUDA runtime);
    nb_server_poll rejects NULL arguments before touching any server."""
    L = nabla.lib()
    half = nabla.nb_allocator(None, nabla._ALLOC_FN(lambda c, n, s: None), nabla._RELEASE_FN())
    assert L.nb_set_allocator(ctypes.byref(half)) == nabla.NB_EINVAL
    assert b"both" in L.nb_last_error()
    assert L.nb_set_allocator(None) == nabla.NB_OK
    done, res = ctypes.c_int32(), nabla.nb_result()
    assert L.nb_server_poll(None, 1, ctypes.byref(done), ctypes.byref(res)) == nabla.NB_EINVAL


def _classic_like_pl(N):
    o = oracle.row_nx(N)
    pl = (np.round(o * 1.1 / 5) * 5 + (np.arange(2 * N) % 3 == 0)).astype(np.int32)
    pl[N:] = pl[:N][::-1]
    return pl


@pytest.mark.parametrize("kind,N", [("F", 8), ("F", 80), ("P", 6), ("P", 32)])
def test_other_grid_families_match_the_oracle(kind, N):
    """Regular F<N> (Sec. 4.2.3.6) and PL-array grids (Sec. 4.2.3.7): same
    points bit for bit and the same triangles as the independent oracle."""
    pl = oracle.regular_nx(N) if kind == "F" else _classic_like_pl(N)
    g = nabla.Grid.regular(N) if kind == "F" else nabla.Grid.reduced(pl)
    assert g.N == N and np.array_equal(g.pl(), pl)
    lat, lon = oracle.grid_lonlat(N, pl)
    ll = g.lonlat()
    assert np.array_equal(ll[:, 0], lon) and np.array_equal(ll[:, 1], lat)
    canon = lambda t: {tuple(np.roll(r, -int(np.argmin(r)))) for r in t}  # oriented triangles
    otri = canon(oracle.triangulate(N, pl))
    for reorder in (0, 1):
        m = nabla.Mesh(g, reorder)
        assert (m.V, m.E, m.F) == (g.size, 3 * g.size - 6, 2 * g.size - 4)
        assert canon(m.permutation()[m.triangles()]) == otri


def test_grid_names_and_pl_checks():
    assert nabla.Grid.named("O32").size == 5248
    assert nabla.Grid.named("F16").size == 8 * 16 * 16
    for bad in ("N16", "X16", "O", "O16x", "F0", ""):
        with pytest.raises(nabla.NablaError) as e:
            nabla.Grid.named(bad)
        assert e.value.code == nabla.NB_EINVAL
    for bad in ([20, 24, 20], [20, 2, 2, 20], [20]):
        with pytest.raises(nabla.NablaError):
            nabla.Grid.reduced(bad)


def test_last_error_is_per_thread():
    """nb_last_error() is thread-local: an error raised on one thread does not
    overwrite the message another thread reads."""
    import ctypes
    import threading
    L = nabla.lib()
    barrier = threading.Barrier(2)
    seen = {}

    def worker(name, bad_call):
        rc = bad_call()
        barrier.wait()          # both threads have failed before either reads
        seen[name] = (rc, L.nb_last_error().decode())

    g = ctypes.c_void_p()
    t1 = threading.Thread(target=worker, args=("grid", lambda: L.nb_grid_create_octahedral(0, ctypes.byref(g))))
    t2 = threading.Thread(target=worker, args=("mesh", lambda: L.nb_mesh_create(None, 1, ctypes.byref(g))))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert seen["grid"][0] == nabla.NB_EINVAL and seen["mesh"][0] == nabla.NB_EINVAL
    assert seen["grid"][1] and seen["mesh"][1]
    assert seen["grid"][1] != seen["mesh"][1], seen


@pytest.mark.parametrize("grid", ["O32", "O96", "F16", "PL"])
def test_fused_laplacian_plans_fit_their_layout(grid):
    """The single-pass Laplacian's planner grows tiles with incrementally
    counted rings; the library then recounts every tile's rings exactly and
    refuses a plan in which one does not fit the kernel's shared memory.
    Every plan it builds must pass that check, with pole-row tiles last."""
    pl = [20, 27, 33, 40, 44, 47, 47, 44, 40, 33, 27, 20]
    g = {"O32": lambda: nabla.Grid(32), "O96": lambda: nabla.Grid(96), "F16": lambda: nabla.Grid.regular(16),
         "PL": lambda: nabla.Grid.reduced(pl)}[grid]()
    m = nabla.Mesh(g, 1)
    for nlev in (16, 37, 91, 137, 300):
        ntiles, nmain, max_gnodes, fits = m.lap_plan(nlev)
        assert fits == 1, (grid, nlev)
        assert 0 < nmain < ntiles <= m.V
        assert max_gnodes >= 2
    with pytest.raises(nabla.NablaError):
        m.lap_plan(8)


def test_corrupted_tile_plans_are_refused_on_the_host():
    """The plan check the library runs before uploading a plan: a valid plan
    passes; a halo node out of range, a neighbour mapped to the wrong staged
    row, and tiles out of order are each refused with NB_EINVAL (no GPU)."""
    m = nabla.Mesh(nabla.Grid(24), 1)
    node0, hptr, halo, lnbr, _ = m.tile_plan(rcap=160, nmax=64)
    m.check_tile_plan(node0, hptr, halo, lnbr)
    bad_halo = halo.copy()
    bad_halo[len(bad_halo) // 2] = m.V + 5
    bad_rows = lnbr.copy()
    rp, _nbr = m.csr()
    p = int(rp[len(rp) // 2])
    bad_rows[p] = (int(bad_rows[p]) + 1) % 60000
    bad_order = node0.copy()
    bad_order[3], bad_order[4] = bad_order[4], bad_order[3]
    for args, what in (((node0, hptr, bad_halo, lnbr), "halo"), ((node0, hptr, halo, bad_rows), "staged"),
                       ((bad_order, hptr, halo, lnbr), "order")):
        with pytest.raises(nabla.NablaError) as ei:
            m.check_tile_plan(*args)
        assert ei.value.code == nabla.NB_EINVAL, what


def test_new_control_calls_check_their_arguments_on_the_host():
    """The failure-injection, probe, plan-check and kernel-control calls reject
    NULL or out-of-range arguments with NB_EINVAL before any device work."""
    L = nabla.lib()
    assert L.nb_server_inject_failure(None, 1, 0) == nabla.NB_EINVAL
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert L.nb_probe_fp64_rate(0, None, ctypes.byref(tf), ctypes.byref(ms)) == nabla.NB_EINVAL
    assert L.nb_probe_fp64_rate(1000, None, None, ctypes.byref(ms)) == nabla.NB_EINVAL
    assert L.nb_method_set_wait_limit(None, 0) == nabla.NB_EINVAL
    assert L.nb_method_set_item_shape(None, 0, -1) == nabla.NB_EINVAL
    assert L.nb_method_set_node_pairs(None, -1) == nabla.NB_EINVAL
    assert L.nb_batch_graph_nodes(None, None, None) == nabla.NB_EINVAL
    assert L.nb_mesh_node_pairs(None, None) == nabla.NB_EINVAL
    assert L.nb_method_set_laplacian_route(None, 0) == nabla.NB_EINVAL
    assert L.nb_check_tile_plan(None, 1, None, None, None, None) == nabla.NB_EINVAL
    m = nabla.Mesh(nabla.Grid(16), 1)
    node0, hptr, halo, lnbr, _ = m.tile_plan(rcap=160, nmax=64)
    empty = np.zeros(1, dtype=np.int32)
    # zero tiles do not cover a mesh with nodes
    assert L.nb_check_tile_plan(m.handle, 0, empty.ctypes.data, empty.ctypes.data, empty.ctypes.data,
                                lnbr.ctypes.data) == nabla.NB_EINVAL
    assert b"cover" in L.nb_last_error() or b"tiles" in L.nb_last_error()


def test_nb_debug_logs_setup_steps_to_stderr():
    """NB_DEBUG=1 makes the library log its setup steps (here a mesh build)
    to stderr; unset, it prints nothing."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1908_06091_b300 import nabla\n"
            "nabla.Mesh(nabla.Grid(16), 1)\n") % ROOT
    env = dict(os.environ)
    env.pop("NB_DEBUG", None)
    quiet = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    env["NB_DEBUG"] = "1"
    loud = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert quiet.returncode == 0 and loud.returncode == 0
    assert "[nabla_b300]" not in quiet.stderr
    assert "[nabla_b300] mesh: 1600 nodes, 4794 edges, 3196 triangles" in loud.stderr


@pytest.mark.parametrize("N,reorder", [(24, 1), (48, 1), (32, 0)])
def test_node_pairs_are_adjacent_six_neighbour_nodes_with_reordered_rows(N, reorder):
    """Node pairs (nb_mesh_node_pairs) are mutual, adjacent six-neighbour
    nodes outside the pole rows at most 16 places apart, with exactly two
    common neighbours; each paired row starts with those two (ascending),
    then the partner, then the rest ascending; unpaired rows are ascending.
    Neighbour sets are checked against the triangles, independently of the
    CSR."""
    m = nabla.Mesh(nabla.Grid(N), reorder)
    rp, nbr = m.csr()
    mate = m.node_pairs()
    tri = m.triangles()
    adj = [set() for _ in range(m.V)]
    for a, b, c in tri:
        adj[a] |= {b, c}
        adj[b] |= {a, c}
        adj[c] |= {a, b}
    idx = np.flatnonzero(mate >= 0)
    assert len(idx) > 0.85 * m.V
    assert np.array_equal(mate[mate[idx]], idx)
    assert np.all(idx < m.cap_begin) and np.all(np.abs(mate[idx] - idx) <= 16)
    for i in range(m.V):
        row = nbr[rp[i]:rp[i + 1]].tolist()
        assert set(row) == adj[i] and len(row) == len(adj[i])
        j = int(mate[i])
        if j < 0:
            assert row == sorted(row)
            continue
        common = sorted(adj[i] & adj[j])
        assert len(row) == 6 and len(adj[j]) == 6 and len(common) == 2
        assert row[:2] == common and row[2] == j and row[3:] == sorted(row[3:])
    # greedy along the node order: no unpaired six-neighbour node has an
    # unpaired neighbour it could have been matched with
    free = set(np.flatnonzero(mate < 0).tolist())
    for i in free:
        if i >= m.cap_begin or len(adj[i]) != 6:
            continue
        for j in adj[i]:
            if j in free and j < m.cap_begin and abs(j - i) <= 16 and len(adj[j]) == 6:
                assert len(adj[i] & adj[j]) != 2, (i, j)


def _slot_lists(node0, mate):
    """Slot lists in the format the staged plans use: per tile its pairs of
    mates that are both own nodes (li | lj << 16), then its other nodes
    (li | li << 16), each list padded to a multiple of 4."""
    sptr, npairs, slots = [], [], []
    for t in range(len(node0) - 1):
        a, b = int(node0[t]), int(node0[t + 1])
        sptr.append(len(slots))
        for k in range(a, b):
            j = int(mate[k])
            if k < j < b:
                slots.append((k - a) | (j - a) << 16)
        npairs.append(len(slots) - sptr[-1])
        for k in range(a, b):
            j = int(mate[k])
            if not (a <= j < b):
                slots.append((k - a) * 0x10001)
        while len(slots) % 4:
            slots.append(0)
    sptr.append(len(slots))
    return (np.array(sptr, dtype=np.int32), np.array(npairs, dtype=np.int32), np.array(slots, dtype=np.uint32))


def test_slot_lists_are_checked_on_the_host():
    """nb_check_slot_lists accepts slot lists built from a tile plan and the
    node pairs, and refuses each kind of corruption the pair path relies on
    (NB_EINVAL, nothing launched): a node left out, a pair of non-mates, a
    pair count beyond the tile's pairs, a slot range past the array."""
    m = nabla.Mesh(nabla.Grid(24), 1)
    mate = m.node_pairs()
    node0, hptr, halo, lnbr, _ = m.tile_plan(rcap=160, nmax=64)
    sptr, npairs, slots = _slot_lists(node0, mate)
    assert npairs.sum() > 0.3 * m.V
    m.check_slot_lists(node0, sptr, npairs, slots)
    t = int(np.argmax(npairs))  # a tile with pairs
    q0 = int(sptr[t])
    cases = {}
    s = slots.copy()
    s[q0 + npairs[t]] = s[q0]  # a single slot repeating a pair's node: one node twice, one left out
    cases["node left out"] = (sptr, npairs, s)
    s = slots.copy()
    li, lj = int(s[q0] & 0xFFFF), int(s[q0] >> 16)
    s[q0] = li | ((lj + 1) % (int(node0[t + 1]) - int(node0[t])) << 16)
    cases["non-mates"] = (sptr, npairs, s)
    npr = npairs.copy()
    npr[t] += 1
    cases["pair count"] = (sptr, npr, slots)
    sp = sptr.copy()
    sp[-1] += 4
    cases["range"] = (sp, npairs, slots)
    for what, (a, b, c) in cases.items():
        with pytest.raises(nabla.NablaError) as ei:
            m.check_slot_lists(node0, a, b, c)
        assert ei.value.code == nabla.NB_EINVAL, what
