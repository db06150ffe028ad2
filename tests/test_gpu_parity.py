"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element in grid order.

Gates: relative L2 <= 1e-12 on the FP64 path and <= 1e-5 on the FP32 path
(inputs rounded to FP32 first and given to the oracle exactly, so the
comparison measures arithmetic error, not input rounding)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1908_06091_b300 import nabla
from gpu_helpers import (error_stats, inputs, oracle_mesh, oracle_op, pole_mask, product, rel_l2,
                         run_op, to_device, to_grid)

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
# Per-node gate: max |x - ref| <= MAXTOL * max |ref| (the bound is derived in
# the docstring of _path_case).
MAXTOL = {torch.float64: 1e-12, torch.float32: 1e-5}
OPS = ["grad", "div", "curl", "lap"]


def _case(N, nlev, dtype, lmax=10, reorder=1, variant=nabla.KERNEL_AUTO, comp=True, pad=True,
          ops=OPS, levels=None):
    g, m, meth = product(N, reorder)
    meth.set_kernel(variant)
    meth.set_compensated(comp)
    om = oracle_mesh(N)
    f, uv = inputs(om, nlev, lmax, dtype)
    perm = m.permutation()
    fs = nabla.NodeColumns(meth, nlev, dtype)
    fd = to_device(fs, f, perm, 1, pad)
    uvd = to_device(fs, uv, perm, 2, pad)
    errs = {}
    for op in ops:
        xin = fd if op in ("grad", "lap") else uvd
        out = to_grid(run_op(meth, fs, op, xin), perm)
        xo = f if op in ("grad", "lap") else uv
        if levels is not None:
            out = out[:, levels]
            xo = xo[:, levels]
        ref = oracle_op(om, op, xo.astype(np.float64))
        assert np.isfinite(out).all(), op
        errs[op] = rel_l2(out, ref)
    meth.set_kernel(nabla.KERNEL_AUTO)
    meth.set_compensated(True)
    return errs


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("nlev", [1, 7, 137])
def test_o32_all_ops(nlev, dtype):
    errs = _case(32, nlev, dtype)
    assert max(errs.values()) <= TOL[dtype], errs


@pytest.mark.parametrize("nlev", [1, 2, 3, 5, 6, 9])
@pytest.mark.parametrize("pad", [True, False], ids=["padded", "unpadded"])
def test_ragged_levels_and_layouts(nlev, pad):
    for dtype in (torch.float32, torch.float64):
        errs = _case(16, nlev, dtype, pad=pad)
        assert max(errs.values()) <= TOL[dtype], (dtype, errs)


@pytest.mark.parametrize("variant", [nabla.KERNEL_DIRECT, nabla.KERNEL_TILED])
def test_kernel_variants_agree_with_oracle(variant):
    for dtype in (torch.float32, torch.float64):
        errs = _case(48, 40, dtype, variant=variant)
        assert max(errs.values()) <= TOL[dtype], (variant, dtype, errs)


def test_grid_order_mesh():
    errs = _case(24, 9, torch.float32, reorder=0)
    assert max(errs.values()) <= 1e-5, errs


def test_plain_fp32_accumulation_also_within_gate():
    errs = _case(32, 9, torch.float32, comp=False)
    assert max(errs.values()) <= 1e-5, errs


def _levels_to_grid(t: torch.Tensor, perm: np.ndarray, levels) -> np.ndarray:
    """Device field -> grid-order float64 host array of the chosen levels."""
    x = (t if levels is None else t[:, levels]).detach().cpu().numpy().astype(np.float64)
    out = np.empty_like(x)
    out[perm] = x
    return out


def _path_case(N, nlev, dtype, lmax, levels=None):
    """Every call of the operator path on one set of seeded inputs, in the
    default launch configuration (the one bench.py times): the single
    operators, nb_nabla_gradlap (the gradient and the divergence of it, the
    Laplacian), nb_nabla_divcurl and the standalone Laplacian.  Returns the
    error figures of gpu_helpers.error_stats for each output against the
    oracle on `levels` (all levels when None).

    The per-node bound.  In the FP32 path each output is a sum of at most
    d + 1 terms (d <= 7 neighbours in the main region, plus the self term of
    div and curl), and each term is of the size of the result: the
    difference form multiplies a weight of size |S|/V ~ 1/h by a difference
    of size h |grad x|.  The sum is rounded at most d + 3 times (one FMA per
    term, the combination of the partial sums, the two vector halves), so
    |err| <= (d + 3) u sum|term| ~ 10 * 2^-24 * 7 max|ref| ~ 4e-6 max|ref| at
    the node where the terms are largest; the pole rows run in FP64 and are
    rounded once to FP32.  The gate is 1e-5 of max|ref|, the same figure as
    the relative-L2 gate.  The FP64 path differs from the oracle only in
    summation order and in the projection of the weights (a few tens of
    roundings of 1.1e-16 of terms of the result's size), so 1e-12 of
    max|ref| leaves a wide margin.  The pole rows alone are gated by their
    relative L2 at the dtype's tolerance."""
    g, m, meth = product(N)
    om = oracle_mesh(N)
    f, uv = inputs(om, nlev, lmax, dtype)
    perm = m.permutation()
    fs = nabla.NodeColumns(meth, nlev, dtype)
    fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
    sel = slice(None) if levels is None else levels
    refs = {"grad": oracle_op(om, "grad", f[:, sel].astype(np.float64)),
            "lap": oracle_op(om, "lap", f[:, sel].astype(np.float64)),
            "div": oracle_op(om, "div", uv[:, sel].astype(np.float64)),
            "curl": oracle_op(om, "curl", uv[:, sel].astype(np.float64))}
    del f, uv
    pole = pole_mask(om)
    nan = float("nan")
    G, Lg = fs.create_field(nvar=2, fill=nan), fs.create_field(fill=nan)
    D, Z = fs.create_field(fill=nan), fs.create_field(fill=nan)
    nabla.gradlap(meth, fd, G, Lg)
    nabla.divcurl(meth, uvd, D, Z)
    torch.cuda.synchronize()
    assert nabla.device_status() == 0
    got = {"gradlap.grad": (G, "grad"), "gradlap.lap": (Lg, "lap"),
           "divcurl.div": (D, "div"), "divcurl.curl": (Z, "curl")}
    stats = {}
    for name, (t, op) in got.items():
        x = _levels_to_grid(t, perm, levels)
        assert np.isfinite(x).all(), name
        stats[name] = error_stats(x, refs[op], pole)
    del G, Lg, D, Z, got
    for op in ("grad", "div", "curl", "lap"):
        x = _levels_to_grid(run_op(meth, fs, op, fd if op in ("grad", "lap") else uvd), perm, levels)
        assert np.isfinite(x).all(), op
        stats[op] = error_stats(x, refs[op], pole)
    return stats


def _gate(stats, dtype):
    for name, s in stats.items():
        print(f"{name:14s} rel_l2 {s['rel_l2']:.3e}  max_rel {s['max_rel']:.3e}  "
              f"max_abs {s['max_abs']:.3e}  pole_rel_l2 {s['pole_rel_l2']:.3e}")
    bad = {n: s for n, s in stats.items()
           if not (s["rel_l2"] <= TOL[dtype] and s["max_rel"] <= MAXTOL[dtype]
                   and s["pole_rel_l2"] <= TOL[dtype])}
    assert not bad, bad


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_o640_137_levels_every_call(dtype):
    """O640 x 137, every node and level (the workload of the second
    configuration), both precisions: relative-L2, per-node maximum and
    pole-row gates on every call of the operator path."""
    _gate(_path_case(640, 137, dtype, 40), dtype)


def test_o1280_137_levels_every_timed_call():
    """O1280 x 137 FP32, the benchmark workload in its launch configuration.
    The GPU computes all levels; levels {0, 68, 136} of the gradient and the
    Laplacian of nb_nabla_gradlap, the div and curl of nb_nabla_divcurl and
    the single-operator calls are compared with the oracle over all nodes,
    with the relative-L2, per-node maximum and pole-row gates."""
    _gate(_path_case(1280, 137, torch.float32, 40, levels=[0, 68, 136]), torch.float32)


def test_gradient_of_constant_is_zero_on_gpu():
    g, m, meth = product(32)
    for dtype in (torch.float32, torch.float64):
        fs = nabla.NodeColumns(meth, 9, dtype)
        f = fs.create_field(fill=2.5)
        out = run_op(meth, fs, "grad", f)
        assert torch.count_nonzero(out).item() == 0


def test_conservation_on_gpu():
    g, m, meth = product(32)
    vol = torch.as_tensor(meth.dual_volumes(), device="cuda")
    fs = nabla.NodeColumns(meth, 3, torch.float64)
    uv = fs.create_field(nvar=2)
    uv.copy_(torch.randn(uv.shape, dtype=torch.float64, generator=torch.Generator().manual_seed(1)))
    for op in ("div", "curl"):
        d = run_op(meth, fs, op, uv)
        r = (vol[:, None] * d).sum(0).abs() / (vol[:, None] * d.abs()).sum(0)
        assert r.max().item() < 1e-13


def test_results_are_deterministic():
    g, m, meth = product(48)
    om = oracle_mesh(48)
    f, uv = inputs(om, 37, 10, torch.float32)
    fs = nabla.NodeColumns(meth, 37, torch.float32)
    perm = m.permutation()
    fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
    for op, x in (("grad", fd), ("div", uvd), ("curl", uvd), ("lap", fd)):
        a = run_op(meth, fs, op, x)
        b = run_op(meth, fs, op, x)
        assert torch.equal(a, b), op


def test_laplacian_with_caller_scratch_equals_library_scratch():
    g, m, meth = product(32)
    om = oracle_mesh(32)
    f, _ = inputs(om, 13, 10, torch.float32)
    fs = nabla.NodeColumns(meth, 13, torch.float32)
    fd = to_device(fs, f, m.permutation(), 1)
    scratch = fs.create_field(nvar=2)
    a = run_op(meth, fs, "lap", fd, scratch=scratch)
    b = run_op(meth, fs, "lap", fd)
    assert torch.equal(a, b)


def _raw(t, dtype, nvar, nlev=None, node_stride=None, lev_stride=None, nnodes=None):
    f = nabla.nb_field()
    f.data = t.data_ptr()
    f.dtype = dtype
    f.nvar = nvar
    f.nnodes = t.shape[0] if nnodes is None else nnodes
    f.nlev = t.shape[1] if nlev is None else nlev
    f.reserved = 0
    f.node_stride = t.stride(0) if node_stride is None else node_stride
    f.lev_stride = nvar if lev_stride is None else lev_stride
    return f


def _call(meth, op, fi, fo):
    import ctypes
    return nabla.lib().nb_nabla_apply(meth.handle, op, ctypes.byref(fi), ctypes.byref(fo), None,
                                      ctypes.c_void_p(0))


def test_c_abi_rejects_bad_fields_before_any_launch():
    g, m, meth = product(16)
    fs = nabla.NodeColumns(meth, 4, torch.float32)
    f = fs.create_field()
    gv = fs.create_field(nvar=2)
    before = nabla.launch_count()
    F32, F64 = nabla.NB_F32, nabla.NB_F64
    ok_in, ok_out = _raw(f, F32, 1), _raw(gv, F32, 2)
    assert _call(meth, nabla.OP_GRAD, _raw(f, F32, 1), _raw(f, F32, 1)) == nabla.NB_ESHAPE  # nvar
    assert _call(meth, nabla.OP_GRAD, ok_in, _raw(gv, F64, 2)) == nabla.NB_EDTYPE          # dtype
    assert _call(meth, nabla.OP_GRAD, _raw(f, 7, 1), ok_out) == nabla.NB_EDTYPE            # unknown
    assert _call(meth, nabla.OP_GRAD, ok_in, _raw(gv, F32, 2, nnodes=m.V - 1)) == nabla.NB_ESHAPE
    assert _call(meth, nabla.OP_GRAD, ok_in, _raw(gv, F32, 2, nlev=3)) == nabla.NB_ESHAPE  # levels
    assert _call(meth, nabla.OP_GRAD, ok_in, _raw(gv, F32, 2, node_stride=6)) == nabla.NB_ESHAPE
    assert _call(meth, nabla.OP_GRAD, ok_in, _raw(gv, F32, 2, lev_stride=1)) == nabla.NB_ESHAPE
    assert _call(meth, 9, ok_in, ok_out) == nabla.NB_EINVAL                                  # op
    # output overlapping the input
    assert _call(meth, nabla.OP_DIV, _raw(gv, F32, 2), _raw(gv, F32, 1, node_stride=gv.stride(0),
                                                              lev_stride=1)) in (nabla.NB_EINVAL,)
    assert nabla.launch_count() == before
    assert nabla.lib().nb_last_error()


def test_device_status_reports_ok_after_normal_runs():
    assert nabla.device_status(clear=True) in (0,)
    assert nabla.device_status() == 0


def test_host_buffer_entry_point_matches_device_call():
    g, m, meth = product(32)
    om = oracle_mesh(32)
    f, _ = inputs(om, 9, 10, torch.float32)
    fs = nabla.NodeColumns(meth, 9, torch.float32)
    fd = to_device(fs, f, m.permutation(), 1)
    ref = run_op(meth, fs, "lap", fd)
    host_in = fd._base.cpu().pin_memory()
    out = fs.create_field()
    host_out = torch.empty_like(out._base, device="cpu").pin_memory()
    nabla.apply_host(meth, "lap", host_in, host_out, fd, out)
    assert torch.equal(host_out[:, :9], ref.cpu())


def test_field_upload_and_download_round_trip_on_streams():
    g, m, meth = product(32)
    fs = nabla.NodeColumns(meth, 9, torch.float32)
    src = torch.randn((m.V, fs.lp, 2), dtype=torch.float32).pin_memory()
    dev = fs.create_field(nvar=2, fill=0.0)
    back = torch.zeros_like(src).pin_memory()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nabla.upload(dev, src, 2, stream=s1)
    ev = torch.cuda.Event()
    ev.record(s1)
    s2.wait_event(ev)
    nabla.download(back, dev, 2, stream=s2)
    s2.synchronize()
    assert torch.equal(back, src)
    with pytest.raises(nabla.NablaError):
        fv = nabla.field_view(dev, 2)
        nabla.check(nabla.lib().nb_field_upload(None, None, None))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("nlev,pad", [(1, True), (7, True), (7, False), (137, True)])
def test_edge_variant_equals_direct_kernels_bitwise(nlev, pad, dtype):
    """NB_KERNEL_EDGE (per-edge differences materialised, then reduced per
    node) reproduces the direct kernels bit for bit."""
    g, m, meth = product(32)
    om = oracle_mesh(32)
    f, uv = inputs(om, nlev, 10, dtype)
    perm = m.permutation()
    fs = nabla.NodeColumns(meth, nlev, dtype)
    fd, uvd = to_device(fs, f, perm, 1, pad), to_device(fs, uv, perm, 2, pad)
    lv = slice(0, nlev)
    for op in OPS:
        x = fd if op in ("grad", "lap") else uvd
        meth.set_kernel(nabla.KERNEL_EDGE)
        got = run_op(meth, fs, op, x)
        meth.set_kernel(nabla.KERNEL_DIRECT)
        ref = run_op(meth, fs, op, x)
        meth.set_kernel(nabla.KERNEL_AUTO)
        assert torch.equal(got[:, lv], ref[:, lv]), (op, nlev, pad)


def test_o32_one_level_fp64_with_the_solid_body_wind():
    """The first configuration as stated: O32, one level, FP64, a seeded
    spherical-harmonic scalar (degree <= 10) and the solid-body wind
    u = 20 m/s cos(lat), v = 0, all four operators against the oracle.  The
    discrete divergence of solid-body rotation is near zero (a truncation
    residue), so it is gated by its absolute difference from the oracle,
    scaled by the curl's magnitude (~2U/R)."""
    from paper_1908_06091_b300 import synth
    N = 32
    g, m, meth = product(N)
    om = oracle_mesh(N)
    perm = m.permutation()
    f, _ = inputs(om, 1, 10, torch.float64)
    uv = synth.solid_body_wind(om.lat)
    uv = np.asarray(uv, dtype=np.float64).reshape(om.V, 1, 2)
    fs = nabla.NodeColumns(meth, 1, torch.float64)
    fd, uvd = to_device(fs, f, perm, 1), to_device(fs, uv, perm, 2)
    for op, x, xin in (("grad", f, fd), ("lap", f, fd)):
        ref = oracle_op(om, op, x)
        assert rel_l2(to_grid(run_op(meth, fs, op, xin), perm), ref) <= 1e-12, op
    z_ref = oracle_op(om, "curl", uv)
    z = to_grid(run_op(meth, fs, "curl", uvd), perm)
    assert rel_l2(z, z_ref) <= 1e-12
    d_ref = oracle_op(om, "div", uv)
    d = to_grid(run_op(meth, fs, "div", uvd), perm)
    assert np.abs(d - d_ref).max() <= 1e-12 * np.abs(z_ref).max()
    assert np.abs(d_ref).max() < 1e-2 * np.abs(z_ref).max()  # the divergence is a small residue
