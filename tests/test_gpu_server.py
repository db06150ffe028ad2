"""Continuous-batching server: same result alone and in a mix, correct
against the oracle, budget admission, trace replay."""
import numpy as np
import pytest
import torch

import oracle
from paper_1908_06091_b300 import nabla, synth
from gpu_helpers import oracle_mesh, product, rel_l2

pytestmark = pytest.mark.gpu

R = oracle.EARTH_RADIUS_M


def _bases(N):
    """Scalar and wind bases of grid O<N> in functionspace order."""
    g, m, meth = product(N)
    ll = g.lonlat()[m.permutation()]
    lat, lon = ll[:, 1], ll[:, 0]
    sb = synth.scalar_basis(lat, lon, 10, 99).numpy()
    wb = synth.wind_basis(lat, lon, 10, 99, R).numpy()
    return meth, sb, wb


def _splitmix64(z):
    z = (z + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def _weights(seed, f, nlev):
    w = np.zeros((nlev, 8))
    for k in range(nlev):
        for b in range(8):
            z = _splitmix64(seed ^ (f << 40) ^ (k << 8) ^ b)
            w[k, b] = (2.0 * (z >> 11) / 2.0 ** 53 - 1.0) * (1.0 + k / nlev)
    return w


@pytest.fixture(scope="module")
def server():
    s = nabla.Server(int(2e9), nstreams=4, max_inflight=8)
    for N in (16, 24):
        meth, sb, wb = _bases(N)
        s.add_grid(meth, sb, wb)
    return s


def test_result_is_the_same_alone_and_in_the_mix(server):
    probe = nabla.Server.request("lap", 24, 37, nfields=2, seed=123, keep_output=True)
    alone = server.output(server.wait(server.submit(probe)).ticket, probe)
    rng = np.random.default_rng(1)
    tickets, probes = [], []
    for k in range(40):
        r = nabla.Server.request(["grad", "div", "curl", "lap"][k % 4], int(rng.choice([16, 24])),
                                 int(rng.choice([1, 7, 37])), nfields=int(rng.integers(1, 5)),
                                 dtype=nabla.NB_F32 if k % 3 else nabla.NB_F64, seed=int(k))
        tickets.append(server.submit(r))
        if k % 10 == 5:  # the probe again, in the middle of the mix
            probes.append(server.submit(probe))
    for t in tickets:
        assert server.wait(t).status == nabla.NB_OK
    for t in probes:
        assert server.wait(t).status == nabla.NB_OK
        assert np.array_equal(server.output(t, probe), alone)
    assert server.stats()["peak_used"] <= int(2e9)


@pytest.mark.parametrize("op", ["grad", "div", "curl", "lap"])
def test_served_result_meets_the_oracle_gate(server, op):
    """The server's own inputs (kept) through the oracle vs its outputs."""
    N, nlev, seed = 24, 5, 77
    req = nabla.Server.request(op, N, nlev, nfields=2, seed=seed, keep_input=True)
    t = server.wait(server.submit(req)).ticket
    out, xin = server.output(t, req), server.input(t, req)
    perm = product(N)[1].permutation()
    om = oracle_mesh(N)
    for f in range(2):
        xg = np.empty(xin[f].shape)
        xg[perm] = xin[f]
        ref = {"grad": oracle.grad, "div": oracle.div, "curl": oracle.curl, "lap": oracle.lap}[op](om, xg)
        got = np.empty(out[f].shape)
        got[perm] = out[f]
        assert rel_l2(got, ref) <= 1e-5, (op, f, rel_l2(got, ref))


def test_served_inputs_follow_the_documented_recipe(server):
    """Inputs are per-level SplitMix64 mixtures of the registered bases."""
    N, nlev, seed = 16, 3, 5
    req = nabla.Server.request("grad", N, nlev, nfields=2, seed=seed, keep_input=True)
    t = server.wait(server.submit(req)).ticket
    xin = server.input(t, req)
    meth, sb, wb = _bases(N)
    for f in range(2):
        w = _weights(seed, f, nlev).astype(np.float32).astype(np.float64)
        x = sb.astype(np.float32).astype(np.float64) @ w.T
        assert np.allclose(xin[f], x, rtol=1e-5, atol=1e-5 * np.abs(x).max())


def test_admission_respects_the_budget_and_refuses_oversize():
    meth, sb, wb = _bases(16)
    V = meth.mesh.V
    one = 2 * V * 40 * 4 * (1 + 2)  # grad, 37 levels (Lp 40), 2 fields: in + out
    s = nabla.Server(int(one * 1.5), nstreams=2, max_inflight=4)  # room for one at a time
    s.add_grid(meth, sb, wb)
    ts = [s.submit(nabla.Server.request("grad", 16, 37, nfields=2, seed=k)) for k in range(12)]
    for t in ts:
        assert s.wait(t).status == nabla.NB_OK
    st = s.stats()
    assert st["peak_used"] <= int(one * 1.5) and st["used"] == 0
    with pytest.raises(nabla.NablaError) as e:
        s.submit(nabla.Server.request("grad", 16, 37, nfields=8, seed=1))
    assert e.value.code == nabla.NB_EBUDGET
    with pytest.raises(nabla.NablaError):
        s.submit(nabla.Server.request("grad", 48, 37))  # grid not resident


def test_trace_replay_orders_times(server):
    rng = np.random.default_rng(4)
    n = 60
    arrivals = np.cumsum(rng.exponential(1.0 / 2000.0, n))
    reqs = [nabla.Server.request(["grad", "div", "curl", "lap"][k % 4], 16, 37, nfields=1, seed=k)
            for k in range(n)]
    res = server.run_trace(reqs, arrivals)
    for k in range(n):
        assert res[k].status == nabla.NB_OK
        assert res[k].arrival_s <= res[k].admit_s <= res[k].done_s
        assert res[k].arrival_s >= arrivals[k] - 1e-3


def test_poll_reports_pending_then_the_waited_result(server):
    import time
    req = nabla.Server.request("lap", 24, 137, nfields=8, seed=9)
    t = server.submit(req)
    seen_pending = server.poll(t) is None
    deadline = time.monotonic() + 60.0
    res = None
    while res is None and time.monotonic() < deadline:
        res = server.poll(t)
        time.sleep(0.001)
    assert res is not None and res.status == nabla.NB_OK
    w = server.wait(t, 0.0)
    assert (w.ticket, w.done_s, w.node_levels) == (res.ticket, res.done_s, res.node_levels)
    assert isinstance(seen_pending, bool)
    with pytest.raises(nabla.NablaError):
        server.poll(t + 10_000)


def test_injected_failure_mid_request_spares_the_requests_beside_it(server):
    """A request whose fifth device allocation is refused (host-side
    injection: the second column block's output buffer, after the first
    block's synthesis and operator have been enqueued) ends with NB_EOOM,
    returns its budget, and leaves the requests in flight beside it bitwise
    equal to their runs alone; the same request succeeds once the injection
    is removed."""
    mix = [nabla.Server.request(op, N, L, nfields=nf, dtype=dt, seed=500 + k, keep_output=True)
           for k, (op, N, L, nf, dt) in enumerate([("lap", 24, 37, 3, nabla.NB_F32),
                                                   ("grad", 16, 7, 2, nabla.NB_F64),
                                                   ("div", 24, 37, 4, nabla.NB_F32),
                                                   ("curl", 16, 37, 1, nabla.NB_F32),
                                                   ("lap", 16, 1, 8, nabla.NB_F64)])]
    alone = [server.output(server.wait(server.submit(r)).ticket, r) for r in mix]
    # 8 fields of 37 levels: 3 fields per column block of at most 144 levels
    bad = nabla.Server.request("grad", 24, 37, nfields=8, seed=999, keep_output=True)
    server.inject_failure(999, 4)  # weights, block 0 in/out, block 1 in, block 1 out
    try:
        tickets = []
        for k, r in enumerate(mix):
            tickets.append(server.submit(r))
            if k == 1:
                t_bad = server.submit(bad)
        assert server.wait(t_bad).status == nabla.NB_EOOM
        for t, r, ref in zip(tickets, mix, alone):
            assert server.wait(t).status == nabla.NB_OK
            assert np.array_equal(server.output(t, r), ref)
    finally:
        server.inject_failure(999, -1)
    assert server.wait(server.submit(bad)).status == nabla.NB_OK
    st = server.stats()
    assert st["used"] == 0 and st["inflight"] == 0 and st["pending"] == 0
    with pytest.raises(nabla.NablaError):
        server.inject_failure(1, -2)
