"""GPU tests of the solve server: continuous admission under a memory budget,
overlapping requests on separate streams, and results that are the same
alone and in the mix (the kernels are deterministic per request)."""

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dw():
    import paper_1204_5463_gb300 as pkg

    return pkg


def _requests():
    """Mixed lattices, masses, fields and rhs counts (tiny, so the oracle can check them)."""
    out = []
    specs = [((4, 4, 4, 4), (2, 2, 2, 2), 0.3, -0.5, 1), ((4, 4, 4, 8), (2, 2, 2, 2), 0.4, -0.3, 3),
             ((8, 4, 4, 4), (2, 2, 2, 2), 0.5, 0.0, 2), ((4, 4, 4, 4), (2, 2, 2, 2), 0.6, 0.2, 5),
             ((4, 8, 4, 4), (2, 2, 2, 2), 0.3, -0.4, 1), ((8, 8, 4, 4), (2, 2, 2, 2), 0.45, -0.2, 4)]
    for i, (dims, block, eps, m0, nrhs) in enumerate(specs):
        U = fg.gauge_field(dims, eps, seed=10 + i)
        b = np.ascontiguousarray(fg.gaussian_source(dims, 20 + i, nrhs=nrhs))
        out.append(dict(dims=dims, block=block, m0=m0, U=U, b=b, nrhs=nrhs))
    return out


def _params(dw, nrhs, **kw):
    return dw.dw_default_params(m=16, k=4, tol=1e-10, sap_cycles=3, mr_steps=3, nrhs=nrhs, **kw)


def _alone(dw, q):
    x = np.zeros_like(q["b"])
    c = dw.dw_create(q["dims"], q["block"], q["m0"])
    try:
        dw.dw_set_gauge(c, q["U"], False)
        dw.fgmresdr_solve(c, q["b"], x, _params(dw, q["nrhs"], host_buffers=1))
    finally:
        dw.dw_destroy(c)
    return x


def test_server_results_equal_alone_and_in_mix(dw):
    reqs = _requests()
    srv = dw.dw_server_create(8 << 30, 4)
    try:
        ids, xs, keep = [], [], []
        for q in reqs:
            x = np.zeros_like(q["b"])
            r = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], x, _params(dw, q["nrhs"]))
            keep.append(r)
            ids.append(dw.dw_server_submit(srv, r))
            xs.append(x)
        for rid in ids:
            status, S, lat = dw.dw_server_wait(srv, rid, 300)
            assert status == dw.DW_OK and lat > 0
        info = dw.dw_server_info(srv)
        assert info["completed"] == len(reqs) and info["running"] == 0
        assert info["in_use_bytes"] <= info["budget_bytes"]  # idle cached contexts only
        # the requests really overlapped: several were solving at the same time
        assert info["peak_running"] >= 2
    finally:
        dw.dw_server_destroy(srv)
    for q, x in zip(reqs, xs):
        for r in range(q["nrhs"]):
            res = q["b"][r] - oracle.dw(q["U"], x[r], q["dims"], q["m0"])
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(q["b"][r])
        x1 = _alone(dw, q)
        assert np.abs(x1 - x).max() <= 1e-13 * np.abs(x1).max()


def test_server_respects_memory_budget(dw):
    reqs = _requests()
    bytes_ = []
    srv0 = None
    for q in reqs:
        r = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], q["b"], _params(dw, q["nrhs"]))
        bytes_.append(dw.dw_request_bytes(r))
    budget = int(max(bytes_) * 1.5)  # at most one large request at a time
    srv = dw.dw_server_create(budget, 6)
    try:
        ids, keep, xs = [], [], []
        for q in reqs:
            x = np.zeros_like(q["b"])
            r = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], x, _params(dw, q["nrhs"]))
            keep.append(r)
            xs.append(x)
            ids.append(dw.dw_server_submit(srv, r))
        for rid in ids:
            status, _, _ = dw.dw_server_wait(srv, rid, 300)
            assert status == dw.DW_OK
        info = dw.dw_server_info(srv)
        assert info["peak_bytes"] <= budget
        assert info["completed"] == len(reqs)
    finally:
        dw.dw_server_destroy(srv)


def test_server_rejects_and_cancels(dw):
    q = _requests()[5]
    x = np.zeros_like(q["b"])
    r = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], x, _params(dw, q["nrhs"]))
    small = dw.dw_server_create(1 << 20, 1)
    try:
        with pytest.raises(dw.DwError) as e:
            dw.dw_server_submit(small, r)
        assert e.value.code == dw.DW_ENOMEM
    finally:
        dw.dw_server_destroy(small)
    srv = dw.dw_server_create(8 << 30, 1)
    try:
        keep, ids = [], []
        for _ in range(4):
            xx = np.zeros_like(q["b"])
            rr = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], xx, _params(dw, q["nrhs"]))
            keep.append((rr, xx))
            ids.append(dw.dw_server_submit(srv, rr))
        dw.dw_server_cancel(srv, ids[-1])  # one slot: the last request is still queued
        status, _, _ = dw.dw_server_wait(srv, ids[-1], 60)
        assert status == dw.DW_ECANCELLED
        for rid in ids[:-1]:
            status, _, _ = dw.dw_server_wait(srv, rid, 300)
            assert status == dw.DW_OK
    finally:
        dw.dw_server_destroy(srv)


def test_server_reuses_resident_gauge_field(dw):
    """A second request on the same gauge buffer takes over the cached context
    (gauge copy and workspace stay on the device) and gives the same answer."""
    q = _requests()[1]
    srv = dw.dw_server_create(8 << 30, 1)
    try:
        xs, keep = [], []
        for _ in range(2):
            x = np.zeros_like(q["b"])
            r = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], x, _params(dw, q["nrhs"]))
            keep.append(r)
            xs.append(x)
            rid = dw.dw_server_submit(srv, r)
            status, _, _ = dw.dw_server_wait(srv, rid, 300)
            assert status == dw.DW_OK
        assert dw.dw_server_info(srv)["reused"] == 1
        assert np.array_equal(xs[0], xs[1])
    finally:
        dw.dw_server_destroy(srv)


def test_server_cancels_a_running_request(dw):
    """A request that would run for long (an unreachable tolerance) is
    cancelled while it solves: it stops between two Arnoldi steps with
    DW_ECANCELLED, the server stays usable, and the next request on the same
    gauge field (taking over the cancelled request's context) is exact."""
    import time

    q = _requests()[1]
    srv = dw.dw_server_create(8 << 30, 1)
    try:
        x = np.zeros_like(q["b"])
        # restarted FGMRES (no eigenproblem to break down at the rounding floor);
        # 2000 cycles bound the request to seconds should the cancel be missed
        P = dw.dw_default_params(m=16, k=0, tol=1e-30, max_cycles=2000, sap_cycles=3, mr_steps=3,
                                 nrhs=q["nrhs"])
        r = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], x, P)
        rid = dw.dw_server_submit(srv, r)
        t0 = time.time()
        while dw.dw_server_info(srv)["running"] == 0 and time.time() - t0 < 60:
            time.sleep(0.01)
        time.sleep(0.2)  # a few hundred steps
        dw.dw_server_cancel(srv, rid)
        status, S, lat = dw.dw_server_wait(srv, rid, 60)
        assert status == dw.DW_ECANCELLED
        assert S.iterations > 0
        with pytest.raises(dw.DwError):
            dw.dw_server_cancel(srv, rid)  # finished now
        x2 = np.zeros_like(q["b"])
        r2 = dw.make_request(q["dims"], q["block"], q["m0"], q["U"], q["b"], x2, _params(dw, q["nrhs"]))
        status, _, _ = dw.dw_server_wait(srv, dw.dw_server_submit(srv, r2), 300)
        assert status == dw.DW_OK
        assert dw.dw_server_info(srv)["reused"] == 1
        assert np.array_equal(x2, _alone(dw, q))
    finally:
        dw.dw_server_destroy(srv)
