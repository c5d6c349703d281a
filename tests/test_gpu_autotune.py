"""GPU test of the domain-tile autotuner: every candidate obeys the
red-black constraint of Sec. 2, the winner is the fastest converged
candidate, solving with it meets the tolerance, and the choice is cached."""

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).reshape(-1).copy()).cuda()


def test_autotune_picks_fastest_admissible_block():
    import paper_1204_5463_gb300 as dw

    dims = (8, 8, 8, 8)
    m0 = -0.2
    U = fg.gauge_field(dims, 0.4, seed=3)
    b = fg.gaussian_source(dims, 4)
    P = dw.dw_default_params(m=16, k=4, tol=1e-8, sap_cycles=3, mr_steps=3)
    best, table = dw.dw_autotune_block(dims, m0, _dev(U), _dev(b), P)
    assert len(table) >= 3
    for blk, secs, iters, status in table:
        for d, bb in zip(dims, blk):
            assert d % bb == 0 and (d // bb) % 2 == 0
        assert 32 <= np.prod(blk) <= 1024
    ok = [t for t in table if t[3] == dw.DW_OK]
    assert best == min(ok, key=lambda t: t[1])[0]
    # solving with the chosen block meets the tolerance (checked with the oracle's D)
    ctx = dw.dw_create(dims, best, m0)
    try:
        dw.dw_set_gauge(ctx, U, False)
        x = np.zeros_like(b)
        dw.fgmresdr_solve(ctx, np.ascontiguousarray(b), x,
                          dw.dw_default_params(m=16, k=4, tol=1e-10, sap_cycles=3, mr_steps=3, host_buffers=1))
    finally:
        dw.dw_destroy(ctx)
    r = b - oracle.dw(U, x, dims, m0)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    # cached: same answer without a table
    again, t2 = dw.dw_autotune_block(dims, m0, _dev(U), _dev(b), P, with_results=False)
    assert again == best and t2 == []


def test_autotune_sap_picks_fastest_converged_pair():
    """The (SAP cycles, MR steps) tuner times every pair of its grid on the
    given block and returns the fastest converged one; solving with it meets
    the tolerance (checked with the oracle's D); the choice is cached."""
    import paper_1204_5463_gb300 as dw

    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    m0 = -0.2
    U = fg.gauge_field(dims, 0.4, seed=3)
    b = fg.gaussian_source(dims, 4)
    P = dw.dw_default_params(m=16, k=4, tol=1e-8)
    best, table = dw.dw_autotune_sap(dims, block, m0, _dev(U), _dev(b), P)
    assert len(table) == 36
    assert {(t[0], t[1]) for t in table} == {(c, m) for c in (2, 3, 4, 5, 6, 8) for m in (3, 4, 5, 6, 8, 10)}
    ok = [t for t in table if t[4] == dw.DW_OK]
    assert best == min(ok, key=lambda t: t[2])[:2]
    ctx = dw.dw_create(dims, block, m0)
    try:
        dw.dw_set_gauge(ctx, U, False)
        x = np.zeros_like(b)
        dw.fgmresdr_solve(ctx, np.ascontiguousarray(b), x,
                          dw.dw_default_params(m=16, k=4, tol=1e-10, sap_cycles=best[0], mr_steps=best[1],
                                               host_buffers=1))
    finally:
        dw.dw_destroy(ctx)
    r = b - oracle.dw(U, x, dims, m0)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    again, t2 = dw.dw_autotune_sap(dims, block, m0, _dev(U), _dev(b), P, with_results=False)
    assert again == best and t2 == []
