"""Edge cases of the solver through the C ABI: a zero right-hand side, a batch
that mixes a zero and non-zero right-hand sides (per-rhs convergence masks),
an exact initial guess, the largest parameters the ABI accepts (nrhs = 16,
m = 63, k = 16), and parameters it must reject."""

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


def dev(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).reshape(-1).copy()).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


@pytest.fixture(scope="module")
def tiny():
    cfg = fg.lattice_configs()["tiny_4x4x4x4"]
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    return cfg, U


def _ctx(dw, cfg, U):
    h = dw.dw_create(cfg["dims"], cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    Ud = dev(U)
    dw.dw_set_gauge(h, Ud, True)
    return h, Ud


def _params(dw, cfg, **kw):
    opts = dict(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"], mr_steps=cfg["mr_steps"])
    opts.update(kw)
    return dw.dw_default_params(**opts)


def test_zero_rhs_gives_zero_solution(dw, tiny):
    cfg, U = tiny
    h, _ = _ctx(dw, cfg, U)
    try:
        b = np.zeros((fg.volume(cfg["dims"]), 4, 3), dtype=np.complex128)
        x = dev(np.ones_like(b))
        S = dw.fgmresdr_solve(h, dev(b), x, _params(dw, cfg))
        assert S.converged == 1 and S.iterations == 0
        assert np.abs(host(x, b.shape)).max() == 0.0
    finally:
        dw.dw_destroy(h)


def test_batch_with_a_zero_rhs(dw, tiny):
    cfg, U = tiny
    h, _ = _ctx(dw, cfg, U)
    try:
        bs = fg.gaussian_source(cfg["dims"], 21, nrhs=3)
        bs[1] = 0.0
        x = torch.zeros(bs.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(h, dev(bs), x, _params(dw, cfg, nrhs=3))
        xs = host(x, bs.shape)
        assert S.converged == 3
        assert S.iterations_rhs[1] == 0 and S.iterations_rhs[0] > 0 and S.iterations_rhs[2] > 0
        assert np.abs(xs[1]).max() == 0.0
        for r in (0, 2):
            rr = bs[r] - oracle.dw(U, xs[r], cfg["dims"], cfg["m0"])
            assert np.linalg.norm(rr) <= cfg["tol"] * np.linalg.norm(bs[r])
    finally:
        dw.dw_destroy(h)


def test_exact_initial_guess_needs_no_iteration(dw, tiny):
    cfg, U = tiny
    h, _ = _ctx(dw, cfg, U)
    try:
        b = fg.gaussian_source(cfg["dims"], 22)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        dw.fgmresdr_solve(h, dev(b), x, _params(dw, cfg, tol=1e-12))
        S = dw.fgmresdr_solve(h, dev(b), x, _params(dw, cfg, use_x0=1))
        assert S.converged == 1 and S.iterations == 0
    finally:
        dw.dw_destroy(h)


def test_largest_accepted_parameters(dw, tiny):
    cfg, U = tiny
    h, _ = _ctx(dw, cfg, U)
    try:
        bs = fg.gaussian_source(cfg["dims"], 23, nrhs=dw.DW_MAX_RHS)
        x = torch.zeros(bs.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(h, dev(bs), x, _params(dw, cfg, m=63, k=16, nrhs=dw.DW_MAX_RHS))
        xs = host(x, bs.shape)
        assert S.converged == dw.DW_MAX_RHS
        for r in range(0, dw.DW_MAX_RHS, 5):
            rr = bs[r] - oracle.dw(U, xs[r], cfg["dims"], cfg["m0"])
            assert np.linalg.norm(rr) <= cfg["tol"] * np.linalg.norm(bs[r])
    finally:
        dw.dw_destroy(h)


@pytest.mark.parametrize("kw", [dict(m=64), dict(k=20), dict(m=10, k=10), dict(nrhs=17), dict(tol=0.0),
                                dict(outer_prec=2), dict(outer_prec=1, sap_prec=0)])
def test_invalid_parameters_rejected(dw, tiny, kw):
    cfg, U = tiny
    h, _ = _ctx(dw, cfg, U)
    try:
        b = fg.gaussian_source(cfg["dims"], 24, nrhs=kw.get("nrhs", 1))
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        with pytest.raises(dw.DwError) as e:
            dw.fgmresdr_solve(h, dev(b), x, _params(dw, cfg, **kw))
        assert e.value.code == dw.DW_EINVAL
    finally:
        dw.dw_destroy(h)
