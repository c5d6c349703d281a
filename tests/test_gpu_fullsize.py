"""GPU parity at the benchmark workloads' full sizes, in the launch
configuration bench.py times (4^4 domains, 256-thread SAP CTAs, FP32 SAP,
double-float Arnoldi basis):

* D on the full 16^3 x 32 and 24^3 x 48 lattices against the oracle's D,
  element by element (FP64, FP32, FP16 storage; same tolerances as the small
  lattices);
* one and five SAP cycles of the 16^3 x 32 workload against the oracle's
  Algorithm 2;
* the full 16^3 x 32 solve (double-float and FP32 basis): the true residual
  computed by the oracle's FP64 D is <= tol, a property that holds at any size;
  with an FP64 Arnoldi product its step count is the oracle's complete solve's
  (stored in tests/golden by tests/golden/make_golden.py) within 5%, and the
  FP32 product costs at most one extra cycle of refinement (Sec. 5.7);
* the 24^3 x 48 point-source solve (FP16 SAP), two of the twelve sources.
"""

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DW_TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}


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
def wilson():
    cfg = fg.lattice_configs()["wilson_16x16x16x32"]
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    return cfg, U


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dw_full_16x16x16x32(dw, wilson, prec):
    cfg, U = wilson
    psi = fg.gaussian_source(cfg["dims"], 11)
    ref = oracle.dw(U, psi, cfg["dims"], cfg["m0"])
    ctx = dw.dw_create(cfg["dims"], cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda")
        dw.dw_apply(ctx, dev(psi), out, prec, 1)
        got = host(out, psi.shape)
    finally:
        dw.dw_destroy(ctx)
    assert relmax(got, ref) <= DW_TOL[prec]


def test_dw_full_24x24x24x48_fp32(dw):
    dims = (24, 24, 24, 48)
    U = fg.gauge_field(dims, 0.5, 0)
    psi = fg.gaussian_source(dims, 7)
    ref = oracle.dw(U, psi, dims, -0.5)
    ctx = dw.dw_create(dims, (4, 4, 4, 4), -0.5, torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda")
        dw.dw_apply(ctx, dev(psi), out, 1, 1)
        got = host(out, psi.shape)
    finally:
        dw.dw_destroy(ctx)
    assert relmax(got, ref) <= DW_TOL[1]


@pytest.mark.parametrize("ncyc", [1, 5])
def test_sap_full_16x16x16x32_fp32(dw, wilson, ncyc):
    cfg, U = wilson
    v = fg.gaussian_source(cfg["dims"], 12)
    ref = oracle.sap(U, v, cfg["dims"], cfg["block"], cfg["m0"], ncyc, cfg["mr_steps"])
    ctx = dw.dw_create(cfg["dims"], cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        z = torch.empty(v.size * 2, dtype=torch.float64, device="cuda")
        dw.sap_precondition(ctx, dev(v), z, ncyc, cfg["mr_steps"], 1, 1)
        got = host(z, v.shape)
    finally:
        dw.dw_destroy(ctx)
    assert rel2(got, ref) <= 4 * 2.0 ** -24  # 4 u of FP32 (measured 1.4 u after 1 and 5 cycles)


@pytest.mark.parametrize("outer", [4, 1])
def test_solve_full_16x16x16x32(dw, wilson, outer):
    cfg, U = wilson
    b = fg.gaussian_source(cfg["dims"], 1)
    ctx = dw.dw_create(cfg["dims"], cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], sap_prec=1, matvec_prec=1, outer_prec=outer)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(ctx, dev(b), x, P)
        xh = host(x, b.shape)
    finally:
        dw.dw_destroy(ctx)
    assert S.converged == 1
    r = b - oracle.dw(U, xh, cfg["dims"], cfg["m0"])
    assert np.linalg.norm(r) <= cfg["tol"] * np.linalg.norm(b)
    assert 60 <= S.iterations <= 120  # the bench workload takes 81 steps


def test_point_sources_full_24x24x24x48(dw):
    cfg = fg.lattice_configs()["batched_24x24x24x48"]
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    b = fg.point_sources(dims)[[0, 7]]
    ctx = dw.dw_create(dims, cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], sap_prec=2, matvec_prec=1, nrhs=2)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(ctx, dev(b), x, P)
        xh = host(x, b.shape)
    finally:
        dw.dw_destroy(ctx)
    assert S.converged == 2
    for r in range(2):
        rr = b[r] - oracle.dw(U, xh[r], dims, cfg["m0"])
        assert np.linalg.norm(rr) <= cfg["tol"] * np.linalg.norm(b[r])


def test_solve_full_16x16x16x32_step_count_against_oracle(dw, wilson):
    import json
    import os

    cfg, U = wilson
    with open(os.path.join(os.path.dirname(__file__), "golden", "wilson_16x16x16x32_oracle.json")) as f:
        gold = json.load(f)
    if abs(gold["config"]["m0"] - cfg["m0"]) > 1e-12:
        pytest.skip("stored oracle solve is for another bare mass")
    b = fg.gaussian_source(cfg["dims"], 1)
    ctx = dw.dw_create(cfg["dims"], cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        steps = {}
        for mv in (0, 1):  # FP64 and FP32 Arnoldi product, FP32 SAP, double-float basis
            P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                     mr_steps=cfg["mr_steps"], sap_prec=1, matvec_prec=mv)
            x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
            S = dw.fgmresdr_solve(ctx, dev(b), x, P)
            assert S.converged == 1
            steps[mv] = S.iterations
    finally:
        dw.dw_destroy(ctx)
    n = gold["iterations"]
    assert abs(steps[0] - n) <= max(1, round(0.05 * n)), (steps, n)
    assert steps[1] <= n + (cfg["m"] - cfg["k"]), (steps, n)
