"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py
from the FP64 oracle only): the oracle still reproduces them (CPU), and the
CUDA path in FP64 reproduces them without running the oracle (GPU)."""

import json
import os

import numpy as np
import pytest

import fieldgen as fg

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "tiny_4x4x4x4_fgmresdr.json")


def load():
    with open(GOLD) as f:
        g = json.load(f)
    c = g["config"]
    U = fg.gauge_field(tuple(c["dims"]), c["eps"], c["seed"])
    b = fg.gaussian_source(tuple(c["dims"]), c["rhs_seed"])
    return g, c, U, b


def cplx(a):
    return np.array([complex(x, y) for x, y in a])


def test_oracle_reproduces_golden():
    import oracle

    g, c, U, b = load()
    res = oracle.solve(U, b, tuple(c["dims"]), tuple(c["block"]), c["m0"], c["sap_cycles"], c["mr_steps"], c["m"],
                       c["k"], c["tol"])
    assert res.iterations == g["iterations"] and res.cycles == g["cycles"]
    assert res.clean_restarts == g["clean_restarts"]
    for h, hg in zip(res.history, g["history"]):
        assert h[0] == hg[0]
        assert abs(h[2] - hg[2]) <= 1e-6 * hg[2]
    assert abs(np.linalg.norm(res.x) - g["x_norm"]) <= 1e-12 * g["x_norm"]
    Db = oracle.dw(U, b, tuple(c["dims"]), c["m0"]).reshape(-1)[:24]
    assert np.abs(Db - cplx(g["Db_head"])).max() <= 1e-13 * np.abs(cplx(g["Db_head"])).max()


@pytest.mark.gpu
def test_cuda_fp64_path_reproduces_golden():
    torch = pytest.importorskip("torch")
    import paper_1204_5463_gb300 as dw

    g, c, U, b = load()

    def dev(a):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        return torch.from_numpy(a.view(np.float64).reshape(-1).copy()).cuda()

    ctx = dw.dw_create(tuple(c["dims"]), tuple(c["block"]), c["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(ctx, Ud, True)
        bd = dev(b)
        out = torch.empty_like(bd)
        dw.dw_apply(ctx, bd, out, dw.DW_F64, 1)
        Db = out.cpu().numpy().view(np.complex128)[:24]
        ref = cplx(g["Db_head"])
        assert np.abs(Db - ref).max() <= 1e-12 * np.abs(ref).max()
        P = dw.dw_default_params(m=c["m"], k=c["k"], tol=c["tol"], sap_cycles=c["sap_cycles"],
                                 mr_steps=c["mr_steps"], sap_prec=dw.DW_F64, matvec_prec=dw.DW_F64,
                                 outer_prec=dw.DW_F64)
        x = torch.zeros_like(bd)
        S = dw.fgmresdr_solve(ctx, bd, x, P)
        assert S.iterations == g["iterations"] and S.cycles == g["cycles"]
        assert S.true_rel_res[0] <= c["tol"]
        assert abs(S.true_rel_res[0] - g["true_rel_res"]) <= 0.05 * g["true_rel_res"]
        xh = x.cpu().numpy().view(np.complex128)
        assert abs(np.linalg.norm(xh) - g["x_norm"]) <= 1e-9 * g["x_norm"]
        assert np.abs(xh[:24] - cplx(g["x_head"])).max() <= 1e-8 * np.abs(cplx(g["x_head"])).max()
        # the per-cycle residual history (the paper's plots): the same cycle
        # ends; implicit and explicit residuals agree while they lie well above
        # the rounding of the two Gram-Schmidt variants (MGS printed, CGS here)
        hist = dw.dw_residual_history(ctx, 0)
        assert [h[0] for h in hist] == [hg[0] for hg in g["history"]]
        for h, hg in zip(hist, g["history"]):
            for a, e in ((h[1], hg[1]), (h[2], hg[2])):
                assert abs(a - e) <= 1e-3 * e + 1e-13
    finally:
        dw.dw_destroy(ctx)
