"""GPU parity of the clover-improved operator (the site-diagonal term of the
operators of Sec. 6) against the FP64 oracle: the clover field computed on
the device enters D, the SAP sweeps and the solver exactly as the oracle's
A does. Tolerances as for the plain operator."""

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CSW = 1.91
# the tolerances of tests/test_gpu_parity.py (derived there from the unit
# roundoff of the storage format)
DW_TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3, 3: 1e-2}
SAP_TOL = {0: 1e-11, 1: 4 * 2.0 ** -24, 2: 2 * 2.0 ** -11}


@pytest.fixture(scope="module")
def dw():
    import paper_1204_5463_gb300 as pkg

    return pkg


def dev(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).reshape(-1).copy()).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


class Ctx:
    def __init__(self, dw, dims, block, m0, U, csw=CSW):
        self.dw = dw
        self.h = dw.dw_create(dims, block, m0, torch.cuda.current_stream().cuda_stream)
        self.Ud = dev(U)
        dw.dw_set_gauge(self.h, self.Ud, True)
        dw.dw_set_clover(self.h, csw)

    def apply(self, psi, prec):
        out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda")
        self.dw.dw_apply(self.h, dev(psi), out, prec, 1)
        return host(out, psi.shape)

    def close(self):
        self.dw.dw_destroy(self.h)


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((6, 4, 2, 6), (3, 2, 1, 3)),
                                        ((8, 8, 8, 16), (4, 4, 4, 4))])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_clover_dw_matches_oracle(dw, dims, block, prec):
    U = fg.gauge_field(dims, 0.5, seed=41)
    psi = fg.gaussian_source(dims, 42)
    m0 = -0.3
    A = oracle.clover(U, dims, CSW)
    ref = oracle.dw(U, psi, dims, m0, A=A)
    c = Ctx(dw, dims, block, m0, U)
    try:
        got = c.apply(psi, prec)
    finally:
        c.close()
    assert relmax(got, ref) <= DW_TOL[prec]


def test_clover_off_and_gauge_update(dw):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = fg.gauge_field(dims, 0.5, seed=43)
    U2 = fg.gauge_field(dims, 0.7, seed=44)
    psi = fg.gaussian_source(dims, 45)
    c = Ctx(dw, dims, block, 0.1, U)
    try:
        c.dw.dw_set_clover(c.h, 0.0)
        assert relmax(c.apply(psi, 0), oracle.dw(U, psi, dims, 0.1)) <= 1e-12
        c.dw.dw_set_clover(c.h, CSW)
        U2d = dev(U2)
        c.dw.dw_set_gauge(c.h, U2d, True)  # the clover term follows the new links
        ref = oracle.dw(U2, psi, dims, 0.1, A=oracle.clover(U2, dims, CSW))
        assert relmax(c.apply(psi, 0), ref) <= 1e-12
    finally:
        c.close()


@pytest.mark.parametrize("dims,block,ncyc,nmr", [((4, 4, 4, 4), (2, 2, 2, 2), 3, 4),
                                                 ((8, 8, 8, 8), (4, 4, 4, 4), 2, 3)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_clover_sap_matches_oracle(dw, dims, block, ncyc, nmr, prec):
    U = fg.gauge_field(dims, 0.4, seed=46)
    v = fg.gaussian_source(dims, 47)
    m0 = -0.2
    A = oracle.clover(U, dims, CSW)
    ref = oracle.sap(U, v, dims, block, m0, ncyc, nmr, A=A)
    c = Ctx(dw, dims, block, m0, U)
    try:
        z = torch.empty(v.size * 2, dtype=torch.float64, device="cuda")
        dw.sap_precondition(c.h, dev(v), z, ncyc, nmr, prec, 1)
        got = host(z, v.shape)
    finally:
        c.close()
    err = relmax(got, ref) if prec == 0 else rel2(got, ref)
    assert err <= SAP_TOL[prec], err


def test_clover_fp64_solve_matches_oracle_iterates(dw):
    cfg = fg.lattice_configs()["tiny_4x4x4x4"]
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(dims, 1)
    A = oracle.clover(U, dims, CSW)
    ref = oracle.solve(U, b, dims, cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"], cfg["m"], cfg["k"],
                       cfg["tol"], clov=A)
    c = Ctx(dw, dims, cfg["block"], cfg["m0"], U)
    try:
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], sap_prec=0, matvec_prec=0, outer_prec=0)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(c.h, dev(b), x, P)
        xh = host(x, b.shape)
    finally:
        c.close()
    assert S.converged == 1 and ref.converged
    assert S.iterations == ref.iterations and S.cycles == ref.cycles
    assert rel2(xh.reshape(-1), ref.x) <= 1e-9


@pytest.mark.parametrize("sap_prec,outer", [(1, 4), (2, 4), (1, 1)])
def test_clover_solve_true_residual(dw, sap_prec, outer):
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    U = fg.gauge_field(dims, 0.45, seed=0)
    b = fg.gaussian_source(dims, 3)
    m0 = -0.3
    A = oracle.clover(U, dims, CSW)
    c = Ctx(dw, dims, block, m0, U)
    try:
        P = dw.dw_default_params(m=30, k=10, tol=1e-10, sap_cycles=5, mr_steps=4, sap_prec=sap_prec,
                                 matvec_prec=1, outer_prec=outer)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(c.h, dev(b), x, P)
        xh = host(x, b.shape)
    finally:
        c.close()
    assert S.converged == 1
    r = b - oracle.dw(U, xh, dims, m0, A=A)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def test_clover_sap_rejects_large_domains(dw):
    dims, block = (16, 8, 8, 8), (8, 4, 4, 4)  # 512-site domains
    U = fg.gauge_field(dims, 0.3, seed=48)
    v = fg.gaussian_source(dims, 49)
    c = Ctx(dw, dims, block, 0.0, U)
    try:
        z = torch.empty(v.size * 2, dtype=torch.float64, device="cuda")
        with pytest.raises(dw.DwError) as ei:
            dw.sap_precondition(c.h, dev(v), z, 1, 2, 1, 1)
        assert ei.value.code == dw.DW_EINVAL
    finally:
        c.close()


@pytest.mark.parametrize("outer", [4, 1])
def test_clover_batched_equals_single(dw, outer):
    """Several right-hand sides per launch (column tables in the SAP sweeps,
    the Arnoldi product and the residual) give the single-rhs iterates."""
    cfg = fg.lattice_configs()["tiny_4x4x4x4"]
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    bs = fg.gaussian_source(dims, 9, nrhs=3)
    c = Ctx(dw, dims, cfg["block"], cfg["m0"], U)
    try:
        P = dw.dw_default_params(m=cfg["m"], k=3, tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], sap_prec=1, matvec_prec=1, outer_prec=outer, nrhs=3)
        xb = torch.zeros(bs.size * 2, dtype=torch.float64, device="cuda")
        Sb = dw.fgmresdr_solve(c.h, dev(bs), xb, P)
        xbh = host(xb, bs.shape)
        assert Sb.converged == 3
        for r in range(3):
            P1 = dw.dw_default_params(m=cfg["m"], k=3, tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                      mr_steps=cfg["mr_steps"], sap_prec=1, matvec_prec=1, outer_prec=outer)
            x1 = torch.zeros(bs[r].size * 2, dtype=torch.float64, device="cuda")
            S1 = dw.fgmresdr_solve(c.h, dev(bs[r]), x1, P1)
            assert S1.iterations == Sb.iterations_rhs[r]
            assert rel2(xbh[r].reshape(-1), host(x1, bs[r].shape).reshape(-1)) <= 1e-12
    finally:
        c.close()
