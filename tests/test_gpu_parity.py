"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Element-wise comparisons on seeded synthetic inputs at sizes the oracle
finishes in seconds (several domains/tiles and a ragged tail of the 256-site
thread blocks), plus edge cases: a 2^4 lattice (n + j == n - j), domains of
one site in a direction, several right-hand sides per launch.

Tolerances (relative, max-norm over the field unless stated):
  D:   FP64 1e-12, FP32 1e-5, FP16 storage 5e-3 (the stated ones), BF16 storage
       1e-2 (2.6 u of BF16)
  SAP: FP64 1e-11 (max-norm); FP32 2.4e-7 = 4 u, FP16 9.8e-4 = 2 u, BF16
       7.8e-3 = 2 u of the storage format (2-norm)
With 16-bit storage the rounding of the stored input and output dominates
(u = 2^-11 for FP16, 2^-8 for BF16; the FP32 arithmetic adds ~2^-24 per
operation), so the errors sit below one u: measured on these cases D 0.73 u
(FP16) and 0.9 u (BF16) in the max-norm, SAP 0.6 u (FP16, BF16) in the 2-norm.
FP32 SAP accumulates FP32 rounding over its MR steps and cycles: measured
1.4 u (2-norm), hence 4 u.
"""

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DW_TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3, 3: 1e-2}
SAP_TOL = {0: 1e-11, 1: 4 * 2.0 ** -24, 2: 2 * 2.0 ** -11, 3: 2 * 2.0 ** -8}


@pytest.fixture(scope="module")
def dw():
    import paper_1204_5463_gb300 as pkg

    return pkg


def dev(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).reshape(-1).copy()).cuda()


def host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


class Ctx:
    def __init__(self, dw, dims, block, m0, U):
        self.dw = dw
        self.h = dw.dw_create(dims, block, m0, torch.cuda.current_stream().cuda_stream)
        self.Ud = dev(U)
        dw.dw_set_gauge(self.h, self.Ud, True)

    def close(self):
        self.dw.dw_destroy(self.h)


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


LATTICES = [
    ((4, 4, 4, 4), (2, 2, 2, 2)),
    ((2, 2, 2, 2), (1, 1, 1, 1)),
    ((6, 4, 2, 6), (3, 2, 1, 3)),     # 288 sites: ragged tail of a 256-thread block
    ((8, 8, 8, 16), (4, 4, 4, 4)),
]


@pytest.mark.parametrize("dims,block", LATTICES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_dw_apply_matches_oracle(dw, dims, block, prec):
    U = fg.gauge_field(dims, 0.5, seed=1)
    psi = fg.gaussian_source(dims, 2)
    m0 = -0.3
    ref = oracle.dw(U, psi, dims, m0)
    c = Ctx(dw, dims, block, m0, U)
    try:
        out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda")
        dw.dw_apply(c.h, dev(psi), out, prec, 1)
        torch.cuda.synchronize()
        got = host(out, psi.shape)
    finally:
        c.close()
    assert relmax(got, ref) <= DW_TOL[prec]


def test_dw_apply_batched_rhs_equal_single(dw):
    dims, block = (6, 4, 2, 6), (3, 2, 1, 3)
    U = fg.gauge_field(dims, 0.5, seed=1)
    psi = fg.gaussian_source(dims, 3, nrhs=3)
    c = Ctx(dw, dims, block, 0.1, U)
    try:
        out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda")
        dw.dw_apply(c.h, dev(psi), out, 1, 3)
        got = host(out, psi.shape)
        for r in range(3):
            o1 = torch.empty(psi[r].size * 2, dtype=torch.float64, device="cuda")
            dw.dw_apply(c.h, dev(psi[r]), o1, 1, 1)
            assert np.array_equal(host(o1, psi[r].shape), got[r])
            assert relmax(got[r], oracle.dw(U, psi[r], dims, 0.1)) <= DW_TOL[1]
    finally:
        c.close()


SAP_CASES = [
    ((4, 4, 4, 4), (2, 2, 2, 2), 4, 4),
    ((8, 8, 8, 8), (4, 4, 4, 4), 2, 3),
    ((4, 8, 4, 4), (2, 4, 1, 2), 3, 2),
]


@pytest.mark.parametrize("dims,block,ncyc,nmr", SAP_CASES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_sap_precondition_matches_oracle(dw, dims, block, ncyc, nmr, prec):
    U = fg.gauge_field(dims, 0.4, seed=5)
    v = fg.gaussian_source(dims, 6)
    m0 = -0.2
    ref = oracle.sap(U, v, dims, block, m0, ncyc, nmr)
    c = Ctx(dw, dims, block, m0, U)
    try:
        z = torch.empty(v.size * 2, dtype=torch.float64, device="cuda")
        dw.sap_precondition(c.h, dev(v), z, ncyc, nmr, prec, 1)
        got = host(z, v.shape)
    finally:
        c.close()
    err = relmax(got, ref) if prec == 0 else rel2(got, ref)
    assert err <= SAP_TOL[prec], err


def _tiny():
    cfg = fg.lattice_configs()["tiny_4x4x4x4"]
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(cfg["dims"], 1)
    return cfg, U, b


def _solve(dw, cfg, U, b, nrhs=1, **kw):
    c = Ctx(dw, cfg["dims"], cfg["block"], cfg["m0"], U)
    try:
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], nrhs=nrhs)
        for k_, v_ in kw.items():
            setattr(P, k_, v_)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(c.h, dev(b), x, P)
        return host(x, b.shape), S
    finally:
        c.close()


@pytest.mark.parametrize("outer", [0, 4])
def test_fgmresdr_fp64_matches_oracle_iterates(dw, outer):
    """FP64 SAP and FP64 Arnoldi product: same decisions as the oracle, so the
    same number of iterations and cycles, and the same solution to ~cond*eps
    (outer vectors in FP64, or double-float with a 48-bit significand)."""
    cfg, U, b = _tiny()
    ref = oracle.solve(U, b, cfg["dims"], cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"], cfg["m"],
                       cfg["k"], cfg["tol"])
    x, S = _solve(dw, cfg, U, b, sap_prec=0, matvec_prec=0, outer_prec=outer)
    assert S.converged == 1
    assert S.iterations == ref.iterations and S.cycles == ref.cycles
    assert rel2(x.reshape(-1), ref.x) <= 1e-9
    r = b - oracle.dw(U, x, cfg["dims"], cfg["m0"])
    assert np.linalg.norm(r) <= cfg["tol"] * np.linalg.norm(b)


@pytest.mark.parametrize("sap_prec", [1, 2, 3])
def test_fgmresdr_low_precision_sap_converges(dw, sap_prec):
    """Flexible outer loop with FP32/FP16/BF16 SAP: converges to the FP64 true
    residual tol (checked with the oracle's D), close to the oracle solution."""
    cfg, U, b = _tiny()
    ref = oracle.solve(U, b, cfg["dims"], cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"], cfg["m"],
                       cfg["k"], cfg["tol"])
    x, S = _solve(dw, cfg, U, b, sap_prec=sap_prec, matvec_prec=1)
    assert S.converged == 1
    r = b - oracle.dw(U, x, cfg["dims"], cfg["m0"])
    assert np.linalg.norm(r) <= cfg["tol"] * np.linalg.norm(b)
    assert S.true_rel_res[0] <= cfg["tol"]
    # cond(D) ~ 30 on this lattice: both solutions are within cond*tol of x*
    assert rel2(x.reshape(-1), ref.x) <= 100 * cfg["tol"]
    if sap_prec == 1:
        assert abs(S.iterations - ref.iterations) <= max(3, 0.15 * ref.iterations)


@pytest.mark.parametrize("sap_prec", [1, 2])
def test_fgmresdr_fp32_basis_converges(dw, sap_prec):
    """Single-precision Arnoldi process with double-float refinement (Sec. 5.7):
    the FP32 basis still reaches the 1e-10 true residual (checked with the
    oracle's D), within cond*tol of the oracle solution, in a comparable number
    of Arnoldi steps."""
    cfg, U, b = _tiny()
    ref = oracle.solve(U, b, cfg["dims"], cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"], cfg["m"],
                       cfg["k"], cfg["tol"])
    x, S = _solve(dw, cfg, U, b, sap_prec=sap_prec, matvec_prec=1, outer_prec=1)
    assert S.converged == 1
    r = b - oracle.dw(U, x, cfg["dims"], cfg["m0"])
    assert np.linalg.norm(r) <= cfg["tol"] * np.linalg.norm(b)
    assert rel2(x.reshape(-1), ref.x) <= 100 * cfg["tol"]
    assert S.iterations <= 1.5 * ref.iterations + 5


def test_fgmresdr_fp32_basis_larger_lattice(dw):
    """8^3 x 16 near criticality: the FP32 basis converges to the true residual
    with at most 30% more Arnoldi steps than the double-float basis."""
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    U = fg.gauge_field(dims, 0.45, seed=0)
    b = fg.gaussian_source(dims, 3)
    m0 = fg.tuned_m0(dims, 0.45, 0, 1e-2)  # smallest |eigenvalue| about 1e-2: a slow solve
    cfg = {"dims": dims, "block": block, "m0": m0, "m": 30, "k": 10, "tol": 1e-10, "sap_cycles": 5, "mr_steps": 4}
    x64, S64 = _solve(dw, cfg, U, b, sap_prec=1, matvec_prec=1, outer_prec=4)
    x32, S32 = _solve(dw, cfg, U, b, sap_prec=1, matvec_prec=1, outer_prec=1)
    assert S64.converged == 1 and S32.converged == 1
    r = b - oracle.dw(U, x32, dims, m0)
    assert np.linalg.norm(r) <= cfg["tol"] * np.linalg.norm(b)
    assert S32.iterations <= 1.3 * S64.iterations + 5


@pytest.mark.parametrize("k", [0, 3])
@pytest.mark.parametrize("outer", [0, 4, 1])
def test_fgmresdr_batched_equals_single(dw, k, outer):
    cfg, U, _ = _tiny()
    bs = fg.gaussian_source(cfg["dims"], 7, nrhs=3)
    kw = dict(k=k, outer_prec=outer) if outer != 1 else dict(k=k, outer_prec=outer, sap_prec=1, matvec_prec=1)
    xb, Sb = _solve(dw, cfg, U, bs, nrhs=3, **kw)
    assert Sb.converged == 3
    for r in range(3):
        x1, S1 = _solve(dw, cfg, U, bs[r], **kw)
        assert S1.iterations == Sb.iterations_rhs[r]
        assert rel2(xb[r].reshape(-1), x1.reshape(-1)) <= 1e-12


def test_fgmresdr_point_sources_batch(dw):
    cfg, U, _ = _tiny()
    b = fg.point_sources(cfg["dims"])
    x, S = _solve(dw, cfg, U, b, nrhs=12, sap_prec=2)
    assert S.converged == 12
    for r in range(12):
        rr = b[r] - oracle.dw(U, x[r], cfg["dims"], cfg["m0"])
        assert np.linalg.norm(rr) <= cfg["tol"] * np.linalg.norm(b[r])


def test_fgmresdr_host_buffers_equal_device(dw):
    cfg, U, b = _tiny()
    xd, Sd = _solve(dw, cfg, U, b)
    c = Ctx(dw, cfg["dims"], cfg["block"], cfg["m0"], U)
    try:
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], host_buffers=1)
        bh = np.ascontiguousarray(b, dtype=np.complex128)
        xh = np.zeros_like(bh)
        S = dw.fgmresdr_solve(c.h, bh, xh, P)
    finally:
        c.close()
    assert S.iterations == Sd.iterations
    assert np.array_equal(xh, xd)


def test_fgmresdr_nonfinite_rhs_reports_error(dw):
    cfg, U, b = _tiny()
    b = b.copy()
    b[3, 1, 2] = np.nan
    with pytest.raises(dw.DwError) as e:
        _solve(dw, cfg, U, b)
    assert e.value.code == dw.DW_ENONFINITE


def test_fgmresdr_iteration_limit(dw):
    cfg, U, b = _tiny()
    c = Ctx(dw, cfg["dims"], cfg["block"], cfg["m0"], U)
    try:
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=1e-14, sap_cycles=1, mr_steps=1, max_iterations=7)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(c.h, dev(b), x, P, allow_notconv=True)
        assert S.status == dw.DW_ENOTCONV and S.iterations == 7
    finally:
        c.close()


def test_profile_counters(dw):
    cfg, U, b = _tiny()
    c = Ctx(dw, cfg["dims"], cfg["block"], cfg["m0"], U)
    try:
        dw.dw_profile(c.h, True)
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"])
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(c.h, dev(b), x, P)
        prof = dw.dw_profile_read(c.h, reset=True)
    finally:
        c.close()
    assert prof["sap_sweep"]["launches"] == S.iterations * 2 * cfg["sap_cycles"]
    assert prof["dw_matvec"]["launches"] == S.iterations
    assert all(v["total_ms"] > 0 for v in prof.values())
