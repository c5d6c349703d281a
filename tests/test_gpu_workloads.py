"""GPU tests of the remaining workloads and solver properties, through the C ABI:

* the mixed-precision 32^3 x 64 workload (min |lambda| ~ 1e-3): FGMRES-DR(40, 16)
  with FP16 and BF16 SAP storage reaches a true residual <= 1e-10, computed
  with the oracle's FP64 D;
* SAP as a stand-alone solver (Sec. 3; Sec. 6, Fig. 5): s cycles of the GPU
  preconditioner equal the oracle's s SAP iterations, the residual falls for
  a mass above the spectral edge and grows for one below it;
* right-hand sides scaled by 1e+30 and 1e-30 (outside the useful range of
  FP32 squares) solve like unscaled ones;
* the flexible Arnoldi relation A Z_m = V_{m+1} Hhat_m (Eq. "arnoldilike")
  and the orthonormality of V, read back from the GPU basis of the 16^3 x 32
  workload's last cycle, for the double-float and the FP32 basis;
* dw_cancel stops a solve running in another thread.
"""

import threading
import time

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


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _ctx(dw, dims, block, m0, Ud):
    c = dw.dw_create(dims, block, m0, torch.cuda.current_stream().cuda_stream)
    dw.dw_set_gauge(c, Ud, True)
    return c


# --------------------------------------------------------------------------- 32^3 x 64, FP16 / BF16 SAP
@pytest.fixture(scope="module")
def mixed():
    cfg = fg.lattice_configs()["mixed_32x32x32x64"]
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    return cfg, U


@pytest.mark.parametrize("sap_prec", [2, 3])
def test_mixed_32x32x32x64_deflated_solve_reaches_tolerance(dw, mixed, sap_prec):
    cfg, U = mixed
    dims = cfg["dims"]
    b = fg.gaussian_source(dims, 1)
    ctx = _ctx(dw, dims, cfg["block"], cfg["m0"], dev(U))
    try:
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], sap_prec=sap_prec, matvec_prec=1)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(ctx, dev(b), x, P)
        xh = host(x, b.shape)
    finally:
        dw.dw_destroy(ctx)
    assert S.converged == 1
    r = b - oracle.dw(U, xh, dims, cfg["m0"])
    assert np.linalg.norm(r) <= cfg["tol"] * np.linalg.norm(b)
    assert abs(S.true_rel_res[0] - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-12


# --------------------------------------------------------------------------- SAP as a solver
SAP_DIMS, SAP_BLOCK, SAP_NMR = (8, 8, 8, 16), (4, 4, 4, 4), 4


@pytest.fixture(scope="module")
def sapfield():
    eps = 0.6
    U = fg.gauge_field(SAP_DIMS, eps, 0)
    edge = fg.spectral_edges()[fg.edge_key(SAP_DIMS, eps, 0)]["edge_re"]
    return U, edge


@pytest.mark.parametrize("delta", [0.2, -0.2])
def test_sap_as_solver_matches_oracle_and_converges_or_diverges(dw, sapfield, delta):
    """x_s = M_s b (s SAP cycles from 0) on the GPU (FP32) equals the oracle's
    s SAP iterations; the residual ||b - D x_s|| falls monotonically for a
    mass above the spectral edge (delta > 0) and, below it, grows to more
    than ten times its minimum within 24 cycles (Sec. 3, Fig. 5)."""
    U, edge = sapfield
    m0 = delta - edge
    b = fg.gaussian_source(SAP_DIMS, 1)
    bn = np.linalg.norm(b)
    ctx = _ctx(dw, SAP_DIMS, SAP_BLOCK, m0, dev(U))
    hist_gpu, hist_orc = [], []
    x_orc = np.zeros_like(b)
    try:
        bd = dev(b)
        z = torch.empty_like(bd)
        for s in range(1, 25):
            dw.sap_precondition(ctx, bd, z, s, SAP_NMR, dw.DW_F32, 1)
            xg = host(z, b.shape)
            x_orc = oracle.sap(U, b, SAP_DIMS, SAP_BLOCK, m0, 1, SAP_NMR, x0=x_orc)
            assert rel2(xg, x_orc) <= 1e-4, s
            hist_gpu.append(np.linalg.norm(b - oracle.dw(U, xg, SAP_DIMS, m0)) / bn)
            hist_orc.append(np.linalg.norm(b - oracle.dw(U, x_orc, SAP_DIMS, m0)) / bn)
    finally:
        dw.dw_destroy(ctx)
    hg, ho = np.array(hist_gpu), np.array(hist_orc)
    assert np.all(np.abs(hg - ho) <= 1e-3 * ho + 1e-6)
    if delta > 0:
        assert np.all(np.diff(hg) < 0)
        assert hg[-1] < 1e-4
    else:
        assert hg.argmin() <= 8
        assert hg[-1] > 10 * hg.min()


# --------------------------------------------------------------------------- scaled right-hand sides
@pytest.mark.parametrize("outer", [4, 1])
def test_extreme_rhs_scales_solve_like_unscaled(dw, sapfield, outer):
    U, edge = sapfield
    m0 = 0.05 - edge
    b = fg.gaussian_source(SAP_DIMS, 3)
    ctx = _ctx(dw, SAP_DIMS, SAP_BLOCK, m0, dev(U))
    xs, stats = {}, {}
    try:
        P = dw.dw_default_params(m=30, k=10, tol=1e-10, sap_cycles=5, mr_steps=4, sap_prec=1, matvec_prec=1,
                                 outer_prec=outer)
        for scale in (1.0, 1e30, 1e-30):
            bs = b * scale
            x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
            stats[scale] = dw.fgmresdr_solve(ctx, dev(bs), x, P)
            xs[scale] = host(x, b.shape)
            r = bs - oracle.dw(U, xs[scale], SAP_DIMS, m0)
            assert np.isfinite(xs[scale]).all()
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(bs), scale
    finally:
        dw.dw_destroy(ctx)
    for scale in (1e30, 1e-30):
        # two solutions of the same system to a residual of 1e-10 differ by at
        # most cond(D) * 2e-10 (cond ~ 8 / 0.05 here)
        assert rel2(xs[scale] / scale, xs[1.0]) <= 1e-6
        if outer != 1:
            # FP64-class outer vectors: the solve does not depend on the scale
            # (the FP32 basis of the single-precision scheme takes a different
            # number of steps for every rounding of b; only its result is checked)
            assert stats[scale].iterations == stats[1.0].iterations


# --------------------------------------------------------------------------- the GPU basis
@pytest.fixture(scope="module")
def wilson():
    cfg = fg.lattice_configs()["wilson_16x16x16x32"]
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    return cfg, U


# ||V^H V - I||_max, and the relation ||D z_j - V Hhat e_j|| / ||D z_j|| per
# column. The columns the last cycle added (j >= k) hold the relation to the
# rounding of w = D z in FP32. The k rotated columns of a deflated cycle carry
# in row k the explicit residual injected by the refinement of Sec. 5.7 in
# place of V_{m+1} q_{k+1}, so there the relation holds only as well as the
# explicit and the updated residual agree in direction (measured 1e-3 to 1e-2).
# The double-float basis stays orthogonal to 2e-11; the FP32 basis of the
# single-precision scheme, whose second Gram-Schmidt pass is taken only below
# ||w'|| / ||w|| = 6e-3, had lost orthogonality to 7e-4 by its last restart.
BASIS_TOL = {4: dict(orth=1e-10, new=2e-6, rotated=5e-2), 1: dict(orth=3e-3, new=2e-6, rotated=5e-2)}


@pytest.mark.parametrize("outer", [4, 1])
def test_gpu_basis_is_orthonormal_and_satisfies_the_arnoldi_relation(dw, wilson, outer):
    cfg, U = wilson
    dims = cfg["dims"]
    V = fg.volume(dims)
    b = fg.gaussian_source(dims, 1)
    ctx = _ctx(dw, dims, cfg["block"], cfg["m0"], dev(U))
    try:
        P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                 mr_steps=cfg["mr_steps"], sap_prec=1, matvec_prec=1, outer_prec=outer)
        x = torch.zeros(b.size * 2, dtype=torch.float64, device="cuda")
        S = dw.fgmresdr_solve(ctx, dev(b), x, P)
        assert S.converged == 1
        mm = dw.dw_debug_basis(ctx, 0)
        assert mm >= 1
        Vd = torch.empty((mm + 1) * 24 * V, dtype=torch.float64, device="cuda")
        Zd = torch.empty(mm * 24 * V, dtype=torch.float64, device="cuda")
        H = np.zeros(((mm + 1) * mm), dtype=np.complex128)
        assert dw.dw_debug_basis(ctx, 0, Vd, Zd, H, 64) == mm
        Vh = host(Vd, (mm + 1, 12 * V))
        Zh = host(Zd, (mm, 12 * V))
    finally:
        dw.dw_destroy(ctx)
    H = H.reshape(mm + 1, mm)
    orth = np.abs(Vh.conj() @ Vh.T - np.eye(mm + 1)).max()
    DZ = np.stack([oracle.dw(U, Zh[j].reshape(V, 4, 3), dims, cfg["m0"]).reshape(-1) for j in range(mm)])
    R = DZ - H.T @ Vh
    col = np.linalg.norm(R, axis=1) / np.linalg.norm(DZ, axis=1)
    # a deflated last cycle has a dense leading (k+1) x k block; a plain one is Hessenberg throughout
    k = cfg["k"]
    deflated = mm > k and np.abs(H[k + 1:, :k]).max(initial=0.0) == 0.0 and np.abs(H[2:k + 1, 0]).max() > 0
    first_new = k if deflated else 0
    tol = BASIS_TOL[outer]
    print(f"outer {outer}: {mm} columns ({'deflated' if deflated else 'plain'} cycle), "
          f"||V^H V - I||_max = {orth:.2e}, relation new columns {col[first_new:].max():.2e}"
          + (f", rotated columns {col[:k].max():.2e}" if deflated else ""))
    assert orth <= tol["orth"]
    assert col[first_new:].max() <= tol["new"]
    if deflated:
        assert col[:k].max() <= tol["rotated"]
    # Hhat's shape: below the subdiagonal only inside the leading (k+1) x k block
    for j in range(mm):
        low = H[max(j + 2, k + 1 if (deflated and j < k) else j + 2):, j]
        assert np.abs(low).max(initial=0.0) == 0.0


# --------------------------------------------------------------------------- dw_cancel
def test_dw_cancel_stops_a_running_solve(dw, sapfield):
    U, edge = sapfield
    m0 = 0.05 - edge
    b = fg.gaussian_source(SAP_DIMS, 4)
    ctx = _ctx(dw, SAP_DIMS, SAP_BLOCK, m0, dev(U))
    try:
        # restarted FGMRES towards an unreachable tolerance, bounded by its cycles
        P = dw.dw_default_params(m=20, k=0, tol=1e-30, max_cycles=3000, sap_cycles=2, mr_steps=2, sap_prec=1,
                                 matvec_prec=1)
        bd = dev(b)
        x = torch.zeros_like(bd)
        torch.cuda.synchronize()
        out = {}

        def run():
            t = time.time()
            out["S"] = dw.fgmresdr_solve(ctx, bd, x, P, allow_cancelled=True, allow_notconv=True)
            out["t"] = time.time() - t

        th = threading.Thread(target=run)
        th.start()
        time.sleep(0.5)
        dw.dw_cancel(ctx)
        th.join(120)
        assert not th.is_alive()
        assert out["S"].status == dw.DW_ECANCELLED
        assert out["S"].iterations > 0
        # the context stays usable: a normal solve afterwards converges
        P2 = dw.dw_default_params(m=30, k=10, tol=1e-10, sap_prec=1, matvec_prec=1)
        x2 = torch.zeros_like(bd)
        S2 = dw.fgmresdr_solve(ctx, bd, x2, P2)
        assert S2.converged == 1
    finally:
        dw.dw_destroy(ctx)
