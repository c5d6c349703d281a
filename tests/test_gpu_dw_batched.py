"""Several right-hand sides in one stencil launch against one launch per
right-hand side and against the FP64 oracle.

The CTAs of a multi-rhs launch run the same operations on each right-hand
side as a single-rhs launch, so the two must agree bit for bit: for every
storage precision, with the clover term, with a last thread block that runs
past the end of the lattice and with the most right-hand sides a launch
takes. A batched solve with converged right-hand sides masked out matches
single solves to the solver tolerance.
"""

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


CASES = [
    ((8, 8, 8, 16), (4, 4, 4, 4)),
    ((6, 6, 6, 6), (3, 3, 3, 3)),   # 1296 sites: the last tile is partly outside the lattice
    ((2, 2, 2, 2), (1, 1, 1, 1)),   # 16 sites: one tile, half empty; n + mu == n - mu
    ((6, 4, 2, 6), (3, 2, 1, 3)),
]


@pytest.mark.parametrize("dims,block", CASES)
@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("nrhs", [2, 5, 16])
def test_batched_equals_single(dw, dims, block, prec, nrhs):
    U = fg.gauge_field(dims, 0.5, seed=11)
    src = fg.gaussian_source(dims, 12, nrhs=nrhs)
    h = dw.dw_create(dims, block, -0.3, torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(h, Ud, True)
        ind = dev(src)
        out = torch.full_like(ind, float("nan"))
        dw.dw_apply(h, ind, out, prec, nrhs)
        n = ind.numel() // nrhs
        for r in range(nrhs):
            one = torch.full_like(ind[:n], float("nan"))
            dw.dw_apply(h, ind[r * n:(r + 1) * n].clone(), one, prec, 1)
            assert torch.equal(out[r * n:(r + 1) * n], one), r
    finally:
        dw.dw_destroy(h)


@pytest.mark.parametrize("prec", [1, 2])
def test_batched_equals_single_clover(dw, prec):
    dims, block, nrhs = (8, 8, 8, 16), (4, 4, 4, 4), 3
    U = fg.gauge_field(dims, 0.5, seed=11)
    src = fg.gaussian_source(dims, 13, nrhs=nrhs)
    h = dw.dw_create(dims, block, -0.1, torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(h, Ud, True)
        dw.dw_set_clover(h, 1.91)
        ind = dev(src)
        out = torch.empty_like(ind)
        dw.dw_apply(h, ind, out, prec, nrhs)
        n = ind.numel() // nrhs
        for r in range(nrhs):
            one = torch.empty_like(ind[:n])
            dw.dw_apply(h, ind[r * n:(r + 1) * n].clone(), one, prec, 1)
            assert torch.equal(out[r * n:(r + 1) * n], one), r
    finally:
        dw.dw_destroy(h)


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (2, 5e-3), (3, 3e-2)])
def test_batched_matches_oracle(dw, prec, tol):
    dims, block, nrhs = (6, 6, 6, 6), (3, 3, 3, 3), 4
    m0 = -0.3
    U = fg.gauge_field(dims, 0.5, seed=2)
    src = fg.gaussian_source(dims, 14, nrhs=nrhs)
    h = dw.dw_create(dims, block, m0, torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(h, Ud, True)
        out = torch.empty(src.size * 2, dtype=torch.float64, device="cuda")
        dw.dw_apply(h, dev(src), out, prec, nrhs)
        got = out.cpu().numpy().view(np.complex128).reshape(src.shape)
    finally:
        dw.dw_destroy(h)
    for r in range(nrhs):
        ref = oracle.dw(U, src[r], dims, m0)
        err = np.abs(got[r] - ref).max() / np.abs(ref).max()
        assert err <= tol, (r, err)


def test_batched_solver_rhs_subset(dw):
    """In the batched solve the stencil runs with some right-hand sides
    masked out (converged ones): the batched solve of 3 rhs gives the same
    solutions as three single solves, to the solver tolerance."""
    cfg = fg.lattice_configs()["tiny_4x4x4x4"]
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(cfg["dims"], 21, nrhs=3)
    h = dw.dw_create(cfg["dims"], cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    try:
        Ud = dev(U)
        dw.dw_set_gauge(h, Ud, True)
        P3 = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                  mr_steps=cfg["mr_steps"], nrhs=3, sap_prec=dw.DW_F32, matvec_prec=dw.DW_F32)
        bd = dev(b)
        x3 = torch.zeros_like(bd)
        S3 = dw.fgmresdr_solve(h, bd, x3, P3)
        assert S3.converged == 3
        n = bd.numel() // 3
        P1 = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                  mr_steps=cfg["mr_steps"], nrhs=1, sap_prec=dw.DW_F32, matvec_prec=dw.DW_F32)
        for r in range(3):
            x1 = torch.zeros_like(bd[:n])
            dw.fgmresdr_solve(h, bd[r * n:(r + 1) * n].clone(), x1, P1)
            xr = x3[r * n:(r + 1) * n]
            assert (torch.linalg.norm(xr - x1) / torch.linalg.norm(x1)).item() < 1e-8
    finally:
        dw.dw_destroy(h)
