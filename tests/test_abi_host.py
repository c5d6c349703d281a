"""Host-side checks of the C-ABI library (no GPU needed).

* the shared library loads and exports every function that include/*.h declares;
* the small dense FP64 routines of the outer loop (eigenproblem of Lemma 1a,
  QR of G_{k+1}, Givens least squares of Sec. 5.2 and 5.6, LU solve) agree with
  numpy.linalg on random matrices.
"""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dw():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1204_5463_gb300 as pkg

    return pkg


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][A-Za-z_0-9]*[\s*]+)+([a-z_][a-z_0-9]*)\s*\(", txt, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(dw):
    lib = ctypes.CDLL(dw.lib_path())
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"
    assert set(names) == set(dw.EXPORTED)


def test_error_reporting_without_gpu_work(dw):
    with pytest.raises(dw.DwError) as e:
        dw.dw_create((4, 4, 4, 3), (2, 2, 2, 1), 0.0)
    assert e.value.code == dw.DW_EINVAL
    assert "even" in dw.dw_last_error() or "divide" in dw.dw_last_error()
    with pytest.raises(dw.DwError):
        dw.dw_create((4, 4, 4, 4), (4, 4, 4, 4), 0.0)  # one domain per direction: no red-black


# extents whose product overflows 64 bits or wraps to a small value
WRAPPING_DIMS = [(1 << 16, 1 << 16, 1 << 16, 1 << 16), (2, 1 << 30, 1 << 30, 1 << 30), (2, 2, 2, -2),
                 ((1 << 31) - 1, 2, 2, 2)]


@pytest.mark.parametrize("dims", WRAPPING_DIMS)
def test_huge_or_wrapping_extents_are_rejected_before_any_gpu_work(dw, dims):
    with pytest.raises(dw.DwError) as e:
        dw.dw_create(dims, (2, 2, 2, 2), 0.0)
    assert e.value.code == dw.DW_EINVAL
    with pytest.raises(dw.DwError) as e:
        dw.dw_apply_f32_noalloc(dims, 0.0, 16, 16, 16)  # never dereferenced: rejected first
    assert e.value.code == dw.DW_EINVAL
    assert "4096" in dw.dw_last_error()


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40])
def test_dense_eig(dw, n):
    rng = np.random.default_rng(n)
    A = _crand(rng, n, n)
    lam = np.zeros(n, dtype=np.complex128)
    vec = np.zeros((n, n), dtype=np.complex128)
    dw.dw_dense_eig(n, A, lam, vec)
    ref = np.linalg.eigvals(A)
    for l in ref:
        assert np.min(np.abs(lam - l)) <= 1e-10 * max(1.0, abs(l))
    for kk in range(n):
        v = vec[:, kk]
        assert abs(np.linalg.norm(v) - 1) < 1e-12
        assert np.linalg.norm(A @ v - lam[kk] * v) <= 1e-10 * np.linalg.norm(A)


def test_dense_eig_harmonic_ritz_matrix(dw):
    """Eigenvalues of H_m + f h^H for a Hessenberg-like H (the Lemma 1a matrix)."""
    rng = np.random.default_rng(3)
    m = 30
    H = np.triu(_crand(rng, m + 1, m), -1)
    Hm, h = H[:m], H[m]
    f = np.linalg.solve(Hm.conj().T, h.conj())
    A = Hm + np.outer(f, h)
    lam = np.zeros(m, dtype=np.complex128)
    vec = np.zeros((m, m), dtype=np.complex128)
    dw.dw_dense_eig(m, np.ascontiguousarray(A), lam, vec)
    ref = np.linalg.eigvals(A)
    assert np.allclose(np.sort(np.abs(lam)), np.sort(np.abs(ref)), rtol=1e-9)


@pytest.mark.parametrize("rows,cols", [(5, 1), (21, 6), (41, 17)])
def test_dense_qr(dw, rows, cols):
    rng = np.random.default_rng(rows)
    G = _crand(rng, rows, cols)
    G[-1, : cols - 1] = 0  # the structure of G_{k+1}: last row zero except the last column
    Q = np.zeros((rows, cols), dtype=np.complex128)
    R = np.zeros((cols, cols), dtype=np.complex128)
    dw.dw_dense_qr(rows, cols, G, Q, R)
    assert np.abs(Q.conj().T @ Q - np.eye(cols)).max() < 1e-13
    assert np.abs(Q @ R - G).max() < 1e-12 * np.abs(G).max()
    assert np.all(np.abs(np.tril(R, -1)) == 0)
    d = np.diagonal(R)
    assert np.all(d.real > 0) and np.all(d.imag == 0)
    if cols > 1:
        assert np.abs(Q[-1, : cols - 1]).max() < 1e-15  # Q_k keeps the zero last row


@pytest.mark.parametrize("k", [0, 1, 5])
def test_dense_givens_least_squares(dw, k):
    rng = np.random.default_rng(10 + k)
    m = 25
    H = np.triu(_crand(rng, m + 1, m), -1)
    H[: k + 1, :k] = _crand(rng, k + 1, k)  # dense leading block of a deflated cycle
    H[k + 1:, :k] = 0
    c = np.zeros(m + 1, dtype=np.complex128)
    c[: k + 1] = _crand(rng, k + 1)
    eta = np.zeros(m, dtype=np.complex128)
    res = np.zeros(m)
    dw.dw_dense_lstsq(m + 1, m, k + 1, np.ascontiguousarray(H), c, eta, res)
    ref = np.linalg.lstsq(H, c, rcond=None)[0]
    assert np.linalg.norm(eta - ref) <= 1e-10 * np.linalg.norm(ref)
    for j in range(m):
        e = np.linalg.lstsq(H[:, : j + 1], c, rcond=None)[0]
        assert abs(res[j] - np.linalg.norm(c - H[:, : j + 1] @ e)) <= 1e-10 * np.linalg.norm(c)


def test_dense_solve(dw):
    rng = np.random.default_rng(1)
    A = _crand(rng, 30, 30)
    b = _crand(rng, 30)
    x = b.copy()
    dw.dw_dense_solve(30, A, x)
    assert np.linalg.norm(A @ x - b) < 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("k,outer", [(10, None), (0, None), (10, "f32")])
def test_request_bytes_formula(dw, k, outer):
    """Admission estimate: gauge copies (FP64, staging, FP32, FP16, double-float,
    the 16-bit SAP links packed per domain)
    + per-rhs Krylov workspace (V in the basis format; Z in FP32 when a 16-bit
    SAP is deflated, with the SAP output buffer; x, b, r; SAP input copy;
    canonical staging) + rotation scratch."""
    kw = dict(m=30, k=k, nrhs=3, sap_prec=dw.DW_F16)
    if outer == "f32":
        kw["outer_prec"] = dw.DW_F32
    P = dw.dw_default_params(**kw)
    dims = (16, 16, 16, 32)
    V = 16 * 16 * 16 * 32
    req = dw.make_request(dims, (4, 4, 4, 4), -0.6, 1, 1, 1, P)
    sb = 52 * V
    zb = 96 * V if k > 0 else sb
    fv = 96 * V if outer == "f32" else 192 * V
    gauge = 576 * V + 576 * V + 288 * V + 144 * V + 576 * V + 144 * V  # last: SAP links packed per domain
    per_rhs = 31 * fv + 30 * zb + 3 * 192 * V + sb + 24 * 8 * V
    per_rhs += sb if zb != sb else 0
    per_rhs += fv if outer == "f32" else 0
    expect = gauge + 3 * per_rhs + max(k, 1) * zb + (8 << 20)
    assert dw.dw_request_bytes(req) == expect


@pytest.mark.parametrize("prec,lb", [("f32", 288), ("f16", 144)])
def test_request_bytes_ragged_domains(dw, prec, lb):
    """The per-domain link images are laid out for whole warps: domains of
    3x2x1x3 = 18 sites are packed for 32-thread CTAs, so the image holds
    lb * 32 bytes per domain, not lb * 18."""
    P = dw.dw_default_params(m=20, k=5, nrhs=1, sap_prec=dw.PREC[prec])
    dims, block = (6, 4, 2, 6), (3, 2, 1, 3)
    V, ndom = 6 * 4 * 2 * 6, 16
    # the same request with one 288-site block (not a valid red-black
    # decomposition: only the estimate is compared) differs in the image term alone
    other = dw.dw_request_bytes(dw.make_request(dims, (6, 4, 2, 6), -0.3, 1, 1, 1, P))
    got = dw.dw_request_bytes(dw.make_request(dims, block, -0.3, 1, 1, 1, P))
    assert got - other == lb * 32 * ndom - lb * 288 * 1
