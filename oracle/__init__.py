"""FP64 CPU oracle of the SAP-preconditioned FGMRES-DR solver.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct statement of what
the GPU path computes. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it. It shares no code with the CUDA
library (``paper_1204_5463_gb300``) and never imports it.

Pieces and the passages they follow (Frommer, Nobile, Zingler, "Deflation and
Flexible SAP-Preconditioning of GMRES in Lattice QCD Simulation"):

* ``dw``, ``dw_local`` -- Eq. "Dw" and Eq. "Dw_local" (Sec. 2), in C
  (``dw_oracle.c``), mass form ``D = (4+m0) - 1/2 H_hop = D_kappa/(2 kappa)``.
* ``sap`` -- Algorithm 2 (SAP iteration) with minimal-residual local solves
  (Sec. 4), in C.
* ``clover`` -- the site-diagonal clover term of the improved operators of
  Sec. 6 (a reading: the paper cites it without a formula), in C; ``dw``,
  ``dw_local`` and ``sap`` add it when given.
* ``flexible_arnoldi`` -- Algorithm 3 (flexible Arnoldi, modified Gram-Schmidt
  as printed).
* ``fgmresdr`` -- Algorithm 4 (F-GMRES-DR) with the harmonic Ritz extraction of
  Lemma 1a, the deflated restart of Eqs. "G_kplus1", "tildeV_Vplus1", "hatHk",
  and the explicit-residual injection and clean restart of Sec. 5.7. ``k = 0``
  gives restarted FGMRES (Sec. 5.2-5.3). ``fgmresdr_steps`` is the same
  iteration as a generator over Arnoldi steps (``fgmresdr`` drives it).
* ``tune_m0_schur``, ``tune_m0_arnoldi``, ``tune_m0`` -- the bare mass that
  puts the leftmost eigenvalue of D at a chosen real part delta, from the
  identity spec(D_m0) = spec(D_0) + m0 and the leftmost Ritz value of D_0
  (thick-restarted Arnoldi ``krylov_schur_edge``, a single Arnoldi process
  ``arnoldi_ritz``, or ARPACK), each with the residual norm of its Ritz pair;
  ``harmonic_ritz_nearest`` -- the eigenvalues nearest the origin by harmonic
  Ritz values (Lemma 1a) with the thick restart of GMRES-DR, used to place and
  verify the smallest |eigenvalue| of each workload's D. Not from the paper,
  which quotes kappa values of thermalised fields: these set up the synthetic
  workloads near the critical mass of Sec. 6.

Small dense steps use numpy.linalg library routines (lstsq, qr, eig, solve).
Readings where the paper is silent are stated next to the code that takes them.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdworacle.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (plain C11 + OpenMP)."""
    src = os.path.join(_HERE, "dw_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_dw.argtypes = [P, ctypes.c_double, P, P, P]
        lib.oracle_dw.restype = None
        lib.oracle_dw_local.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int]
        lib.oracle_dw_local.restype = None
        lib.oracle_sap.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int, ctypes.c_int]
        lib.oracle_sap.restype = ctypes.c_int
        lib.oracle_gamma.argtypes = [ctypes.c_int, P]
        lib.oracle_gamma.restype = None
        lib.oracle_site_colours.argtypes = [P, P, P]
        lib.oracle_site_colours.restype = None
        lib.oracle_mr_history.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_mr_history.restype = ctypes.c_int
        lib.oracle_dw_c.argtypes = [P, ctypes.c_double, P, P, P, P]
        lib.oracle_dw_c.restype = None
        lib.oracle_dw_local_c.argtypes = [P, P, ctypes.c_double, P, P, P, P, ctypes.c_int]
        lib.oracle_dw_local_c.restype = None
        lib.oracle_sap_c.argtypes = [P, P, ctypes.c_double, P, P, P, P, ctypes.c_int, ctypes.c_int]
        lib.oracle_sap_c.restype = ctypes.c_int
        lib.oracle_clover.argtypes = [P, ctypes.c_double, P, P]
        lib.oracle_clover.restype = None
        _lib_handle = lib
    return _lib_handle


def _ivec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _cvec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# Operator and preconditioner (C)
# ----------------------------------------------------------------------------

def gamma(mu: int) -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    _lib().oracle_gamma(int(mu), _ptr(out))
    return out


def clover(U, dims, csw: float) -> np.ndarray:
    """The clover term A[site] (12 x 12 complex, index 3*spin + colour) with
    coefficient csw: c_sw (i/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu} from the
    clover-leaf field strength (the reading stated in dw_oracle.c)."""
    U = _cvec(U)
    V = int(np.prod(dims))
    A = np.empty((V, 12, 12), dtype=np.complex128)
    _lib().oracle_clover(_ptr(_ivec(dims)), float(csw), _ptr(U), _ptr(A))
    return A


def dw(U, psi, dims, m0: float, A=None) -> np.ndarray:
    """D psi on the full periodic lattice (Eq. "Dw"), plus the clover term A psi
    when A is given; psi shape (V,4,3) or flat."""
    U = _cvec(U)
    psi = _cvec(psi)
    out = np.empty_like(psi)
    d = _ivec(dims)
    if A is None:
        _lib().oracle_dw(_ptr(d), float(m0), _ptr(U), _ptr(psi), _ptr(out))
    else:
        A = _cvec(A)
        _lib().oracle_dw_c(_ptr(d), float(m0), _ptr(U), _ptr(A), _ptr(psi), _ptr(out))
    return out


def dw_local(U, psi, dims, block, m0: float, colour: int = -1, A=None) -> np.ndarray:
    """Block-diagonal D^l psi on all domains (colour=-1) or the domains of one colour."""
    U = _cvec(U)
    psi = _cvec(psi)
    out = np.empty_like(psi)
    if A is None:
        _lib().oracle_dw_local(_ptr(_ivec(dims)), _ptr(_ivec(block)), float(m0), _ptr(U), _ptr(psi), _ptr(out),
                               int(colour))
    else:
        A = _cvec(A)
        _lib().oracle_dw_local_c(_ptr(_ivec(dims)), _ptr(_ivec(block)), float(m0), _ptr(U), _ptr(A), _ptr(psi),
                                 _ptr(out), int(colour))
    return out


def sap(U, b, dims, block, m0: float, ncycles: int, nmr: int, x0=None, A=None) -> np.ndarray:
    """``ncycles`` SAP iterations (Algorithm 2) from x0 (default 0); nmr=0: exact local solves."""
    U = _cvec(U)
    b = _cvec(b)
    x = np.zeros_like(b) if x0 is None else _cvec(x0).copy()
    if A is None:
        rc = _lib().oracle_sap(_ptr(_ivec(dims)), _ptr(_ivec(block)), float(m0), _ptr(U), _ptr(b), _ptr(x),
                               int(ncycles), int(nmr))
    else:
        A = _cvec(A)
        rc = _lib().oracle_sap_c(_ptr(_ivec(dims)), _ptr(_ivec(block)), float(m0), _ptr(U), _ptr(A), _ptr(b),
                                 _ptr(x), int(ncycles), int(nmr))
    if rc != 0:
        raise RuntimeError(f"oracle_sap failed ({rc})")
    return x


def site_colours(dims, block) -> np.ndarray:
    V = int(np.prod(dims))
    out = np.zeros(V, dtype=np.int32)
    _lib().oracle_site_colours(_ptr(_ivec(dims)), _ptr(_ivec(block)), _ptr(out))
    return out


def mr_history(U, r, dims, block, m0: float, colour: int, nmr: int):
    """Squared MR residual norm summed over one colour after 0..nmr steps, and y."""
    U = _cvec(U)
    r = _cvec(r)
    y = np.zeros_like(r)
    norms = np.zeros(nmr + 1)
    _lib().oracle_mr_history(_ptr(_ivec(dims)), _ptr(_ivec(block)), float(m0), _ptr(U), _ptr(r), _ptr(y),
                             int(colour), int(nmr), _ptr(norms))
    return norms, y


def dense_operator(apply, n: int) -> np.ndarray:
    """Dense matrix of a linear map on C^n, column by column (small n only)."""
    A = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for c in range(n):
        e[c] = 1.0
        A[:, c] = np.asarray(apply(e)).reshape(-1)
        e[c] = 0.0
    return A


# ----------------------------------------------------------------------------
# Krylov layer (numpy)
# ----------------------------------------------------------------------------

def flexible_arnoldi(A, M, r0, m: int):
    """Algorithm 3: m steps of the flexible Arnoldi process started from r0.

    Returns (V[m+1, n], Z[m, n], Hhat[m+1, m]) with A Z^T = V^T Hhat
    (vectors are stored as rows).
    """
    n = r0.size
    V = np.zeros((m + 1, n), dtype=np.complex128)
    Z = np.zeros((m, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    beta = np.linalg.norm(r0)
    V[0] = r0 / beta
    for j in range(m):
        Z[j] = M(V[j])
        w = A(Z[j]).astype(np.complex128, copy=True)
        for i in range(j + 1):  # modified Gram-Schmidt, as printed
            H[i, j] = np.vdot(V[i], w)
            w -= H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    return V, Z, H


def harmonic_ritz(Hhat: np.ndarray):
    """Lemma 1a: eigenpairs of H_m + f_m h_m^H with H_m^H f_m = h_m.

    ``Hhat`` is (mm+1) x mm = [H_m; h_m^H]. Returns (lambda, G) from numpy eig.
    """
    mm = Hhat.shape[1]
    Hm = Hhat[:mm, :mm]
    hmH = Hhat[mm, :mm]          # the row h_m^H
    f = np.linalg.solve(Hm.conj().T, hmH.conj())
    lam, G = np.linalg.eig(Hm + np.outer(f, hmH))
    return lam, G


def select_smallest(lam: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k harmonic Ritz values of smallest modulus.

    Reading: ties in modulus are broken by the position in the eigenvalue list
    (stable sort).
    """
    return np.argsort(np.abs(lam), kind="stable")[:k]


def deflated_restart(V, Z, H, mm: int, k: int, r):
    """Deflated restart at the top of the repeat loop of Algorithm 4.

    From the previous cycle's basis V (rows 0..mm), Z (rows 0..mm-1),
    Hessenberg-like Hhat = H[:mm+1, :mm] and the explicit residual r:

    * harmonic Ritz pairs of Lemma 1a, the k of smallest modulus -> G_k,
    * G_{k+1} = [[G_k, g], [0, gamma]] with [g; gamma] = V_{m+1}^H r (the
      explicit residual in the old basis, Sec. 5.7), QR with real positive
      diag(R),
    * Hhat_k = Q_{k+1}^H Hhat Q_k (Eq. "hatHk"), V_{k+1} = V_{m+1} Q_{k+1},
      Z_k = Z_m Q_k (Eq. "tildeV_Vplus1"),
    * v_{k+1} := r orthonormalised against V_k (Sec. 5.7),
    * c = [V_{k+1}^H r].

    Returns (V_{k+1} rows, Z_k rows, Hhat_k, c, selected Ritz values).
    """
    Hhat = H[:mm + 1, :mm].copy()
    lam, G = harmonic_ritz(Hhat)
    sel = select_smallest(lam, k)
    Gk1 = np.zeros((mm + 1, k + 1), dtype=np.complex128)
    Gk1[:mm, :k] = G[:, sel]
    Gk1[:, k] = V[:mm + 1].conj() @ r
    Q, R = np.linalg.qr(Gk1)
    d = np.diagonal(R)
    Q = Q * np.where(d == 0, 1.0, d / np.abs(d))[None, :]
    Qk = Q[:mm, :k]
    Hk = Q.conj().T @ Hhat @ Qk
    Vk1 = Q.T @ V[:mm + 1]
    Zk = Qk.T @ Z[:mm]
    w = r.copy()
    for _ in range(2):
        w -= Vk1[:k].T @ (Vk1[:k].conj() @ w)
    Vk1[k] = w / np.linalg.norm(w)
    ck = Vk1.conj() @ r
    return Vk1, Zk, Hk, ck, lam[sel].copy()


class SolveResult:
    def __init__(self):
        self.x = None
        self.converged = False
        self.iterations = 0        # Arnoldi steps = preconditioned matvecs
        self.cycles = 0
        self.clean_restarts = 0
        self.true_rel_res = np.inf
        self.history = []          # per cycle: (iterations, implicit rel res, explicit rel res)
        self.ritz = []             # per deflated restart: selected harmonic Ritz values


def fgmresdr(A, M, b, m: int, k: int, tol: float, max_cycles: int = 1000, t_clean: float = 4.0,
             x0=None, max_iterations: int | None = None, on_cycle=None) -> SolveResult:
    """Algorithm 4 (F-GMRES-DR) with the refinement scheme of Sec. 5.7
    (Algorithm 5), run to the end: see ``fgmresdr_steps`` for the readings."""
    it = fgmresdr_steps(A, M, b, m, k, tol, max_cycles, t_clean, x0, max_iterations, on_cycle)
    while True:
        try:
            next(it)
        except StopIteration as stop:
            return stop.value


def fgmresdr_steps(A, M, b, m: int, k: int, tol: float, max_cycles: int = 1000, t_clean: float = 4.0,
                   x0=None, max_iterations: int | None = None, on_cycle=None):
    """Algorithm 4 (F-GMRES-DR) with the refinement scheme of Sec. 5.7
    (Algorithm 5), as a generator: it yields the running SolveResult after
    every Arnoldi step (so a caller can time a solve in pieces) and returns the
    final SolveResult (``StopIteration.value``).

    Readings taken (the paper leaves these open):

    * ``m`` is the total basis dimension of a cycle; a deflated cycle adds
      m - k new vectors.
    * x0 = 0 unless given; convergence is the explicit FP64 relative residual
      ``||b - A x|| / ||b|| <= tol``, checked at the end of every cycle.
    * a cycle ends early once the least-squares (implicit) residual is
      ``<= tol ||b||``; then the explicit check decides.
    * the explicitly recomputed residual r replaces the updated one in three
      places (Sec. 5.7): the last column of G_{k+1} is V_{m+1}^H r, the
      vector v_{k+1} is r orthonormalised (two classical Gram-Schmidt passes)
      against V_k = V_{m+1} Q_k, and c = [V_{k+1}^H r; 0].
    * the QR factorisation of G_{k+1} is the one with a real positive
      diagonal of R, so the injected v_{k+1} has the phase of V_{m+1} q_{k+1}.
    * clean restart when ||r_explicit|| / ||r_implicit|| > t_clean
      (default 4, inside the paper's range 2..10), or when a cycle ended with
      no more than k vectors.
    * happy breakdown: h_{j+1,j} <= 1e-14 ||A z_j|| ends the cycle.
    """
    b = _cvec(b).reshape(-1)
    n = b.size
    bnorm = np.linalg.norm(b)
    res = SolveResult()
    x = np.zeros(n, dtype=np.complex128) if x0 is None else _cvec(x0).reshape(-1).copy()
    r = b - A(x) if x0 is not None else b.copy()
    if bnorm == 0.0:
        res.x, res.converged, res.true_rel_res = x, True, 0.0
        return res
    if np.linalg.norm(r) <= tol * bnorm:
        res.x, res.converged, res.true_rel_res = x, True, np.linalg.norm(r) / bnorm
        return res

    V = np.zeros((m + 1, n), dtype=np.complex128)
    Z = np.zeros((m, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    c = np.zeros(m + 1, dtype=np.complex128)
    deflate = False
    mm = 0
    while res.cycles < max_cycles:
        if not deflate:
            # first cycle (or clean restart): plain flexible GMRES from r
            beta = np.linalg.norm(r)
            V[:] = 0
            Z[:] = 0
            H[:] = 0
            c[:] = 0
            V[0] = r / beta
            c[0] = beta
            j0 = 0
        else:
            # deflated restart (top of the repeat loop of Algorithm 4)
            Vk1, Zk, Hk, ck, ritz = deflated_restart(V, Z, H, mm, k, r)
            res.ritz.append(ritz)
            V[:] = 0
            Z[:] = 0
            H[:] = 0
            c[:] = 0
            V[:k + 1] = Vk1
            Z[:k] = Zk
            H[:k + 1, :k] = Hk
            c[:k + 1] = ck
            j0 = k
        res.cycles += 1
        # (remaining part of the) flexible Arnoldi process
        mm = m
        for j in range(j0, m):
            Z[j] = M(V[j])
            w = np.asarray(A(Z[j]), dtype=np.complex128).copy()
            wnorm0 = np.linalg.norm(w)
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w -= H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            res.iterations += 1
            breakdown = hn <= 1e-14 * wnorm0
            if not breakdown:
                V[j + 1] = w / hn
            eta, _, _, _ = np.linalg.lstsq(H[:j + 2, :j + 1], c[:j + 2], rcond=None)
            res_impl = np.linalg.norm(c[:j + 2] - H[:j + 2, :j + 1] @ eta)
            yield res
            if breakdown or res_impl <= tol * bnorm or (
                    max_iterations is not None and res.iterations >= max_iterations):
                mm = j + 1
                break
        eta, _, _, _ = np.linalg.lstsq(H[:mm + 1, :mm], c[:mm + 1], rcond=None)
        res_impl = np.linalg.norm(c[:mm + 1] - H[:mm + 1, :mm] @ eta)
        x = x + Z[:mm].T @ eta
        r = b - A(x)
        rnorm = np.linalg.norm(r)
        res.history.append((res.iterations, res_impl / bnorm, rnorm / bnorm))
        if on_cycle is not None:
            on_cycle(res)
        if rnorm <= tol * bnorm:
            res.converged = True
            break
        if max_iterations is not None and res.iterations >= max_iterations:
            break
        clean = k == 0 or mm <= k or (res_impl > 0 and rnorm / res_impl > t_clean) or res_impl == 0
        if k > 0 and clean:
            res.clean_restarts += 1
        deflate = not clean
    res.x = x
    res.true_rel_res = np.linalg.norm(b - A(x)) / bnorm
    return res


# ----------------------------------------------------------------------------
# Lattice-level conveniences
# ----------------------------------------------------------------------------

def lattice_operators(U, dims, block, m0, sap_cycles: int, mr_steps: int, clov=None):
    """(A, M) callables on flat complex vectors: A = D (plus the clover term
    clov when given), M = SAP preconditioner built on the same operator."""
    U = _cvec(U)
    V = int(np.prod(dims))

    def A(v):
        return dw(U, np.asarray(v).reshape(V, 4, 3), dims, m0, A=clov).reshape(-1)

    def M(v):
        return sap(U, np.asarray(v).reshape(V, 4, 3), dims, block, m0, sap_cycles, mr_steps, A=clov).reshape(-1)

    return A, M


def solve(U, b, dims, block, m0, sap_cycles, mr_steps, m, k, tol, clov=None, **kw) -> SolveResult:
    A, M = lattice_operators(U, dims, block, m0, sap_cycles, mr_steps, clov=clov)
    return fgmresdr(A, M, np.asarray(b).reshape(-1), m, k, tol, **kw)


def arnoldi_ritz(apply, n: int, m: int, seed: int = 0, return_vectors: bool = False):
    """Ritz values of an m-step Arnoldi process (classical Gram-Schmidt with one
    reorthogonalisation) started from a seeded random vector, with their
    residual norms |h_{m+1,m} e_m^T y| (y the unit eigenvector of H_m), which
    equal ||A x - theta x|| for the unit Ritz vector x = V_m y. Exterior
    eigenvalues converge first. With return_vectors the Ritz vectors are
    returned too, as the columns of an n x m array."""
    rng = np.random.default_rng(seed)
    V = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    V[0] = v / np.linalg.norm(v)
    for j in range(m):
        w = np.asarray(apply(V[j]), dtype=np.complex128)
        for _ in range(2):
            h = (V[:j + 1] @ w.conj()).conj()  # V^H w without copying V
            w = w - V[:j + 1].T @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    theta, Y = np.linalg.eig(H[:m, :m])
    bounds = np.abs(H[m, m - 1] * Y[m - 1, :])
    if return_vectors:
        return theta, bounds, V[:m].T @ Y
    return theta, bounds


def krylov_schur_edge(apply, n: int, m: int = 60, k: int = 20, max_restarts: int = 40, tol: float = 1e-3,
                      seed: int = 0, return_vector: bool = False, log=None):
    """Leftmost eigenvalue estimate by thick-restarted Arnoldi (Krylov-Schur,
    Stewart 2002) in bounded memory.

    Each restart expands the basis to m vectors, takes the Ritz pairs of the
    m x m block H_m and the residual norm of each, |h_{m+1,m} e_m^T y| with y
    the unit eigenvector of H_m (it equals ||A x - theta x|| for the unit Ritz
    vector x = V_m y), stops once the leftmost Ritz value's residual is below
    tol, and otherwise keeps the k Schur vectors of H_m whose Ritz values have
    the smallest real parts (a Schur form ordered so that they lead). Returns
    (theta, residual norm, matvecs), plus the unit Ritz vector with
    return_vector. log, when given, is called with (restart, matvecs, theta,
    residual) after every restart."""
    import scipy.linalg as sla

    rng = np.random.default_rng(seed)
    V = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    V[0] = v / np.linalg.norm(v)
    p = 0
    matvecs = 0
    theta = bound = y = None
    for restart in range(max_restarts):
        for j in range(p, m):
            w = np.asarray(apply(V[j]), dtype=np.complex128)
            matvecs += 1
            for _pass in range(2):
                h = (V[:j + 1] @ w.conj()).conj()
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            V[j + 1] = w / H[j + 1, j]
        # Ritz pairs of H_m and their residual norms (from the eigenvectors)
        lam, Y = np.linalg.eig(H[:m, :m])
        res = np.abs(H[m, m - 1]) * np.abs(Y[m - 1, :]) / np.linalg.norm(Y, axis=0)
        i = int(np.argmin(lam.real))
        theta, bound, y = lam[i], float(res[i]), Y[:, i] / np.linalg.norm(Y[:, i])
        if log is not None:
            log(restart, matvecs, theta, bound)
        if bound < tol or restart == max_restarts - 1:
            break
        # thick restart on the Schur vectors of the k leftmost Ritz values
        cut = np.sort(lam.real)[k - 1]
        T, Z, sdim = sla.schur(H[:m, :m], output="complex", sort=lambda x: x.real <= cut)
        kk = max(1, min(sdim, m - 1))
        Vk = Z[:, :kk].T @ V[:m]
        hrow = H[m, m - 1] * Z[m - 1, :kk]
        vlast = V[m].copy()
        V[:] = 0
        H[:] = 0
        V[:kk] = Vk
        V[kk] = vlast
        H[:kk, :kk] = T[:kk, :kk]
        H[kk, :kk] = hrow
        p = kk
    if return_vector:
        return theta, bound, matvecs, V[:m].T @ y
    return theta, bound, matvecs


def harmonic_ritz_nearest(apply, n: int, m: int = 60, k: int = 20, max_restarts: int = 100, tol: float = 1e-6,
                          nev: int = 4, seed: int = 0, log=None, return_vectors: bool = False,
                          near_factor: float | None = None, stop=None):
    """Eigenvalues of A nearest the origin by harmonic Ritz extraction with
    thick restarts (the deflated restart of GMRES-DR without the linear system).

    Each restart expands A V_m = V_{m+1} Hhat_m to m vectors and takes the
    harmonic Ritz pairs of Lemma 1a: (H_m + f h_m^H) g = theta g with
    H_m^H f = h_m, Hhat_m = [H_m; h_m^H]. The residual of a pair,
    A u - theta u with u = V_m g, equals V_{m+1} (h_m^H g) [-f; 1], so all
    residuals share the direction [-f; 1] and each has the norm
    |h_m^H g| ||[-f; 1]|| / ||g||. The restart keeps the k pairs of smallest
    |theta|: with G_{k+1} = [[G_k], [0]] | [-f; 1] orthonormalised (QR) to
    Q_{k+1}, V_{k+1} = V_{m+1} Q_{k+1} and Hhat_k = Q_{k+1}^H Hhat_m Q_k
    satisfy A V_k = V_{k+1} Hhat_k (Eqs. "G_kplus1", "tildeV_Vplus1",
    "hatHk" with the eigenvector residual in place of the linear system's).
    Stops once the nev pairs of smallest |theta| all have residual norms
    below tol (with near_factor: once those of them with |theta| <= near_factor
    times the smallest |theta| do), or when stop() returns True after a
    restart. Returns (theta[nev], residual norms[nev], matvecs), plus the
    unit vectors u (columns of an n x nev array) with return_vectors."""
    rng = np.random.default_rng(seed)
    V = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    V[0] = v / np.linalg.norm(v)
    p = 0
    matvecs = 0
    theta = res = None
    for restart in range(max_restarts):
        for j in range(p, m):
            w = np.asarray(apply(V[j]), dtype=np.complex128)
            matvecs += 1
            for _pass in range(2):
                h = (V[:j + 1] @ w.conj()).conj()
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            V[j + 1] = w / H[j + 1, j]
        Hm = H[:m, :m]
        hrow = H[m, :m]
        f = np.linalg.solve(Hm.conj().T, hrow.conj())
        lam, G = np.linalg.eig(Hm + np.outer(f, hrow))
        order = np.argsort(np.abs(lam), kind="stable")
        fn = np.sqrt(1.0 + np.linalg.norm(f) ** 2)
        allres = np.abs(hrow @ G) * fn / np.linalg.norm(G, axis=0)
        theta, res = lam[order[:nev]], allres[order[:nev]]
        if log is not None:
            log(restart, matvecs, theta, res)
        watch = res if near_factor is None else res[np.abs(theta) <= near_factor * np.abs(theta[0])]
        if watch.max() < tol or restart == max_restarts - 1 or (stop is not None and stop()):
            if return_vectors:
                Gs = G[:, order[:nev]]
                U = V[:m].T @ (Gs / np.linalg.norm(Gs, axis=0))
                return theta, res, matvecs, U
            break
        Gk1 = np.zeros((m + 1, k + 1), dtype=np.complex128)
        Gk1[:m, :k] = G[:, order[:k]]
        Gk1[:m, k] = -f
        Gk1[m, k] = 1.0
        Q, _ = np.linalg.qr(Gk1)
        Hk = Q.conj().T @ H[:m + 1, :m] @ Q[:m, :k]
        Vk1 = Q.T @ V[:m + 1]
        V[:] = 0
        H[:] = 0
        V[:k + 1] = Vk1
        H[:k + 1, :k] = Hk
        p = k
    return theta, res, matvecs


def tune_m0_schur(U, dims, target: float, m: int = 60, k: int = 20, tol: float = 1e-3, seed: int = 0, clov=None,
                  max_restarts: int = 40, log=None):
    """As tune_m0_arnoldi with a thick-restarted Arnoldi (bounded memory).
    Returns (m0, theta*, its residual norm, matvecs, seconds)."""
    V = int(np.prod(dims))
    U = _cvec(U)
    t0 = time.time()
    theta, bound, mv = krylov_schur_edge(
        lambda v: dw(U, np.asarray(v).reshape(V, 4, 3), dims, 0.0, A=clov).reshape(-1), 12 * V, m, k,
        max_restarts=max_restarts, tol=tol, seed=seed, log=log)
    return target - theta.real, theta, bound, mv, time.time() - t0


def tune_m0_arnoldi(U, dims, target: float, m: int = 200, seed: int = 0, clov=None):
    """Bare mass from the leftmost Ritz value of D at m0 = 0 (with the clover
    term clov when given: it does not depend on m0).

    spec(D_m0) = spec(D_0) + m0, so m0 = target - Re(theta*) with theta* the
    Ritz value of smallest real part of an m-step Arnoldi process on D_0.
    Returns (m0, theta*, its residual bound, seconds)."""
    V = int(np.prod(dims))
    U = _cvec(U)
    t0 = time.time()
    theta, bounds = arnoldi_ritz(
        lambda v: dw(U, np.asarray(v).reshape(V, 4, 3), dims, 0.0, A=clov).reshape(-1), 12 * V, m, seed)
    i = int(np.argmin(theta.real))
    return target - theta[i].real, theta[i], bounds[i], time.time() - t0


def tune_m0(U, dims, target: float, nev: int = 6, ncv: int = 48, tol: float = 1e-6):
    """Bare mass with smallest |eigenvalue| of D_m0 near ``target``.

    spec(D_m0) = spec(D_0) + m0 exactly (D_m0 - D_0 = m0 I), so with mu* the
    eigenvalue of D_0 of smallest real part (found by restarted Arnoldi,
    ARPACK ``which='SR'``), m0 = target - Re(mu*). Returns (m0, mu_list).
    """
    from scipy.sparse.linalg import LinearOperator, eigs

    V = int(np.prod(dims))
    n = 12 * V
    U = _cvec(U)

    def mv(v):
        return dw(U, np.asarray(v, dtype=np.complex128).reshape(V, 4, 3), dims, 0.0).reshape(-1)

    op = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    t0 = time.time()
    vals = eigs(op, k=nev, which="SR", ncv=ncv, tol=tol, return_eigenvectors=False,
                v0=np.ones(n, dtype=np.complex128))
    vals = np.sort_complex(vals)
    mu = vals[np.argmin(vals.real)]
    return target - mu.real, vals, time.time() - t0
