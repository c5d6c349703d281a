"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: closed forms
(free-field plane waves), symmetries (gamma5-hermiticity, gauge covariance),
dense linear algebra on tiny lattices (numpy LU / eig), the series form of the
SAP preconditioner (Sec. 4) and the invariants of the Krylov layer (Eqs.
"arnoldilike", "harmRitz", "hatHk", "r").
"""

import itertools

import numpy as np
import pytest

import fieldgen as fg
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

G5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None]


def coords(dims):
    V = fg.volume(dims)
    return np.stack(np.unravel_index(np.arange(V), dims, order="F"), 1)


def shift_index(dims, mu, sign):
    c = coords(dims)
    c[:, mu] = (c[:, mu] + sign) % dims[mu]
    return np.ravel_multi_index(c.T, dims, order="F")


# --------------------------------------------------------------------------- gamma basis
def test_gamma_defining_relations():
    g = [oracle.gamma(mu) for mu in range(4)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)  # Hermitian
        for b in range(4):
            anti = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(anti, 2.0 * np.eye(4) * (a == b))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


# --------------------------------------------------------------------------- free field
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 8)])
@pytest.mark.parametrize("m0", [-0.5, 0.3])
def test_free_field_plane_waves(dims, m0):
    """U = 1: plane wave e^{ip.n} u with (sum_j gamma_j sin p_j) u = s u is an
    eigenvector of D with eigenvalue (4+m0) - sum_j cos p_j - i s."""
    U = fg.unit_gauge(dims)
    c = coords(dims)
    g = [oracle.gamma(mu) for mu in range(4)]
    rng = np.random.default_rng(7)
    for _ in range(6):
        kvec = [rng.integers(0, d) for d in dims]
        p = np.array([2 * np.pi * kvec[j] / dims[j] for j in range(4)])
        S = sum(g[j] * np.sin(p[j]) for j in range(4))
        s_vals, s_vecs = np.linalg.eigh(S)
        phase = np.exp(1j * (c @ p))
        for a in range(4):
            u = s_vecs[:, a]
            colour = rng.standard_normal(3) + 1j * rng.standard_normal(3)
            psi = phase[:, None, None] * u[None, :, None] * colour[None, None, :]
            lam = (4 + m0) - np.cos(p).sum() - 1j * s_vals[a]
            out = oracle.dw(U, psi, dims, m0)
            assert np.abs(out - lam * psi).max() < 1e-12 * max(1.0, np.abs(psi).max())


def test_free_field_spectrum_closed_form():
    """Dense free-field D on a 2x2x2x4 lattice: its spectrum is the closed form
    with multiplicity 6 (12 when all sin p_j = 0)."""
    dims = (2, 2, 2, 4)
    m0 = -0.2
    U = fg.unit_gauge(dims)
    V = fg.volume(dims)
    A = oracle.dense_operator(lambda v: oracle.dw(U, v.reshape(V, 4, 3), dims, m0).reshape(-1), 12 * V)
    def canon(z):  # sort by rounded (re, im) so round-off cannot reorder equal values
        z = np.asarray(z)
        order = np.lexsort((np.round(z.imag, 8), np.round(z.real, 8)))
        return z[order]

    ev = canon(np.linalg.eigvals(A))
    expect = []
    for kvec in itertools.product(*[range(d) for d in dims]):
        p = np.array([2 * np.pi * kvec[j] / dims[j] for j in range(4)])
        s = np.sqrt((np.sin(p) ** 2).sum())
        base = (4 + m0) - np.cos(p).sum()
        expect += [base + 1j * s] * 6 + [base - 1j * s] * 6
    expect = canon(np.array(expect))
    assert np.abs(ev - expect).max() < 1e-10


# --------------------------------------------------------------------------- symmetries
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (4, 2, 6, 2)])
def test_gamma5_hermiticity(dims):
    U = fg.gauge_field(dims, 0.5, seed=3)
    psi = fg.gaussian_source(dims, 4)
    phi = fg.gaussian_source(dims, 5)
    m0 = -0.4
    lhs = np.vdot(phi, G5 * oracle.dw(U, G5 * psi, dims, m0))
    rhs = np.vdot(oracle.dw(U, phi, dims, m0), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_gauge_covariance(dims):
    V = fg.volume(dims)
    U = fg.gauge_field(dims, 0.6, seed=11)
    psi = fg.gaussian_source(dims, 12)
    g = fg.random_su3(V, 13)
    Ug = np.empty_like(U)
    for mu in range(4):
        t = shift_index(dims, mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ g[t].conj().transpose(0, 2, 1)
    m0 = 0.1
    lhs = oracle.dw(Ug, np.einsum("sab,sxb->sxa", g, psi), dims, m0)
    rhs = np.einsum("sab,sxb->sxa", g, oracle.dw(U, psi, dims, m0))
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_mass_shift():
    dims = (4, 2, 4, 4)
    U = fg.gauge_field(dims, 0.4, seed=2)
    psi = fg.gaussian_source(dims, 3)
    d = oracle.dw(U, psi, dims, 0.37) - oracle.dw(U, psi, dims, 0.0)
    assert np.abs(d - 0.37 * psi).max() < 1e-13


def test_two_site_direction_sums_both_hops():
    """d_j = 2: n + j and n - j are the same site, so both hop terms land on it
    and D is the free-field closed form at p_j in {0, pi}."""
    dims = (2, 4, 4, 4)
    U = fg.unit_gauge(dims)
    c = coords(dims)
    p = np.array([np.pi, 0.0, np.pi / 2, 0.0])
    psi = np.exp(1j * (c @ p))[:, None, None] * np.ones((1, 4, 3))
    out = oracle.dw(U, psi, dims, 0.0)
    g = [oracle.gamma(mu) for mu in range(4)]
    S = sum(g[j] * np.sin(p[j]) for j in range(4))
    expect = (4 - np.cos(p).sum()) * psi - 1j * np.einsum("ab,sbc->sac", S, psi)
    assert np.abs(out - expect).max() < 1e-12


# --------------------------------------------------------------------------- domains
def _dense(U, dims, m0):
    V = fg.volume(dims)
    return oracle.dense_operator(lambda v: oracle.dw(U, v.reshape(V, 4, 3), dims, m0).reshape(-1), 12 * V)


def _domain_index(dims, block):
    c = coords(dims)
    nb = [dims[j] // block[j] for j in range(4)]
    dc = c // np.array(block)[None, :]
    dom = dc[:, 0] + nb[0] * (dc[:, 1] + nb[1] * (dc[:, 2] + nb[2] * dc[:, 3]))
    return dom, dc.sum(1) % 2


SMALL_DIMS, SMALL_BLOCK = (4, 4, 2, 2), (2, 2, 1, 1)  # 64 sites, 16 domains of 4 sites


def test_local_operator_is_principal_submatrix():
    dims, block, m0 = SMALL_DIMS, SMALL_BLOCK, -0.5
    U = fg.gauge_field(dims, 0.3, seed=0)
    V = fg.volume(dims)
    A = _dense(U, dims, m0)
    Al = oracle.dense_operator(lambda v: oracle.dw_local(U, v.reshape(V, 4, 3), dims, block, m0).reshape(-1), 12 * V)
    dom, col = _domain_index(dims, block)
    sd = np.repeat(dom, 12)
    same = sd[:, None] == sd[None, :]
    assert np.abs(Al - np.where(same, A, 0)).max() < 1e-14
    # the colouring: no coupling between distinct domains of the same colour (Sec. 2)
    sc = np.repeat(col, 12)
    cross_same_colour = (sc[:, None] == sc[None, :]) & ~same
    assert np.abs(A[cross_same_colour]).max() == 0.0
    assert np.array_equal(oracle.site_colours(dims, block), col)
    assert col[0] == 0


@pytest.mark.parametrize("s", [1, 2, 3])
def test_sap_exact_local_solves_equal_series(s):
    """SAP with exact domain solves, s cycles from 0, equals
    M = sum_{j<s} (A_L^{-1} A_U)^j A_L^{-1} of the red-black block splitting
    (Sec. 4; colour 0 is the leading block, swept first)."""
    dims, block, m0 = (4, 4, 4, 2), (2, 2, 2, 1), -0.5
    U = fg.gauge_field(dims, 0.3, seed=0)
    V = fg.volume(dims)
    A = _dense(U, dims, m0)
    _, col = _domain_index(dims, block)
    sc = np.repeat(col, 12)
    perm = np.concatenate([np.where(sc == 0)[0], np.where(sc == 1)[0]])
    Ap = A[np.ix_(perm, perm)]
    h = (sc == 0).sum()
    AL = Ap.copy()
    AL[:h, h:] = 0
    AU = -(Ap - AL)
    ALi = np.linalg.inv(AL)
    T = ALi @ AU
    M = np.zeros_like(Ap)
    P = np.eye(Ap.shape[0])
    for _ in range(s):
        M += P @ ALi
        P = T @ P
    v = fg.gaussian_source(dims, 21).reshape(-1)
    z_series = np.empty_like(v)
    z_series[perm] = M @ v[perm]
    z = oracle.sap(U, v.reshape(V, 4, 3), dims, block, m0, s, 0).reshape(-1)
    assert np.linalg.norm(z - z_series) <= 1e-11 * np.linalg.norm(z_series)


def test_mr_monotone_and_converges_to_exact_local_solve():
    dims, block, m0 = (4, 4, 4, 2), (2, 2, 2, 1), 2.0
    U = fg.gauge_field(dims, 0.3, seed=0)
    r = fg.gaussian_source(dims, 9)
    norms, y = oracle.mr_history(U, r, dims, block, m0, 0, 60)
    assert np.all(np.diff(norms) <= 1e-12 * norms[0])
    V = fg.volume(dims)
    col = oracle.site_colours(dims, block)
    r0 = r * (col == 0)[:, None, None]
    # exact block solve on colour 0 via the dense local operator
    Al = oracle.dense_operator(lambda v: oracle.dw_local(U, v.reshape(V, 4, 3), dims, block, m0, 0).reshape(-1),
                               12 * V)
    mask = np.repeat(col == 0, 12)
    y_exact = np.zeros(12 * V, dtype=np.complex128)
    y_exact[mask] = np.linalg.solve(Al[np.ix_(mask, mask)], r0.reshape(-1)[mask])
    assert np.linalg.norm(y.reshape(-1) - y_exact) <= 1e-8 * np.linalg.norm(y_exact)


def test_sap_one_cycle_is_red_then_black_block_gauss_seidel():
    """One SAP cycle with MR solves, written out with the local operator."""
    dims, block, m0, nmr = (4, 4, 4, 4), (2, 2, 2, 2), -0.3, 3
    U = fg.gauge_field(dims, 0.4, seed=1)
    v = fg.gaussian_source(dims, 2)
    col = oracle.site_colours(dims, block)
    x = np.zeros_like(v)
    for c in (0, 1):
        r = v - oracle.dw(U, x, dims, m0)
        r_c = r * (col == c)[:, None, None]
        _, y = oracle.mr_history(U, r_c, dims, block, m0, c, nmr)
        x = x + y * (col == c)[:, None, None]
    z = oracle.sap(U, v, dims, block, m0, 1, nmr)
    assert np.abs(z - x).max() < 1e-13 * np.abs(x).max()


# --------------------------------------------------------------------------- Krylov layer
def _tiny_system(seed=0):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = fg.gauge_field(dims, 0.3, seed=seed)
    return dims, block, U


def test_flexible_arnoldi_relation_and_orthonormality():
    dims, block, U = _tiny_system()
    A, M = oracle.lattice_operators(U, dims, block, -0.5, 2, 2)
    b = fg.gaussian_source(dims, 1).reshape(-1)
    m = 12
    V, Z, H = oracle.flexible_arnoldi(A, M, b, m)
    AZ = np.stack([A(Z[j]) for j in range(m)])
    assert np.linalg.norm(AZ - H.T @ V) <= 1e-12 * np.linalg.norm(AZ)
    assert np.abs(V.conj() @ V.T - np.eye(m + 1)).max() < 1e-12
    assert np.abs(np.tril(H, -2)).max() == 0.0


def test_full_gmres_reaches_dense_solution():
    """M = I, k = 0, m = n on a 2^4 lattice (n = 192): GMRES is exact."""
    dims = (2, 2, 2, 2)
    U = fg.gauge_field(dims, 0.5, seed=4)
    V = fg.volume(dims)
    m0 = -0.3
    A = _dense(U, dims, m0)
    b = fg.gaussian_source(dims, 5).reshape(-1)
    x_star = np.linalg.solve(A, b)
    Aop = lambda v: A @ v
    res = oracle.fgmresdr(Aop, lambda v: v.copy(), b, 12 * V, 0, 1e-12)
    assert res.converged and res.cycles == 1
    assert np.linalg.norm(res.x - x_star) <= 1e-9 * np.linalg.norm(x_star)


def test_exact_preconditioner_converges_in_one_step():
    dims = (2, 2, 2, 2)
    U = fg.gauge_field(dims, 0.5, seed=4)
    A = _dense(U, dims, -0.3)
    Ainv = np.linalg.inv(A)
    b = fg.gaussian_source(dims, 6).reshape(-1)
    res = oracle.fgmresdr(lambda v: A @ v, lambda v: Ainv @ v, b, 10, 3, 1e-11)
    assert res.converged and res.iterations == 1


def test_harmonic_ritz_lemma_1a():
    """(A V_m)^H (A u - lambda u) = 0 for every harmonic Ritz pair (Eq. "harmRitz")."""
    dims, block, U = _tiny_system()
    A, _ = oracle.lattice_operators(U, dims, block, -0.5, 1, 1)
    b = fg.gaussian_source(dims, 1).reshape(-1)
    m = 15
    V, Z, H = oracle.flexible_arnoldi(A, lambda v: v.copy(), b, m)
    lam, G = oracle.harmonic_ritz(H)
    AV = np.stack([A(V[j]) for j in range(m)])
    for i in range(m):
        u = G[:, i] @ V[:m]
        resid = A(u) - lam[i] * u
        assert np.abs(AV.conj() @ resid).max() <= 1e-10 * np.linalg.norm(resid) * np.linalg.norm(AV)


def test_harmonic_ritz_values_approach_smallest_eigenvalues():
    """M = I: after several deflated cycles the k harmonic Ritz values of
    smallest modulus match the k eigenvalues of D nearest the origin."""
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 1.0, seed=2)
    A0 = _dense(U, dims, 0.0)
    ev0 = np.linalg.eigvals(A0)
    m0 = 0.05 - ev0.real.min()
    A = A0 + m0 * np.eye(A0.shape[0])
    ev = ev0 + m0
    near = ev[np.argsort(np.abs(ev))]
    b = fg.gaussian_source(dims, 1).reshape(-1)
    k = 3
    res = oracle.fgmresdr(lambda v: A @ v, lambda v: v.copy(), b, 30, k, 1e-12, max_cycles=60)
    assert res.converged and len(res.ritz) > 5
    ritz = np.sort(np.abs(res.ritz[-1]))
    assert np.allclose(ritz, np.sort(np.abs(near[:k])), rtol=1e-3)


def test_deflated_restart_relation_hatHk():
    """After the restart, A Z_k = V_{k+1} Hhat_k (Eqs. "hatHk", "tilde_Arnoldi")
    and c = V_{k+1}^H r with r in span V_{k+1}."""
    dims, block, U = _tiny_system()
    A, M = oracle.lattice_operators(U, dims, block, -0.5, 2, 2)
    b = fg.gaussian_source(dims, 1).reshape(-1)
    m, k = 14, 4
    V, Z, H = oracle.flexible_arnoldi(A, M, b, m)
    c = np.zeros(m + 1, dtype=np.complex128)
    c[0] = np.linalg.norm(b)
    eta = np.linalg.lstsq(H, c, rcond=None)[0]
    x = Z.T @ eta
    r = b - A(x)
    # the updated residual (Eq. "r") equals the explicit one
    assert np.linalg.norm(V.T @ (c - H @ eta) - r) <= 1e-11 * np.linalg.norm(r)
    Vk1, Zk, Hk, ck, _ = oracle.deflated_restart(V, Z, H, m, k, r)
    AZk = np.stack([A(Zk[i]) for i in range(k)])
    assert np.linalg.norm(AZk - Hk.T @ Vk1) <= 1e-10 * np.linalg.norm(AZk)
    assert np.abs(Vk1.conj() @ Vk1.T - np.eye(k + 1)).max() < 1e-12
    assert np.linalg.norm(Vk1.T @ ck - r) <= 1e-10 * np.linalg.norm(r)


def test_residuals_monotone_and_consistent():
    dims, block, U = _tiny_system()
    b = fg.gaussian_source(dims, 1)
    res = oracle.solve(U, b, dims, block, -0.5, 4, 4, 20, 5, 1e-12)
    assert res.converged
    expl = [h[2] for h in res.history]
    assert all(b_ <= a_ * (1 + 1e-9) for a_, b_ in zip(expl, expl[1:]))
    for _, impl, ex in res.history:
        assert abs(impl - ex) <= 1e-6 * ex + 1e-14
    assert res.true_rel_res <= 1e-12


def test_deflation_reduces_iterations_near_critical():
    """Sec. 6: at fixed m, deflation needs fewer matrix-vector products, most
    visibly near the critical mass."""
    dims, block = (4, 4, 2, 2), (2, 2, 1, 1)
    U = fg.gauge_field(dims, 0.5, seed=0)
    ev = np.linalg.eigvals(_dense(U, dims, 0.0))
    m0 = 0.01 - ev.real.min()
    b = fg.gaussian_source(dims, 1)
    plain = oracle.solve(U, b, dims, block, m0, 1, 2, 8, 0, 1e-10, max_cycles=400)
    defl = oracle.solve(U, b, dims, block, m0, 1, 2, 8, 3, 1e-10, max_cycles=400)
    assert defl.converged
    assert defl.iterations < plain.iterations


def test_tune_m0_places_smallest_eigenvalue():
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 0.5, seed=0)
    m0, vals, _ = oracle.tune_m0(U, dims, 1e-2, nev=4, ncv=40, tol=1e-10)
    ev = np.linalg.eigvals(_dense(U, dims, m0))
    # the leftmost eigenvalue of D_0 sits at Re = target after the shift
    assert abs(ev.real.min() - 1e-2) < 1e-6


def _leftmost(ev, theta):
    """The eigenvalue of smallest real part nearest theta (the leftmost
    eigenvalues of a gamma5-hermitian D come in conjugate pairs)."""
    edge = ev[np.abs(ev.real - ev.real.min()) < 1e-9]
    return edge[np.argmin(np.abs(edge - theta))]


def test_arnoldi_ritz_full_space_reproduces_dense_spectrum():
    """With as many steps as the dimension, the Arnoldi Ritz values are the
    eigenvalues of D (dense numpy eig)."""
    dims = (2, 2, 2, 2)
    U = fg.gauge_field(dims, 0.5, seed=3)
    A = _dense(U, dims, 0.0)
    n = A.shape[0]
    theta, _ = oracle.arnoldi_ritz(lambda v: A @ v, n, n, seed=1)
    ev = np.linalg.eigvals(A)
    # every eigenvalue is matched by a Ritz value and vice versa
    assert max(np.abs(ev - t).min() for t in theta) < 1e-8
    assert max(np.abs(theta - e).min() for e in ev) < 1e-8


def test_arnoldi_ritz_residual_norms_are_true_residuals():
    """The reported residual of every Ritz pair equals ||D x - theta x|| of the
    returned unit Ritz vector, and bounds the distance of theta to the spectrum
    of D in the sense sigma_min(D - theta) <= residual (theta is an exact
    eigenvalue of a perturbation of D of that norm)."""
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 0.5, seed=0)
    A = _dense(U, dims, 0.0)
    n = A.shape[0]
    theta, bounds, X = oracle.arnoldi_ritz(lambda v: A @ v, n, 60, seed=2, return_vectors=True)
    for i in np.argsort(theta.real)[:6]:
        x = X[:, i]
        assert abs(np.linalg.norm(x) - 1.0) < 1e-10
        true = np.linalg.norm(A @ x - theta[i] * x)
        assert abs(true - bounds[i]) <= 1e-9 + 1e-7 * true
        smin = np.linalg.svd(A - theta[i] * np.eye(n), compute_uv=False)[-1]
        assert smin <= bounds[i] * (1 + 1e-8) + 1e-12


def test_krylov_schur_edge_converges_to_leftmost_eigenvalue():
    """Thick-restarted Arnoldi on a 768-dimensional D (several restarts) finds
    the eigenvalue of smallest real part of the dense spectrum, with a residual
    norm below the tolerance that is the true residual of its Ritz vector."""
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 0.5, seed=0)
    A = _dense(U, dims, 0.0)
    n = A.shape[0]
    seen = []
    theta, bound, mv, x = oracle.krylov_schur_edge(lambda v: A @ v, n, m=40, k=12, max_restarts=400, tol=1e-9,
                                                  seed=4, return_vector=True, log=lambda *a: seen.append(a))
    assert mv > 40 and len(seen) > 1              # it did restart
    ev = np.linalg.eigvals(A)
    assert abs(theta.real - ev.real.min()) < 1e-7
    assert abs(theta - _leftmost(ev, theta)) < 1e-7
    assert bound < 1e-9
    assert abs(np.linalg.norm(A @ x - theta * x) - bound) < 1e-10


def test_krylov_schur_reported_residual_is_the_ritz_vectors_at_every_restart():
    """Stopped early (loose tolerance), the returned residual is still the true
    residual of the returned Ritz pair, not that of a Schur vector."""
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 0.6, seed=1)
    A = _dense(U, dims, 0.0)
    n = A.shape[0]
    for restarts in (1, 2, 5):
        theta, bound, mv, x = oracle.krylov_schur_edge(lambda v: A @ v, n, m=30, k=10, max_restarts=restarts,
                                                      tol=0.0, seed=5, return_vector=True)
        true = np.linalg.norm(A @ x - theta * x)
        assert abs(true - bound) <= 1e-10 + 1e-7 * true
        smin = np.linalg.svd(A - theta * np.eye(n), compute_uv=False)[-1]
        assert smin <= bound * (1 + 1e-8) + 1e-12


@pytest.mark.parametrize("how", ["schur", "arnoldi"])
def test_tuned_mass_puts_dense_spectrum_edge_at_target(how):
    """m0 = target - Re(theta*) shifts the leftmost eigenvalue of D_{m0}
    (dense eig) to real part target: a sign error in the shift, or an edge
    taken from the wrong Ritz value, moves it by at least the spread of the
    low spectrum."""
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 0.5, seed=0)
    target = 1e-2
    if how == "schur":
        m0, theta, bound, _, _ = oracle.tune_m0_schur(U, dims, target, m=40, k=12, tol=1e-9, max_restarts=400, seed=4)
    else:
        m0, theta, bound, _ = oracle.tune_m0_arnoldi(U, dims, target, m=12 * fg.volume(dims), seed=4)
    ev = np.linalg.eigvals(_dense(U, dims, m0))
    assert bound < 1e-8
    assert abs(ev.real.min() - target) < 1e-7
    assert abs(_leftmost(ev, target + 1j * theta.imag) - (target + 1j * theta.imag)) < 1e-7
    # every eigenvalue has real part >= target, so min |lambda| >= target (on
    # this small lattice an eigenvalue right of the edge but nearer the real
    # axis is the smallest in modulus)
    assert np.abs(ev).min() >= target - 1e-9


def test_harmonic_ritz_nearest_finds_the_eigenvalues_nearest_the_origin():
    """Thick-restarted harmonic Ritz extraction (Lemma 1a with the
    eigenvector residual as the extra restart vector) on D_{m0} just above the
    critical mass: the values are the dense spectrum's eigenvalues of smallest
    modulus, and each reported residual is ||D u - theta u|| of its vector."""
    dims = (2, 2, 4, 4)
    U = fg.gauge_field(dims, 0.5, seed=0)
    ev0 = np.linalg.eigvals(_dense(U, dims, 0.0))
    m0 = 0.02 - ev0.real.min()
    A = _dense(U, dims, m0)
    n = A.shape[0]
    theta, res, mv, X = oracle.harmonic_ritz_nearest(lambda v: A @ v, n, m=40, k=12, max_restarts=300, tol=1e-9,
                                                     nev=4, seed=6, return_vectors=True)
    assert mv > 40  # restarted
    ev = np.linalg.eigvals(A)
    near = ev[np.argsort(np.abs(ev))[:4]]
    for t in theta:
        assert np.abs(near - t).min() < 1e-7
    assert abs(np.abs(theta).min() - np.abs(ev).min()) < 1e-8
    for i in range(4):
        assert res[i] < 1e-9
        assert abs(np.linalg.norm(A @ X[:, i] - theta[i] * X[:, i]) - res[i]) < 1e-10
    # stopping on the values near the smallest only: those are converged and
    # are the dense eigenvalues; the rest carry their (true) residuals
    theta, res, _, X = oracle.harmonic_ritz_nearest(lambda v: A @ v, n, m=40, k=12, max_restarts=300, tol=1e-9,
                                                    nev=8, seed=6, return_vectors=True, near_factor=1.5)
    near = np.abs(theta) <= 1.5 * np.abs(theta[0])
    assert near.sum() >= 1 and res[near].max() < 1e-9
    for t in theta[near]:
        assert np.abs(ev - t).min() < 1e-7
    for i in range(8):
        assert abs(np.linalg.norm(A @ X[:, i] - theta[i] * X[:, i]) - res[i]) < 1e-10 + 1e-7 * res[i]


# --------------------------------------------------------------------------- clover term
def _abelian_field(dims, b):
    """U_{n,0} = diag(e^{i b n_1}, e^{-i b n_1}, 1), all other links 1: a uniform
    field strength in the (0, 1) plane when b d_1 is a multiple of 2 pi."""
    V = fg.volume(dims)
    U = fg.unit_gauge(dims).copy()
    y = coords(dims)[:, 1]
    U[:, 0, 0, 0] = np.exp(1j * b * y)
    U[:, 0, 1, 1] = np.exp(-1j * b * y)
    assert U.shape == (V, 4, 3, 3)
    return U


def test_clover_free_field_vanishes():
    dims = (4, 2, 4, 2)
    A = oracle.clover(fg.unit_gauge(dims), dims, 1.7)
    assert np.abs(A).max() == 0.0


@pytest.mark.parametrize("csw", [1.0, 1.91])
def test_clover_uniform_abelian_field_closed_form(csw):
    """Every leaf of the (0,1) plane is diag(e^{-ib}, e^{ib}, 1), so
    F_01 = diag(-i sin b, i sin b, 0) and the other planes vanish;
    sigma_01 = (i/2)[gamma_0, gamma_1] = diag(-1, 1, -1, 1) in this basis
    (gamma_0 gamma_1 = diag(i s3, i s3)), hence
    A = (csw/2) diag(-1, 1, -1, 1) (x) diag(sin b, -sin b, 0)."""
    dims = (2, 6, 2, 4)
    b = 2 * np.pi / dims[1]
    A = oracle.clover(_abelian_field(dims, b), dims, csw)
    spin = np.array([-1.0, 1.0, -1.0, 1.0])
    colour = np.array([1.0, -1.0, 0.0])
    expect = np.diag(0.5 * csw * np.sin(b) * np.kron(spin, colour))
    assert np.abs(A - expect[None]).max() < 1e-14
    # the sigma_01 factor from the oracle's own gamma matrices agrees with the closed form
    g = [oracle.gamma(mu) for mu in range(4)]
    assert np.allclose(0.5j * (g[0] @ g[1] - g[1] @ g[0]), np.diag(spin))


def test_clover_hermitian_chiral_and_gauge_covariant():
    dims = (4, 2, 4, 4)
    V = fg.volume(dims)
    U = fg.gauge_field(dims, 0.7, seed=31)
    A = oracle.clover(U, dims, 1.3)
    assert np.abs(A - A.conj().transpose(0, 2, 1)).max() < 1e-15
    g5 = np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3))
    assert np.abs(A @ g5 - g5 @ A).max() < 1e-15
    assert np.abs(A).max() > 1e-2  # not trivially zero
    g = fg.random_su3(V, 32)
    Ug = np.empty_like(U)
    for mu in range(4):
        t = shift_index(dims, mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ g[t].conj().transpose(0, 2, 1)
    G = np.einsum("xy,sab->sxayb", np.eye(4), g).reshape(V, 12, 12)
    Ag = oracle.clover(Ug, dims, 1.3)
    assert np.abs(Ag - G @ A @ G.conj().transpose(0, 2, 1)).max() < 1e-13


def test_clover_operator_gamma5_hermitian_and_local_submatrix():
    dims, block, m0 = SMALL_DIMS, SMALL_BLOCK, -0.4
    V = fg.volume(dims)
    U = fg.gauge_field(dims, 0.5, seed=33)
    A = oracle.clover(U, dims, 1.91)
    psi = fg.gaussian_source(dims, 34)
    phi = fg.gaussian_source(dims, 35)
    lhs = np.vdot(phi, G5 * oracle.dw(U, G5 * psi, dims, m0, A=A))
    rhs = np.vdot(oracle.dw(U, phi, dims, m0, A=A), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # D_sw = D_w + block-diagonal A, and D_sw^l keeps the whole site term
    Dsw = oracle.dense_operator(lambda v: oracle.dw(U, v.reshape(V, 4, 3), dims, m0, A=A).reshape(-1), 12 * V)
    Dw = _dense(U, dims, m0)
    blk = np.zeros_like(Dw)
    for s_ in range(V):
        blk[12 * s_:12 * s_ + 12, 12 * s_:12 * s_ + 12] = A[s_]
    assert np.abs(Dsw - Dw - blk).max() < 1e-14
    Dl = oracle.dense_operator(
        lambda v: oracle.dw_local(U, v.reshape(V, 4, 3), dims, block, m0, A=A).reshape(-1), 12 * V)
    dom, _ = _domain_index(dims, block)
    sd = np.repeat(dom, 12)
    assert np.abs(Dl - np.where(sd[:, None] == sd[None, :], Dsw, 0)).max() < 1e-14


def test_clover_sap_exact_local_solves_equal_series():
    """The series form of SAP (Sec. 4) holds for the clover-improved operator."""
    dims, block, m0 = (4, 4, 4, 2), (2, 2, 2, 1), -0.5
    U = fg.gauge_field(dims, 0.3, seed=0)
    V = fg.volume(dims)
    A = oracle.clover(U, dims, 1.91)
    D = oracle.dense_operator(lambda v: oracle.dw(U, v.reshape(V, 4, 3), dims, m0, A=A).reshape(-1), 12 * V)
    _, col = _domain_index(dims, block)
    sc = np.repeat(col, 12)
    perm = np.concatenate([np.where(sc == 0)[0], np.where(sc == 1)[0]])
    Dp = D[np.ix_(perm, perm)]
    h = (sc == 0).sum()
    AL = Dp.copy()
    AL[:h, h:] = 0
    AU = -(Dp - AL)
    ALi = np.linalg.inv(AL)
    M = ALi + (ALi @ AU) @ ALi
    v = fg.gaussian_source(dims, 36).reshape(-1)
    z_series = np.empty_like(v)
    z_series[perm] = M @ v[perm]
    z = oracle.sap(U, v.reshape(V, 4, 3), dims, block, m0, 2, 0, A=A).reshape(-1)
    assert np.linalg.norm(z - z_series) <= 1e-11 * np.linalg.norm(z_series)
