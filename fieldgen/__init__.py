"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the tests.

This module holds no arithmetic of the solver itself: it only draws the
objects the method operates on (Sec. 2 of the paper defines them):

* a gauge field ``U[site][mu][row][col]`` of SU(3) link matrices,
* right-hand sides ``b[site][spin][colour]`` (Gaussian or point sources),
* random SU(3) gauge transformations ``g[site]`` (used by covariance checks).

Canonical host layout (FP64, complex interleaved as numpy complex128):

* site index ``n = n1 + d1*(n2 + d2*(n3 + d3*n4))`` with ``n4`` the time-like
  direction, so ``dims = (d1, d2, d3, d4)``;
* gauge field shape ``(V, 4, 3, 3)``; spinor fields shape ``(V, 4, 3)``;
  a batch of right-hand sides has shape ``(nrhs, V, 4, 3)``.

Link recipe: ``H = sum_a omega_a * lambda_a / 2`` over the eight Gell-Mann
matrices with ``omega_a ~ N(0, 1)`` drawn from ``numpy.random.default_rng(seed)``
in the order site (lexicographic) -> mu -> a, and ``U = exp(i * eps * H)``
evaluated as ``W diag(exp(i eps theta)) W^H`` from ``(theta, W) = eigh(H)``,
which is unitary with unit determinant to rounding.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "gell_mann",
    "gauge_field",
    "unit_gauge",
    "gaussian_source",
    "point_sources",
    "random_su3",
    "lattice_configs",
]


def volume(dims) -> int:
    d1, d2, d3, d4 = (int(x) for x in dims)
    return d1 * d2 * d3 * d4


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _exp_i_hermitian(H: np.ndarray, eps: float) -> np.ndarray:
    theta, W = np.linalg.eigh(H)
    phase = np.exp(1j * eps * theta)
    return np.einsum("...ij,...j,...kj->...ik", W, phase, W.conj())


def gauge_field(dims, eps: float, seed: int = 0, chunk: int = 1 << 18) -> np.ndarray:
    """SU(3) links ``exp(i eps H)``, H Gaussian traceless Hermitian; shape (V,4,3,3)."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    lam_half = gell_mann() / 2
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for s0 in range(0, V, chunk):
        s1 = min(V, s0 + chunk)
        omega = rng.standard_normal((s1 - s0, 4, 8))
        H = np.einsum("sma,aij->smij", omega, lam_half)
        U[s0:s1] = _exp_i_hermitian(H, eps)
    return U


def unit_gauge(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def gaussian_source(dims, seed: int = 1, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian spinor field(s): real and imaginary parts i.i.d. N(0,1).

    Drawn from ``default_rng(seed)`` as one ``standard_normal`` block of shape
    (nrhs, V, 4, 3, 2) (last axis = re, im). With ``nrhs=None`` returns (V,4,3).
    """
    V = volume(dims)
    rng = np.random.default_rng(seed)
    k = 1 if nrhs is None else int(nrhs)
    z = rng.standard_normal((k, V, 4, 3, 2))
    b = z[..., 0] + 1j * z[..., 1]
    return b[0] if nrhs is None else b


def point_sources(dims, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources ``b^(s,c)_{n,alpha,a} = delta_{n,site} delta_{alpha s} delta_{a c}``.

    Shape (12, V, 4, 3), right-hand side index ``rhs = 3*s + c``.
    """
    V = volume(dims)
    b = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            b[3 * s + c, site, s, c] = 1.0
    return b


def random_su3(V: int, seed: int) -> np.ndarray:
    """Haar-like random SU(3) matrices (QR of a complex Gaussian, det fixed to 1)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((V, 3, 3)) + 1j * rng.standard_normal((V, 3, 3))
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    Q = Q / (det ** (1.0 / 3.0))[:, None, None]
    return Q


def spectral_edges() -> dict:
    """Left spectral edges of D at m0 = 0 for the stored synthetic fields
    (written by ``python -m oracle.tune_masses``; Ritz values of the oracle)."""
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spectral_edges.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def edge_key(dims, eps, seed, csw=0.0) -> str:
    k = f"{'x'.join(map(str, dims))}_eps{eps}_seed{seed}"
    return k + (f"_csw{csw}" if csw else "")


def tuned_m0(dims, eps, seed, target, csw=0.0):
    """Bare mass putting the left spectral edge of D (with the clover term of
    coefficient csw) at ``target`` (spec(D_m0) = spec(D_0) + m0), or None if
    the edge is not stored."""
    e = spectral_edges().get(edge_key(dims, eps, seed, csw))
    return None if e is None else target - e["edge_re"]


def lattice_configs():
    """The synthetic workloads (lattice, field strength, solver settings).

    ``m0`` of the larger lattices puts the left spectral edge of D (found by
    Arnoldi on the oracle's operator) at ``target_min_abs_eig``.
    """
    cfg = _configs()
    for c in cfg.values():
        if c.get("m0") is None:
            c["m0"] = tuned_m0(c["dims"], c["eps"], c["seed"], c["target_min_abs_eig"], c.get("csw", 0.0))
    return cfg


def _configs():
    return {
        "tiny_4x4x4x4": dict(dims=(4, 4, 4, 4), eps=0.3, seed=0, m0=-0.5, block=(2, 2, 2, 2),
                              sap_cycles=4, mr_steps=4, m=20, k=5, tol=1e-10, nrhs=1),
        "wilson_16x16x16x32": dict(dims=(16, 16, 16, 32), eps=0.5, seed=0, m0=None,
                                   target_min_abs_eig=1e-2, block=(4, 4, 4, 4),
                                   sap_cycles=5, mr_steps=4, m=30, k=10, tol=1e-10, nrhs=1),
        "mixed_32x32x32x64": dict(dims=(32, 32, 32, 64), eps=0.6, seed=0, m0=None,
                                  target_min_abs_eig=1e-3, block=(4, 4, 4, 4),
                                  sap_cycles=5, mr_steps=4, m=40, k=16, tol=1e-10, nrhs=1),
        "clover_16x16x16x32": dict(dims=(16, 16, 16, 32), eps=0.5, seed=0, m0=None, csw=1.91,
                                   target_min_abs_eig=1e-2, block=(4, 4, 4, 4),
                                   sap_cycles=5, mr_steps=4, m=30, k=10, tol=1e-10, nrhs=1),
        "batched_24x24x24x48": dict(dims=(24, 24, 24, 48), eps=0.5, seed=0, m0=None,
                                    target_min_abs_eig=5e-3, block=(4, 4, 4, 4),
                                    sap_cycles=5, mr_steps=4, m=30, k=10, tol=1e-10, nrhs=12),
    }
