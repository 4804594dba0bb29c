"""Constitutive pieces: cofactor algebra, polar decomposition, fixed-corotated solid.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

* cof(F)_ab = 1/2 eps_agk eps_bdl F_gd F_kl, i.e. J F^{-T} for invertible F.
  The surface energy of the paper (Eq. pestul, and the discrete energy e(y) in
  section "Momentum Update") integrates |J F^{-T} dA| = |cof(F) dA|.
* dcof(F)[dF]_ab = eps_agk eps_bdl dF_gd F_kl (the derivative of the quadratic form).
* Fixed corotated (section "Constitutive Models"): psi = mu sum (sigma_a - 1)^2
  + lambda/2 (J - 1)^2 with the polar SVD F = U Sigma V^T (U, V rotations, the
  smallest singular value carries the sign of det F); R = U V^T, S = V Sigma V^T.
  P = dpsi/dF = 2 mu (F - R) + lambda (J - 1) cof(F).
  dP = 2 mu (dF - dR) + lambda (cof F : dF) cof F + lambda (J - 1) dcof(F)[dF],
  with dR = R [w]x and (tr(S) I - S) w = axial(R^T dF - dF^T R)
  (from R^T dF = W S + dS with W = R^T dR skew and dS symmetric).
"""
import numpy as np


def levi_civita():
    e = np.zeros((3, 3, 3))
    e[0, 1, 2] = e[1, 2, 0] = e[2, 0, 1] = 1.0
    e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = -1.0
    return e


EPS = levi_civita()


def cof(F):
    """Cofactor matrix of (..., 3, 3) matrices."""
    return 0.5 * np.einsum("agk,bdl,...gd,...kl->...ab", EPS, EPS, F, F)


def dcof(F, dF):
    """Directional derivative of cof at F along dF."""
    return np.einsum("agk,bdl,...gd,...kl->...ab", EPS, EPS, dF, F)


def skew_axial(K):
    """u with [u]x = (K - K^T)/2 for (..., 3, 3) K."""
    return 0.5 * np.stack([K[..., 2, 1] - K[..., 1, 2], K[..., 0, 2] - K[..., 2, 0],
                           K[..., 1, 0] - K[..., 0, 1]], -1)


def cross_matrix(u):
    z = np.zeros(u.shape[:-1])
    return np.stack([np.stack([z, -u[..., 2], u[..., 1]], -1),
                     np.stack([u[..., 2], z, -u[..., 0]], -1),
                     np.stack([-u[..., 1], u[..., 0], z], -1)], -2)


def polar(F):
    """Polar SVD: rotations U, V and signed singular values; returns R, S, sigma."""
    U, sig, Vt = np.linalg.svd(F)
    sig = sig.copy()
    U = U.copy()
    Vt = Vt.copy()
    dU = np.linalg.det(U) < 0
    U[dU, :, 2] *= -1.0
    sig[dU, 2] *= -1.0
    dV = np.linalg.det(Vt) < 0
    Vt[dV, 2, :] *= -1.0
    sig[dV, 2] *= -1.0
    R = U @ Vt
    S = np.einsum("pka,pk,pkb->pab", Vt, sig, Vt)
    return R, S, sig


def fcr_energy(F, mu, lam):
    _, _, sig = polar(F)
    J = np.linalg.det(F)
    return mu * np.sum((sig - 1.0) ** 2, -1) + 0.5 * lam * (J - 1.0) ** 2


def fcr_P(F, mu, lam):
    R, _, _ = polar(F)
    J = np.linalg.det(F)
    return 2.0 * mu[:, None, None] * (F - R) + (lam * (J - 1.0))[:, None, None] * cof(F)


def fcr_dP(F, dF, mu, lam):
    R, S, _ = polar(F)
    J = np.linalg.det(F)
    C = cof(F)
    M = np.einsum("pka,pkb->pab", R, dF)                 # R^T dF
    rhs = 2.0 * skew_axial(M)                            # axial(M - M^T)
    trS = np.trace(S, axis1=1, axis2=2)
    Kmat = trS[:, None, None] * np.eye(3) - S
    w = np.linalg.solve(Kmat, rhs[..., None])[..., 0]
    dR = R @ cross_matrix(w)
    dJ = np.einsum("pab,pab->p", C, dF)
    return (2.0 * mu[:, None, None] * (dF - dR)
            + (lam * dJ)[:, None, None] * C
            + (lam * (J - 1.0))[:, None, None] * dcof(F, dF))
