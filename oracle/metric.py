"""DCT-entropy image-quality metric and stopping rule (Section 2.2), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here (the text is garbled or silent on these):
  * Eq. 1 pairs x with M although x runs over the width; it is read as the
    standard separable orthonormal 2-D DCT-II: column index x (width W) with
    column frequency u, row index y (height H) with row frequency v.
  * Region S (Eq. 6, Fig. 2c) is the upper-left triangle
    {(u, v) : u < X_S, v < Y_S, u*Y_S + v*X_S < X_S*Y_S} (integer test).
  * The prefactor "2/S^2" of Eq. 12 is read as 1/G_S = 2/(X_S*Y_S) (Eq. 6).
  * L_2 in Eq. 12 is the 2-norm of the coefficients in S (default) or of the
    whole DCT (= 2-norm of the image by Parseval) when ``l2_over_region`` is 0.
  * "abslog2" is log2|.|, with 0*log 0 = 0.
  * X_S, Y_S follow Eqs. 7, 9, 10, 11; the result is floored and clamped to
    [min(2, W), W] (resp. H).
  * "Stop when the entropy shows a decreasing trend": the predicted iteration
    is the first k >= 1 with E_{k+1} < E_k; with no decrease it is the first
    argmax of E over the iterations run.
"""
from __future__ import annotations

import math

import numpy as np


def mip_z(v) -> np.ndarray:
    """Maximum projection of a volume v[Nz][H][W] along z (Section 2.2)."""
    return np.asarray(v, dtype=np.float64).max(axis=0)


def dct_basis(Z: int) -> np.ndarray:
    """C[k, x] = c(k, Z) * cos((2x+1) pi k / (2Z)), Eqs. 2-4."""
    k = np.arange(Z, dtype=np.float64)[:, None]
    x = np.arange(Z, dtype=np.float64)[None, :]
    C = np.cos((2.0 * x + 1.0) * math.pi * k / (2.0 * Z))
    C[0, :] *= math.sqrt(1.0 / Z)
    C[1:, :] *= math.sqrt(2.0 / Z)
    return C


def dct2(f) -> np.ndarray:
    """F[v, u] = sum_{y, x} f[y, x] C_u(x; W) C_v(y; H) (Eq. 1 as read above).

    Row index of the result is the row frequency v, column index is the column
    frequency u."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    return dct_basis(H) @ f @ dct_basis(W).T


def region_size(Nnum: int, H: int, W: int, dML_um: float = 150.0, Q: float = 40.0,
                NA: float = 0.95, lambda_um: float = 0.525) -> tuple[int, int]:
    """(X_S, Y_S) from Eqs. 7, 9, 10, 11.

    P_u = d_ML / (Q * Nnum)              (Eq. 7, pixel size in object space)
    d_psf = 1.22 * lambda * Nnum / NA    (Eq. 11)
    X_S = P_u * W / d_psf, Y_S = P_u * H / d_psf   (Eqs. 9, 10)
    """
    P_u = dML_um / (Q * Nnum)
    d_psf = 1.22 * lambda_um * Nnum / NA
    xs = P_u * W / d_psf
    ys = P_u * H / d_psf

    def clamp(val, n):
        return int(min(n, max(min(2, n), math.floor(val))))

    return clamp(xs, W), clamp(ys, H)


def region_mask(XS: int, YS: int) -> np.ndarray:
    """Boolean [YS, XS] mask (rows v, columns u) of the triangle S."""
    v = np.arange(YS)[:, None]
    u = np.arange(XS)[None, :]
    return (u * YS + v * XS) < (XS * YS)


def dct_entropy(f, XS: int, YS: int, l2_over_region: bool = True) -> float:
    """DCT entropy of image f over the triangle S (Eqs. 5, 6, 12)."""
    f = np.asarray(f, dtype=np.float64)
    F = dct2(f)
    coef = F[:YS, :XS][region_mask(XS, YS)]
    norm = math.sqrt(float(np.sum(coef * coef))) if l2_over_region \
        else math.sqrt(float(np.sum(f * f)))
    if norm == 0.0:
        return 0.0
    p = np.abs(coef) / norm
    nz = p > 0
    s = float(np.sum(p[nz] * np.log2(p[nz])))
    G = XS * YS / 2.0
    return -s / G


def predicted_iteration(E) -> int:
    """1-based iteration k at which the entropy first decreases afterwards
    (E_{k+1} < E_k, strict); the first argmax when it never decreases."""
    E = list(E)
    if not E:
        return 0
    for k in range(1, len(E)):
        if E[k] < E[k - 1]:
            return k
    best = 0
    for k in range(1, len(E)):
        if E[k] > E[best]:
            best = k
    return best + 1
