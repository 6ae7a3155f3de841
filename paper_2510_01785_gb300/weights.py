"""Ring quadrature weights (Sec. IV-A): a plan-time computation on the host.

The analysis of Eq. 26-27 weights every pixel of ring y by w_y; Eq. 1 uses
the equal 4 pi / Npix.  ring_weights() returns weights for which the ring
quadrature of the axisymmetric functions lambda_l0 is as exact as the
HEALPix ring latitudes allow:

    sum_y N_y w_y lambda_l0(z_y) = integral of lambda_l0 over the sphere
                                 = sqrt(4 pi) if l = 0 else 0,   l even <= 2 lmax

(odd l hold by the north/south symmetry of the weights).  The rings do not
sit at Gauss nodes, and with 2 nside unknowns the system is either
overdetermined or too ill-conditioned to solve exactly, so it is solved in
the least-squares sense with a Tikhonov term that keeps the weights near the
equal ones (relative deviation d_y = w_y / w_eq - 1, penalty alpha |d|^2),
then scaled so that the total area is exactly 4 pi.  With 2 nside unknowns
and lmax + 1 conditions the system can be met up to lmax of about 1.5 nside;
there the weights cut the analysis error of band-limited maps 5-50 times
(the order of magnitude Sec. IV-A reports), at lmax = 2 nside about twice,
and at 3 nside - 1 not at all: there the error comes from the polar rings,
too short to resolve the high m, which no latitude weight can repair.  The functions lambda_l0
come from Bonnet's recurrence in FP64; the ring latitudes and lengths are
the closed forms of the HEALPix geometry (Sec. III-A).
"""
from __future__ import annotations

import numpy as np


def ring_latitudes(nside: int):
    """(z_y, N_y) of the 4 nside - 1 rings, north to south."""
    i = np.arange(1, 4 * nside, dtype=np.int64)
    ii = np.minimum(i, 4 * nside - i)
    cap = ii < nside
    N = np.where(cap, 4 * ii, 4 * nside)
    z = np.where(cap, 1.0 - ii.astype(np.float64) ** 2 / (3.0 * nside * nside),
                 2.0 * (2 * nside - ii) / (3.0 * nside))
    z = np.where(i > 2 * nside, -z, z)
    return z, N


def _lambda_l0(lmax2: int, z: np.ndarray) -> np.ndarray:
    """[lmax2 + 1][len(z)]: sqrt((2l + 1) / 4 pi) P_l(z), Bonnet's recurrence."""
    out = np.empty((lmax2 + 1, z.size))
    p0, p1 = np.ones_like(z), z.copy()
    out[0] = p0
    if lmax2 >= 1:
        out[1] = p1
    for l in range(2, lmax2 + 1):
        p0, p1 = p1, ((2 * l - 1) * z * p1 - (l - 1) * p0) / l
        out[l] = p1
    return out * np.sqrt((2 * np.arange(lmax2 + 1) + 1) / (4 * np.pi))[:, None]


def quadrature_residual(w: np.ndarray, nside: int, lmax: int) -> float:
    """|| sum_y N_y w_y lambda_l0(z_y) - sqrt(4 pi) delta_l0 || over even l <= 2 lmax."""
    z, N = ring_latitudes(nside)
    lam = _lambda_l0(2 * lmax, z)[0::2]
    b = np.zeros(lam.shape[0])
    b[0] = np.sqrt(4 * np.pi)
    return float(np.linalg.norm(lam @ (N * np.asarray(w, np.float64)) - b))


ALPHAS = (1e-8, 1e-6, 1e-4, 1e-2)
MAX_DEVIATION = 0.2


def _solve(A, b, npair, w_eq, alpha):
    r = b - A @ np.full(npair, w_eq)
    M = np.vstack([A * w_eq, np.sqrt(alpha) * np.eye(npair)])
    d = np.linalg.lstsq(M, np.concatenate([r, np.zeros(npair)]), rcond=None)[0]
    return w_eq * (1.0 + d)


def ring_weights(nside: int, lmax: int, alpha: float | None = None) -> np.ndarray:
    """float64 [4 nside - 1] ring weights, symmetric north/south.

    alpha None: the smallest Tikhonov weight of ALPHAS whose weights all stay
    within MAX_DEVIATION of the equal ones (so positive).  Where the
    conditions can be met (lmax up to about 1.5 nside) that is a tiny alpha
    and the quadrature is nearly exact; beyond, the least-squares solution
    oscillates and a larger alpha keeps it tame."""
    z, N = ring_latitudes(nside)
    npair = 2 * nside
    zp, Np = z[:npair], N[:npair].astype(np.float64)
    mult = np.where(np.arange(npair) == npair - 1, 1.0, 2.0)  # a pair's two rings, the equator once
    lam = _lambda_l0(2 * lmax, zp)[0::2]
    A = lam * (Np * mult)[None, :]
    b = np.zeros(A.shape[0])
    b[0] = np.sqrt(4 * np.pi)
    w_eq = 4 * np.pi / (12.0 * nside * nside)
    for a in ((alpha,) if alpha is not None else ALPHAS):
        wp = _solve(A, b, npair, w_eq, a)
        if alpha is not None or np.max(np.abs(wp / w_eq - 1.0)) < MAX_DEVIATION:
            break
    wp *= 4 * np.pi / float(np.sum(Np * mult * wp))
    return np.concatenate([wp, wp[:-1][::-1]])
