"""Test helpers: force-error metrics and small utilities (no method arithmetic
beyond the conditioning scales used to normalise errors)."""
import numpy as np


def condition_scales(m, xp, vp, eps2, idx, chunk=64):
    """A_i = sum_j m_j/(r^2+eps^2) and K_i = sum_j m_j(|w|/(r^2+eps^2)^{3/2} + 3|r.w||r|/(r^2+eps^2)^{5/2})
    over j != i: the magnitudes the sums would have without cancellation."""
    idx = np.asarray(idx)
    A = np.zeros(idx.size)
    K = np.zeros(idx.size)
    for q0 in range(0, idx.size, chunk):
        ii = idx[q0:q0 + chunk]
        r = xp[None, :, :] - xp[ii][:, None, :]
        w = vp[None, :, :] - vp[ii][:, None, :]
        d2 = np.einsum("ijk,ijk->ij", r, r) + eps2
        rn = np.sqrt(np.einsum("ijk,ijk->ij", r, r))
        wn = np.sqrt(np.einsum("ijk,ijk->ij", w, w))
        rw = np.abs(np.einsum("ijk,ijk->ij", r, w))
        mask = np.ones_like(d2, dtype=bool)
        mask[np.arange(ii.size), ii] = False
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = np.where(mask, m[None, :] / d2, 0.0)
            tk = np.where(mask, m[None, :] * (wn / d2 ** 1.5 + 3 * rw * rn / d2 ** 2.5), 0.0)
        A[q0:q0 + chunk] = ta.sum(1)
        K[q0:q0 + chunk] = tk.sum(1)
    return A, K


def rel_errors(x_gpu, x_ref, scale, cancel=1e-3):
    """Per-particle |dx|/|x_ref|, or |dx|/scale where |x_ref| < cancel * scale (nearly cancelling sums)."""
    d = np.linalg.norm(np.atleast_2d(x_gpu - x_ref).reshape(len(scale), -1), axis=1)
    nr = np.linalg.norm(np.atleast_2d(x_ref).reshape(len(scale), -1), axis=1)
    den = np.where(nr >= cancel * scale, nr, scale)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d == 0.0, 0.0, d / den)   # an exact zero matches an exact zero


def rel_scalar(x_gpu, x_ref):
    d = np.abs(x_gpu - x_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d == 0.0, 0.0, d / np.abs(x_ref))


def stats(e):
    e = np.asarray(e)
    return {"max": float(e.max()), "p99": float(np.percentile(e, 99)), "median": float(np.median(e))}


def pow2_distance(c):
    """Relative distance of c > 0 to the nearest power of two, |c - 2^e| / c."""
    e = np.floor(np.log2(c))
    lo = np.exp2(e)
    return np.minimum(c - lo, 2.0 * lo - c) / c


def aarseth_tie_window(a, k, a2p, a3, dt, ea, ek):
    """Relative change of the Aarseth candidate sqrt(eta N / D),
    N = |a||a2p| + |k|^2, D = |k||a3| + |a2p|^2, that force errors of at most ea
    (acceleration) and ek (jerk) in the new forces can cause.

    The corrector's finite differences carry a force error into a2p = a2 + a3 dt and
    a3 with the factors of the corrector (a2 = -6 da/dt^2 - (4 k0 + 2 k1)/dt,
    a3 = 12 da/dt^3 + 6 (k0 + k1)/dt^2, da = a0 - a1):
      |d a2p| <= 6 ea / dt^2 + 4 ek / dt,   |d a3| <= 12 ea / dt^3 + 6 ek / dt^2.
    With the triangle inequality on every norm and the products expanded in full,
    |dN| <= ea |a2p| + (|a| + ea) |d a2p| + 2 |k| ek + ek^2 and
    |dD| <= ek |a3| + (|k| + ek) |d a3| + (2 |a2p| + |d a2p|) |d a2p|, so the candidate
    changes by a factor within [sqrt((1 - rN)/(1 + rD)), sqrt((1 + rN)/(1 - rD))],
    rN = |dN|/N, rD = |dD|/D. Returns the larger deviation from 1 (inf if rD >= 1).
    Vectors are rows of (s, 3) arrays; dt, ea, ek are (s,) arrays."""
    na, nk = np.linalg.norm(a, axis=1), np.linalg.norm(k, axis=1)
    np_, n3 = np.linalg.norm(a2p, axis=1), np.linalg.norm(a3, axis=1)
    d2p = 6.0 * ea / dt ** 2 + 4.0 * ek / dt
    d3 = 12.0 * ea / dt ** 3 + 6.0 * ek / dt ** 2
    N = na * np_ + nk * nk
    D = nk * n3 + np_ * np_
    dN = ea * np_ + (na + ea) * d2p + 2.0 * nk * ek + ek * ek
    dD = ek * n3 + (nk + ek) * d3 + (2.0 * np_ + d2p) * d2p
    with np.errstate(divide="ignore", invalid="ignore"):
        rN, rD = dN / N, dD / D
        up = np.sqrt((1.0 + rN) / (1.0 - rD)) - 1.0
        down = 1.0 - np.sqrt(np.maximum(1.0 - rN, 0.0) / (1.0 + rD))
    return np.where(rD < 1.0, np.maximum(up, down), np.inf)


def start_tie_window(a, k, ea, ek):
    """Relative change of the start candidate eta |a| / |k| that force errors of at most
    ea, ek can cause (the triangle inequality on both norms)."""
    na, nk = np.linalg.norm(a, axis=1), np.linalg.norm(k, axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        up = (1.0 + ea / na) / (1.0 - ek / nk) - 1.0
        down = 1.0 - (1.0 - ea / na) / (1.0 + ek / nk)
    return np.where(ek < nk, np.maximum(up, down), np.inf)
