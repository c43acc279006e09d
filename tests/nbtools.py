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
