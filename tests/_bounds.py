"""A-priori error bound for one particle's field computed with FP32 pair arithmetic.

Model (u = 2^-24, the FP32 unit roundoff), for target i and source j in the staging
frame (positions p relative to the centroid):
  - each staged coordinate carries a rounding error of at most u |p|, so the FP32
    separation d_ij is off by at most about u (|p_i| + |p_j|) plus one rounding of d;
  - the pair term d / (d^2 + eps^2)^(3/2) amplifies a relative error of d at most
    about three times, and the hardware reciprocal square root adds at most 2^-21;
  - FP32 partial sums over a tile of L terms add at most (L - 1) u sum |terms|
    (the standard recursive-summation bound); the FP64 fold is negligible.
The bound below is eight times the first two terms plus the summation term; a correct
kernel stays far inside it, while a wrong pair, index or sign breaks it at once.
"""
import numpy as np

U32 = 2.0 ** -24


def field_error_bound(pos, w, eps, idx, k_e, tile=256, chunk=256, split=False):
    """Per-target bound on |E_gpu - E_exact| [V/m] for targets idx (all weights w).

    split=True models hi/lo staging: each coordinate then carries about u^2 |p| of
    rounding, so the separation term shrinks by a factor u.
    """
    p = pos - pos.mean(axis=0)
    pn = np.linalg.norm(p, axis=1)
    out = np.empty(len(idx))
    for a in range(0, len(idx), chunk):
        ii = np.asarray(idx[a:a + chunk])
        d = p[ii, None, :] - p[None, :, :]
        d2 = np.einsum("ijk,ijk->ij", d, d)
        dn = np.sqrt(d2)
        s = d2 + eps * eps
        with np.errstate(divide="ignore", invalid="ignore"):
            mag = np.where(s > 0, dn / s ** 1.5, 0.0)
            ratio = np.where(dn > 0, (pn[ii, None] + pn[None, :]) / dn, 0.0)
        mag[np.arange(len(ii)), ii] = 0.0
        ratio[np.arange(len(ii)), ii] = 0.0
        pos_term = 8 * U32 * ratio * (U32 if split else 1.0)
        per_pair = mag * (pos_term + 8 * U32 + 8 * 2.0 ** -21)
        out[a:a + chunk] = per_pair.sum(axis=1) + (tile - 1) * U32 * mag.sum(axis=1)
    return k_e * w * out
