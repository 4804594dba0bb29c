"""Conservative surface-particle resampling (split).

TEST INFRASTRUCTURE ONLY (FP64 oracle).

Paper, section "Conservative Surface Particle Resampling":
* balance particle: b_r = s_r + 2 (x_p(r) - s_r) with p(r) the closest interior
  particle to s_r (Eq. pbal);
* particle groups Pi_p = { r : p(r) = p };
* mass split m~_p = m_p / (2 |Pi_p| + 1) given to x_p and to every s_r, b_r of
  its group, which all take v_p and A_p (Eq. cons_mom keeps the centre of mass).

Reading: ties in the closest-particle search go to the smaller particle index.
Squared distances are formed as (dx*dx + dy*dy) + dz*dz.
"""
import numpy as np


def nearest_parent(x, s, chunk=512):
    """Brute-force argmin_p |x_p - s_r|^2 for every surface sample r."""
    x = np.asarray(x, np.float64)
    s = np.asarray(s, np.float64)
    out = np.empty(s.shape[0], np.int64)
    best = np.empty(s.shape[0])
    for lo in range(0, s.shape[0], chunk):
        sc = s[lo:lo + chunk]
        d0 = sc[:, None, 0] - x[None, :, 0]
        d1 = sc[:, None, 1] - x[None, :, 1]
        d2 = sc[:, None, 2] - x[None, :, 2]
        dist = (d0 * d0 + d1 * d1) + d2 * d2
        out[lo:lo + chunk] = np.argmin(dist, axis=1)  # first minimum = smallest index
        best[lo:lo + chunk] = dist[np.arange(sc.shape[0]), out[lo:lo + chunk]]
    return out, best


def split(x, m, s, parent=None):
    """Returns parent[r], group count |Pi_p|, split mass m~_p and balance positions b_r."""
    if parent is None:
        parent, _ = nearest_parent(x, s)
    count = np.bincount(parent, minlength=x.shape[0]).astype(np.int64)
    mt = m / (2.0 * count + 1.0)
    b = s + 2.0 * (x[parent] - s)
    return parent, count, mt, b
