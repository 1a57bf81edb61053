"""Naive Nystrom pair sum over the quadrature nodes.

y_j = sum_{n != j} G(y_j, y_n) w_n f_n with G = (i/4) H0^(1)(k |x - y|): the
plain quadrature of the volume potential V_Omega[f] at the nodes (Eq. vol_pot,
Eq. linear_system of the paper), the self term n = j omitted.  The VDIM
correction (oracle.vdim) supplies the singular and near-singular part.
"""
import numpy as np

from .bessel import hankel01


def naive_rows(nodes, weights, k, f, rows, block=256):
    """Return y[rows] (complex128) of the naive pair sum for density f."""
    rows = np.asarray(rows, dtype=np.int64)
    wf = weights * f
    out = np.zeros(rows.size, dtype=np.complex128)
    for b0 in range(0, rows.size, block):
        r = rows[b0:b0 + block]
        dx = nodes[r, 0][:, None] - nodes[None, :, 0]
        dy = nodes[r, 1][:, None] - nodes[None, :, 1]
        dist = np.sqrt(dx * dx + dy * dy)
        self_mask = np.zeros(dist.shape, dtype=bool)
        self_mask[np.arange(r.size), r] = True
        dist[self_mask] = 1.0
        h0, _ = hankel01(k * dist)
        g = 0.25j * h0
        g[self_mask] = 0.0
        out[b0:b0 + block] = g @ wf
    return out


def naive_apply(nodes, weights, k, f):
    """Full naive pair sum (all rows)."""
    return naive_rows(nodes, weights, k, f, np.arange(nodes.shape[0]))
