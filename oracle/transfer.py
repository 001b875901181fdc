"""Inter-grid transfer operators (oracle; test infrastructure only).

Sec. 2.2, Eq. (Pstencil): the prolongation's entries are the coarse-grid basis
functions evaluated at the fine-grid nodes, P_ij = phi_j^{k-1}(p_i); restriction is
the adjoint with respect to the mass-weighted inner products, which amounts to
applying P^T to residual vectors.

P is assembled here entry by entry from that definition (no Kronecker factoring).
The fine nodes are located in the coarse mesh in reference coordinates (the levels
are nested in [0,1]^d); for an h-coarsened level each coarse element is the union
of 2^d fine elements, for a p-coarsened level the mesh is the same.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis


def prolongation(fine, coarse, interior=True):
    """Sparse P (fine.N x coarse.N, or interior x interior) with P_ij = phi_j^coarse(p_i)."""
    d = fine.dim
    if fine.dim != coarse.dim:
        raise ValueError("dimension mismatch")
    ratio = []
    for ax in range(d):
        if fine.E[ax] == coarse.E[ax]:
            ratio.append(1)
        elif fine.E[ax] == 2 * coarse.E[ax]:
            ratio.append(2)
        else:
            raise ValueError("levels are not nested")
    # Per axis: for every fine node index I its parent coarse element and the values of
    # the coarse element's 1D Lagrange basis at the node's reference coordinate.
    ec_ax, val_ax = [], []
    for ax in range(d):
        I = np.arange(fine.Nn[ax])
        ef = np.minimum(I // fine.p, fine.E[ax] - 1)
        i = I - ef * fine.p
        xi_c = ((ef % ratio[ax]) + fine.r[i]) / ratio[ax]
        ec_ax.append(ef // ratio[ax])
        val_ax.append(basis.lagrange_values(coarse.r, xi_c))       # (Nf_ax, n_c)
    local = np.indices((coarse.n,) * d).reshape(d, -1)[::-1]       # coarse local nodes, x fastest
    v = np.ones((fine.N, local.shape[1]))
    gc = np.zeros((fine.N, local.shape[1]), dtype=np.int64)
    stride = 1
    for ax in range(d):
        Ig = fine.node_axis_index[ax]                               # fine node index along ax
        v *= val_ax[ax][Ig][:, local[ax]]
        gc += (ec_ax[ax][Ig][:, None] * coarse.p + local[ax][None, :]) * stride
        stride *= coarse.Nn[ax]
    rows = np.broadcast_to(np.arange(fine.N)[:, None], v.shape)
    nz = v != 0.0
    P = sp.coo_matrix((v[nz], (rows[nz], gc[nz])), shape=(fine.N, coarse.N)).tocsr()
    if interior:
        P = P[fine.interior][:, coarse.interior].tocsr()
    return P
