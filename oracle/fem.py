"""Mapped Q_p discretization of -div(mu grad u) = f, u = 0 on the boundary (oracle).

TEST INFRASTRUCTURE ONLY. Follows the paper's problem statement and discretization:

* Eq. (Poisson), Sec. 2: -div(mu grad u) = f in Omega, u = 0 on its boundary, mu >= mu_0 > 0.
* Sec. 2.1: (A_k)_ij = a(phi_i, phi_j) = int mu grad phi_i . grad phi_j,
  (f_k)_j = (f, phi_j), (M_k)_ij = (phi_i, phi_j); integrals by quadrature.
* Sec. 2.3: Omega is the image of [0,1]^d under a smooth map; tensor LGL nodal basis
  on a uniformly refined structured hexahedral (quadrilateral) mesh; isoparametric
  elements (geometry interpolated with the same basis); Jacobians at every
  quadrature point; Gauss quadrature; mu evaluated at each level's quadrature points;
  assembled sparse operators.

Readings where the paper is silent: q = p+1 Gauss points per direction; mu is
evaluated at the isoparametric image of each Gauss point; Dirichlet unknowns are
eliminated (interior numbering); the warp x_i += amp * prod_j sin(pi x_j) and the
coefficient mu = a + b sum_i cos^2(k pi x_i) are parameters of the workload. A user may
instead give the finest level's node coordinates (node_xyz) and a coefficient function
(mu_fn); a coarser level then takes the finest level's isoparametric map evaluated at its
own reference nodes (map_points).

Global nodes are numbered lexicographically, x fastest, boundary nodes included
(N = prod_i (E_i p + 1)); interior unknowns keep that order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis


class Discretization:
    """One level: structured E_1 x ... x E_d mesh of [0,1]^d, order p, mapped by the warp."""

    def __init__(self, dim, nelem, p, warp_amp=0.0, mu_a=1.0, mu_b=0.0, mu_k=2.0, q=None,
                 node_xyz=None, mu_fn=None):
        """node_xyz: optional (dim, N) physical coordinates of the global nodes (replacing the
        warp); mu_fn: optional callable, (dim, n) points -> (n,) coefficient values."""
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim = dim
        self.E = tuple(int(e) for e in (nelem if not np.isscalar(nelem) else (nelem,) * dim))
        self.p = int(p)
        self.n = self.p + 1
        self.q = int(q) if q is not None else self.p + 1
        self.warp_amp = float(warp_amp)
        self.mu_a, self.mu_b, self.mu_k = float(mu_a), float(mu_b), float(mu_k)
        self.node_xyz = None if node_xyz is None else np.asarray(node_xyz, dtype=np.float64)
        self.mu_fn = mu_fn
        self.Nn = tuple(e * self.p + 1 for e in self.E)          # nodes per axis
        self.N = int(np.prod(self.Nn))
        self.n_elem = int(np.prod(self.E))
        self.r = basis.gll_nodes(self.p)                          # 1D LGL nodes on [0,1]
        self.gq, self.gw = basis.gauss_rule(self.q)               # 1D Gauss rule on [0,1]
        idx = np.indices(self.Nn[::-1]).reshape(dim, -1)[::-1]    # idx[axis] per node, x fastest
        on_bd = np.zeros(self.N, dtype=bool)
        for ax in range(dim):
            on_bd |= (idx[ax] == 0) | (idx[ax] == self.Nn[ax] - 1)
        self.node_axis_index = idx
        self.boundary = on_bd
        self.interior = np.flatnonzero(~on_bd)
        self.n_interior = len(self.interior)

    # ---------------------------------------------------------------- geometry
    def reference_coords_1d(self, axis):
        """Reference coordinate in [0,1] of every node index along `axis`."""
        I = np.arange(self.Nn[axis])
        e = np.minimum(I // self.p, self.E[axis] - 1)
        return (e + self.r[I - e * self.p]) / self.E[axis]

    def reference_coords(self):
        """(N, dim) reference coordinates of all global nodes."""
        return np.stack([self.reference_coords_1d(ax)[self.node_axis_index[ax]]
                         for ax in range(self.dim)], axis=1)

    def warp(self, X):
        """x_i = X_i + amp * prod_j sin(pi X_j), applied to all components at once."""
        if self.warp_amp == 0.0:
            return X.copy()
        s = np.prod(np.sin(np.pi * X), axis=1)
        return X + self.warp_amp * s[:, None]

    def node_coords(self):
        """(N, dim) physical node coordinates: the given ones, else the warp of the reference ones."""
        if self.node_xyz is not None:
            return self.node_xyz.T.copy()
        return self.warp(self.reference_coords())

    def mu(self, x):
        """mu(x) for points x of shape (n, dim): mu_fn if given, else a + b sum_i cos^2(k pi x_i)."""
        if self.mu_fn is not None:
            return np.asarray(self.mu_fn(np.ascontiguousarray(x.T)), dtype=np.float64).reshape(-1)
        return self.mu_a + self.mu_b * np.sum(np.cos(self.mu_k * np.pi * x) ** 2, axis=1)

    def map_points(self, Xref):
        """Isoparametric map of this level at reference points Xref (n, dim) in [0,1]^d: the
        element containing each point (either one on an element face), then
        x = sum_a x_a prod_axis l_{a_axis}(xi_axis) over its n^d nodes (Sec. 2.3's
        isoparametric geometry). Returns (n, dim)."""
        Xref = np.asarray(Xref, dtype=np.float64)
        npt = Xref.shape[0]
        X = self.node_coords()
        eid = np.zeros(npt, dtype=np.int64)
        stride = 1
        weights = []
        for ax in range(self.dim):
            t = Xref[:, ax] * self.E[ax]
            e = np.minimum(np.floor(t).astype(np.int64), self.E[ax] - 1)
            e = np.maximum(e, 0)
            weights.append(basis.lagrange_values(self.r, t - e))     # (npt, n)
            eid += e * stride
            stride *= self.E[ax]
        nodes = self.element_nodes(eid)                               # (npt, n^d), x fastest
        w = weights[self.dim - 1]
        for ax in range(self.dim - 2, -1, -1):
            w = (w[:, :, None] * weights[ax][:, None, :]).reshape(npt, -1)
        return np.einsum("pa,pac->pc", w, X[nodes])

    # ---------------------------------------------------------------- elements
    def element_nodes(self, elems=None):
        """(ne, n^d) global node numbers of each element, local order x fastest."""
        n, p, d = self.n, self.p, self.dim
        if elems is None:
            elems = np.arange(self.n_elem)
        elems = np.asarray(elems)
        eidx = []
        rem = elems.copy()
        for ax in range(d):
            eidx.append(rem % self.E[ax])
            rem = rem // self.E[ax]
        loc = np.indices((n,) * d).reshape(d, -1)[::-1]           # loc[axis] per local node, x fastest
        g = np.zeros((len(elems), n ** d), dtype=np.int64)
        stride = 1
        for ax in range(d):
            g += (eidx[ax][:, None] * p + loc[ax][None, :]) * stride
            stride *= self.Nn[ax]
        return g

    def basis_tables(self, q=None):
        """Tensor-product basis and reference gradients at the Gauss points:
        Phi[qp, a] = phi_a(xi_qp), dPhi[k][qp, a] = d phi_a / d xi_k (xi_qp), W[qp]."""
        if q is None:
            gq, gw = self.gq, self.gw
        else:
            gq, gw = basis.gauss_rule(q)
        B = basis.lagrange_values(self.r, gq)
        D = basis.lagrange_derivatives(self.r, gq)

        def kron_axes(factors):
            # factors[axis]; the first kron factor is the slowest (last) axis
            out = factors[self.dim - 1]
            for ax in range(self.dim - 2, -1, -1):
                out = np.kron(out, factors[ax])
            return out

        Phi = kron_axes([B] * self.dim)
        dPhi = []
        for k in range(self.dim):
            fac = [B] * self.dim
            fac[k] = D
            dPhi.append(kron_axes(fac))
        w = gw
        W = kron_axes([w[:, None]] * self.dim)[:, 0]
        return Phi, dPhi, W

    def element_geometry(self, elems, tables=None):
        """Physical quadrature points, Jacobians J[e,qp,i,k] = dx_i/dxi_k, det J."""
        Phi, dPhi, W = tables if tables is not None else self.basis_tables()
        X = self.node_coords_cached()[self.element_nodes(elems)]      # (ne, nd, dim)
        xq = np.einsum("qa,eai->eqi", Phi, X)
        J = np.stack([np.einsum("qa,eai->eqi", dPhi[k], X) for k in range(self.dim)], axis=-1)
        detJ = np.linalg.det(J)
        return xq, J, detJ

    def node_coords_cached(self):
        if not hasattr(self, "_xyz"):
            self._xyz = self.node_coords()
        return self._xyz

    def element_matrices(self, elems, q=None, mass=False):
        """Dense element stiffness K_e[a,b] = sum_qp W |det J| mu (J^-T grad phi_a).(J^-T grad phi_b)
        (or mass M_e[a,b] = sum_qp W |det J| phi_a phi_b)."""
        tables = self.basis_tables(q)
        Phi, dPhi, W = tables
        xq, J, detJ = self.element_geometry(elems, tables)
        if mass:
            c = W[None, :] * np.abs(detJ)
            return np.matmul(Phi.T[None, :, :] * c[:, None, :], Phi[None, :, :])
        Jinv = np.linalg.inv(J)                                       # [e,q,k,i] = dxi_k/dx_i
        ref = np.stack(dPhi, axis=-1)                                 # (q, a, k)
        grad = np.einsum("eqki,qak->eqai", Jinv, ref)                 # physical gradients
        c = W[None, :] * np.abs(detJ) * self.mu(xq.reshape(-1, self.dim)).reshape(detJ.shape)
        ne, nq, na, d = grad.shape
        Gm = grad.transpose(0, 2, 1, 3).reshape(ne, na, nq * d)
        Gc = (grad * c[:, :, None, None]).transpose(0, 2, 1, 3).reshape(ne, na, nq * d)
        return np.matmul(Gc, Gm.transpose(0, 2, 1))

    def assemble(self, mass=False, chunk=None, q=None):
        """Full (N x N, Dirichlet nodes included) CSR stiffness or mass matrix."""
        nd = self.n ** self.dim
        if chunk is None:
            chunk = max(1, int(2.0e6 // (nd * nd)))
        rows, cols, vals = [], [], []
        itype = np.int32 if self.N < 2 ** 31 else np.int64
        for s in range(0, self.n_elem, chunk):
            el = np.arange(s, min(self.n_elem, s + chunk))
            K = self.element_matrices(el, q=q, mass=mass)
            g = self.element_nodes(el).astype(itype)
            rows.append(np.broadcast_to(g[:, :, None], K.shape).ravel())
            cols.append(np.broadcast_to(g[:, None, :], K.shape).ravel())
            vals.append(K.ravel())
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.N, self.N)).tocsr()
        A.sum_duplicates()
        return A

    def stiffness(self):
        """Interior (Dirichlet-eliminated) stiffness matrix A_k, CSR."""
        if not hasattr(self, "_A"):
            A = self.assemble()
            self._A = A[self.interior][:, self.interior].tocsr()
        return self._A

    def rhs(self, f_nodal):
        """b = (f_h, phi_j) for interior j, f_h the nodal interpolant of f (all nodes)."""
        M = self.assemble(mass=True)
        return (M @ np.asarray(f_nodal, dtype=np.float64))[self.interior]

    def to_full(self, v_interior):
        out = np.zeros(self.N)
        out[self.interior] = v_interior
        return out

    # ---------------------------------------------------------- sampled rows
    def apply_rows(self, x_full, rows):
        """(A x)_i for selected global nodes i by the weak form itself:
        (A x)_i = sum over elements e containing node i of
        sum_qp W |det J| mu (J^-T grad u_h) . (J^-T grad phi_i),  u_h = sum_b x_b phi_b,
        with grad u_h evaluated from the dense basis tables (no assembly). Boundary
        entries of x are taken as zero and boundary rows return zero. This is the
        form used at sizes where A cannot be assembled."""
        x_full = np.asarray(x_full, dtype=np.float64).copy()
        x_full[self.boundary] = 0.0
        return self._weak_rows(rows, x_full)

    def diag_rows(self, rows):
        """A_ii = a(phi_i, phi_i) for selected global nodes (the weak form with u_h = phi_i)."""
        return self._weak_rows(rows, None)

    def mass_rows(self, f_full, rows):
        """(M f)_i = (f_h, phi_i) for selected global nodes i (Sec. 2.1's load vector f_k), f_h the
        nodal interpolant of f over all N nodes: sum over the elements e containing node i of
        sum_qp W |det J| f_h(x_qp) phi_i(x_qp), with f_h and phi_i from the dense basis table
        (no assembly). Boundary rows return zero, as the interior load vector has none."""
        f_full = np.asarray(f_full, dtype=np.float64)
        out = np.zeros(len(rows))
        Phi, dPhi, W = tables = self.basis_tables()
        cache = {}
        for r_i, g in enumerate(rows):
            if self.boundary[g]:
                continue
            for e in self._elements_of_node(g):
                e = int(e)
                if e not in cache:
                    _, _, detJ = self.element_geometry([e], tables)
                    gl = self.element_nodes([e])[0]
                    cache[e] = (W * np.abs(detJ[0]), gl, Phi @ f_full[gl])
                c, gl, fq = cache[e]
                a = int(np.flatnonzero(gl == g)[0])
                out[r_i] += np.sum(c * fq * Phi[:, a])
        return out

    def _elements_of_node(self, g):
        p, d = self.p, self.dim
        I = [self.node_axis_index[ax][g] for ax in range(d)]
        cand = []
        for ax in range(d):
            cand.append([e for e in (I[ax] // p - 1, I[ax] // p)
                         if 0 <= e < self.E[ax] and e * p <= I[ax] <= e * p + p])
        elems = []
        for combo in np.array(np.meshgrid(*cand, indexing="ij")).reshape(d, -1).T:
            lin, stride = 0, 1
            for ax in range(d):
                lin += int(combo[ax]) * stride
                stride *= self.E[ax]
            elems.append(lin)
        return np.array(elems)

    def _weak_rows(self, rows, x_full):
        out = np.zeros(len(rows))
        d = self.dim
        tables = self.basis_tables()
        Phi, dPhi, W = tables
        ref = np.stack(dPhi, axis=-1)                                  # (q, a, k)
        cache = {}

        def element(e):
            if e not in cache:
                xq, J, detJ = self.element_geometry([e], tables)
                Jinv = np.linalg.inv(J[0])
                c = W * np.abs(detJ[0]) * self.mu(xq[0])
                gl = self.element_nodes([e])[0]
                gu = None
                if x_full is not None:
                    gu_ref = np.stack([dPhi[m] @ x_full[gl] for m in range(d)], axis=-1)
                    gu = np.einsum("qki,qk->qi", Jinv, gu_ref)
                cache[e] = (Jinv, c, gl, gu)
            return cache[e]

        for r_i, g in enumerate(rows):
            if self.boundary[g]:
                continue
            for e in self._elements_of_node(g):
                Jinv, c, gl, gu = element(int(e))
                a = int(np.flatnonzero(gl == g)[0])
                gphi = np.einsum("qki,qk->qi", Jinv, ref[:, a, :])
                out[r_i] += np.sum(c * np.sum((gphi if gu is None else gu) * gphi, axis=1))
        return out
