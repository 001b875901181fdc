"""h-/p-multigrid hierarchy, point smoothers, V-cycle and the two outer solvers (oracle).

TEST INFRASTRUCTURE ONLY. Follows the paper:

* Sec. 3.1.1 / 3.1.2 and Sec. 4.3: h-multigrid keeps p and halves the mesh; p-multigrid
  halves p down to 1 and then coarsens the mesh; "three meshes" per hierarchy;
  every level is rediscretized (mu evaluated at that level's quadrature points).
* Sec. 3.2.1 / 3.2.2: point-Jacobi with omega = 2/3; Chebyshev-accelerated Jacobi
  targeting [lambda_max/4, lambda_max] of D^-1 A, lambda_max from 10 Arnoldi iterations.
* Sec. 4.4 (Table 7): the l1-Jacobi point smoother, x += omega D_l1^-1 (b - A x) with the
  damping of all its experiments (omega = 2/3).
* Sec. 3.2.3 / 4.4 (Table 7): element-block Jacobi, x += omega M^-1 (b - A x) with M block
  diagonal: the exact element matrix on each element's interior nodes, the diagonal elsewhere.
* Sec. 3.2.2 / 4.3: V-cycle with nu_pre / nu_post smoothing steps and an exact solve
  on the coarsest grid; MG as solver until the residual norm drops by 1e8.
* Algorithm 1: MG-preconditioned CG, one V-cycle per iteration.
* Sec. 3.1.3 / 4.2 (the "low-order MG pCG" column): CG on the order-p system preconditioned by
  the exact inverse of the low-order operator -- Q1 elements on the order-p nodes -- which the
  paper applies by a factorization (here a sparse LU).

Readings where the paper is silent or garbled (the CUDA library follows the same):
* Chebyshev: the three-term recurrence of Saad, "Iterative Methods for Sparse Linear
  Systems" (2nd ed.), Alg. 12.1, applied to D^-1 A with an explicit residual each step;
  the polynomial degree equals the number of smoothing steps.
* Arnoldi: modified Gram-Schmidt on D^-1 A (interior unknowns) from a SplitMix64
  U(-1,1) start vector (counter = global node number, seed 0x1402593800000000 + level),
  lambda = largest real part of the Ritz values; min(10, n) steps on an n-unknown level.
* Algorithm 1 uses rho before computing it; it is read as standard PCG:
  r0 = b - A u0, z0 = V(r0), p0 = z0, then alpha = (z,r)/(p,Ap), ..., beta = (z',r')/(z,r).
* Stopping: ||r||_2 <= rtol * ||r_0||_2 over interior unknowns, u0 = 0.
* Coarsest grid: dense Cholesky factorization (exact solve).
* l1-Jacobi: the added diagonal is the rest of the row's l1 norm, D_l1 = diag(sum_j |a_ij|)
  over the interior unknowns (the paper cites Baker, Falgout, Kolev and Yang 2011 without
  fixing which couplings enter; on one process the full row is the one that changes the method).
* Block Jacobi: the paper inverts the element matrices exactly without saying how blocks of
  elements that share nodes combine. Read as: one block per element on its element-interior
  nodes (local indices 1..p-1 on every axis; such a node belongs to that element alone, so the
  block of the assembled matrix is the element matrix's block), and point Jacobi on the nodes
  that elements share. Overlapping element blocks (summed, or weighted by node multiplicity) and
  blocks of owned nodes were tried against Table 7 and land far from its counts; this reading
  lands next to them (2d-const 32^2, p = 8: 17 / 9 against the printed 16 / 8).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .fem import Discretization
from .transfer import prolongation

ARNOLDI_SEED = 0x1402593800000000


def _splitmix64_uniform(seed, counters):
    """SplitMix64 (Steele, Lea & Flood 2014) in counter form, output mapped to U(-1,1):
    z = seed + (c+1)*0x9E3779B97F4A7C15; z = (z^(z>>30))*0xBF58476D1CE4E5B9;
    z = (z^(z>>27))*0x94D049BB133111EB; z ^= z>>31; u = 2*(z>>11)*2^-53 - 1."""
    mask = (1 << 64) - 1
    out = np.empty(len(counters))
    for k, c in enumerate(counters):
        z = (seed + (int(c) + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z = z ^ (z >> 31)
        out[k] = 2.0 * (z >> 11) * (2.0 ** -53) - 1.0
    return out


def level_shapes(prob):
    """(nelem, p) of every level, finest first (Sec. 4.3)."""
    E = tuple(prob["nelem"])
    p = int(prob["order"])
    out = [(E, p)]
    if prob["hier"] == "p":
        while p > 1:
            p = max(1, p // 2)
            out.append((E, p))
    n_h = int(prob["n_hlevels"])
    for _ in range(n_h - 1):
        if any(e % 2 for e in E):
            raise ValueError("mesh cannot be halved")
        E = tuple(e // 2 for e in E)
        out.append((E, p))
    return out


class Level:
    def __init__(self, disc: Discretization, l1=False, block=False):
        self.disc = disc
        self.A = disc.stiffness()
        if l1:   # l1-Jacobi: D_l1 = diag(sum_j |a_ij|)
            self.dinv = 1.0 / np.asarray(abs(self.A).sum(axis=1)).ravel()
        else:
            self.dinv = 1.0 / self.A.diagonal()
        self.P = None          # prolongation from the next coarser level to this one
        self.lam = None
        self.chol = None
        self.blk_idx = None    # block Jacobi: (E, (p-1)^d) interior-numbered element-interior unknowns
        self.blk_inv = None    # and the inverses of their blocks of A
        if block and disc.p >= 2:
            self.blk_idx = element_interior_unknowns(disc)
            A = self.A.tocsr()
            self.blk_inv = np.stack([np.linalg.inv(A[idx][:, idx].toarray()) for idx in self.blk_idx])
            self.dinv_shared = self.dinv.copy()
            self.dinv_shared[self.blk_idx.ravel()] = 0.0

    def block_precondition(self, r):
        """M^-1 r: the block inverses on element-interior unknowns, D^-1 on the rest."""
        if self.blk_idx is None:
            return self.dinv * r
        z = self.dinv_shared * r
        z[self.blk_idx] = np.einsum("eij,ej->ei", self.blk_inv, r[self.blk_idx])
        return z


def element_interior_unknowns(disc: Discretization):
    """(E, (p-1)^d) interior-numbered unknowns at each element's interior local nodes (every
    local index in 1..p-1), x fastest."""
    n = disc.n
    loc = np.indices((n,) * disc.dim).reshape(disc.dim, -1)
    inner = np.all((loc > 0) & (loc < n - 1), axis=0)
    g = disc.element_nodes()[:, inner]
    pos = -np.ones(disc.N, dtype=np.int64)
    pos[disc.interior] = np.arange(len(disc.interior))
    idx = pos[g]
    assert np.all(idx >= 0)      # an element-interior node is never on the Dirichlet boundary
    return idx


class Hierarchy:
    def __init__(self, prob, arnoldi=True):
        self.prob = prob
        self.levels = []
        for E, p in level_shapes(prob):
            xyz = None
            if prob.get("node_xyz") is not None:
                # finest level: the given coordinates; coarser: the finest map at their nodes
                if not self.levels:
                    xyz = prob["node_xyz"]
                else:
                    ref = Discretization(prob["dim"], E, p).reference_coords()
                    xyz = self.levels[0].disc.map_points(ref).T
            disc = Discretization(prob["dim"], E, p, warp_amp=prob["warp_amp"],
                                  mu_a=prob["mu_a"], mu_b=prob["mu_b"], mu_k=prob["mu_k"],
                                  node_xyz=xyz, mu_fn=prob.get("mu_fn"))
            self.levels.append(Level(disc, l1=prob["smoother"] == "l1jacobi",
                                     block=prob["smoother"] == "blockjacobi"))
        for k in range(len(self.levels) - 1):
            self.levels[k].P = prolongation(self.levels[k].disc, self.levels[k + 1].disc)
        last = self.levels[-1]
        last.chol = sla.cho_factor(last.A.toarray(), lower=True)
        if arnoldi and prob["smoother"] == "cheb":
            for k, L in enumerate(self.levels[:-1]):
                L.lam = arnoldi_lambda_max(L, int(prob["arnoldi_iters"]), ARNOLDI_SEED + k)
        self.fine_applies = 0

    @property
    def fine(self):
        return self.levels[0]

    # ------------------------------------------------------------------ smoothers
    def _apply(self, k, x):
        if k == 0:
            self.fine_applies += 1
        return self.levels[k].A @ x

    def jacobi(self, k, b, x, steps):
        """x <- x + omega D^-1 (b - A x), `steps` times (Sec. 3.2.2, omega = 2/3); with the
        block smoother D^-1 r is M^-1 r (Level.block_precondition)."""
        L, w = self.levels[k], self.prob["omega"]
        block = self.prob["smoother"] == "blockjacobi"
        for s in range(steps):
            r = b if x is None else b - self._apply(k, x)
            x = (0.0 if x is None else x) + w * (L.block_precondition(r) if block else L.dinv * r)
        return x

    def chebyshev(self, k, b, x, steps):
        """Chebyshev acceleration of Jacobi on [lo, hi] = [frac*s*lam, s*lam] (Saad Alg. 12.1)."""
        L = self.levels[k]
        hi = self.prob["cheb_safety"] * L.lam
        lo = self.prob["cheb_lo_frac"] * hi
        theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        r = b if x is None else b - self._apply(k, x)
        d = L.dinv * r / theta
        x = d.copy() if x is None else x + d
        for s in range(1, steps):
            r = b - self._apply(k, x)
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * L.dinv * r
            x = x + d
            rho = rho_new
        return x

    def smooth(self, k, b, x, steps):
        if steps == 0:
            return np.zeros_like(b) if x is None else x
        if self.prob["smoother"] in ("jacobi", "l1jacobi", "blockjacobi"):
            return self.jacobi(k, b, x, steps)
        return self.chebyshev(k, b, x, steps)

    # ------------------------------------------------------------------ V-cycle
    def vcycle(self, b, x=None, k=0):
        """One V(nu_pre, nu_post) cycle on level k; x=None means a zero initial guess."""
        L = self.levels[k]
        if k == len(self.levels) - 1:
            return sla.cho_solve(L.chol, b)
        x = self.smooth(k, b, x, self.prob["nu_pre"])
        r = b - self._apply(k, x)
        rc = L.P.T @ r
        ec = self.vcycle(rc, None, k + 1)
        x = x + L.P @ ec
        return self.smooth(k, b, x, self.prob["nu_post"])

    # ------------------------------------------------------------------ solvers
    def solve_mg(self, b, rtol=1e-8, maxit=1000):
        """MG as solver: V-cycles until ||b - A x|| <= rtol ||b|| (x0 = 0)."""
        x = np.zeros_like(b)
        r0 = np.linalg.norm(b)
        hist = [r0]
        if r0 == 0.0:                       # u = 0 solves it: no cycle
            return x, 0, np.array(hist), True
        for it in range(1, maxit + 1):
            x = self.vcycle(b, None if it == 1 else x)
            r = b - self._apply(0, x)
            hist.append(np.linalg.norm(r))
            if hist[-1] <= rtol * r0:
                return x, it, np.array(hist), True
        return x, maxit, np.array(hist), False

    def solve_pcg(self, b, rtol=1e-8, maxit=1000):
        """Algorithm 1 (read as standard PCG, x0 = 0), one V-cycle per iteration."""
        u = np.zeros_like(b)
        r = b.copy()
        r0 = np.linalg.norm(r)
        hist = [r0]
        if r0 == 0.0:
            return u, 0, np.array(hist), True
        z = self.vcycle(r)
        p = z.copy()
        rho = z @ r
        for it in range(1, maxit + 1):
            h = self._apply(0, p)
            alpha = rho / (p @ h)
            u = u + alpha * p
            r = r - alpha * h
            hist.append(np.linalg.norm(r))
            if hist[-1] <= rtol * r0:
                return u, it, np.array(hist), True
            z = self.vcycle(r)
            rho_new = z @ r
            beta = rho_new / rho
            rho = rho_new
            p = z + beta * p
        return u, maxit, np.array(hist), False


def arnoldi_lambda_max(L: Level, iters: int, seed: int):
    """Largest real part of the Ritz values of D^-1 A after `iters` Arnoldi steps
    (modified Gram-Schmidt) from a seeded start vector."""
    disc = L.disc
    v = _splitmix64_uniform(seed, disc.interior)
    m = min(iters, disc.n_interior)
    H = np.zeros((m + 1, m))
    V = [v / np.linalg.norm(v)]
    for j in range(m):
        w = L.dinv * (L.A @ V[j])
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if j + 1 < m:
            V.append(w / H[j + 1, j])
    ritz = np.linalg.eigvals(H[:m, :m])
    return float(np.max(ritz.real))


def low_order_discretization(disc: Discretization) -> Discretization:
    """Q1 elements whose nodes are disc's nodes (Sec. 3.1.3): p * E elements per axis, the same
    node grid and numbering, node coordinates disc's physical ones, disc's coefficient."""
    return Discretization(disc.dim, tuple(e * disc.p for e in disc.E), 1, mu_a=disc.mu_a, mu_b=disc.mu_b,
                          mu_k=disc.mu_k, node_xyz=disc.node_coords().T, mu_fn=disc.mu_fn)


def solve_pcg_low_order(disc: Discretization, b, rtol=1e-8, maxit=1000):
    """PCG on disc's interior system A_p from u = 0, preconditioned by the exact inverse of the
    low-order interior operator A_1 (sparse LU), stopping at ||r|| <= rtol ||r_0||."""
    A = disc.stiffness()
    lu = spla.splu(low_order_discretization(disc).stiffness().tocsc())
    u = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    hist = [r0]
    if r0 == 0.0:
        return u, 0, np.array(hist), True
    z = lu.solve(r)
    p = z.copy()
    rho = z @ r
    for it in range(1, maxit + 1):
        h = A @ p
        alpha = rho / (p @ h)
        u = u + alpha * p
        r = r - alpha * h
        hist.append(np.linalg.norm(r))
        if hist[-1] <= rtol * r0:
            return u, it, np.array(hist), True
        z = lu.solve(r)
        rho_new = z @ r
        p = z + (rho_new / rho) * p
        rho = rho_new
    return u, maxit, np.array(hist), False
