"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the multigrid method: it only draws random
numbers (SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and describes the workloads as plain parameter sets.

Workloads follow the paper's test problems (Sec. 4.1: unit square/cube, constant
or strongly varying coefficient on a warped domain) at the sizes used by the
benchmarks of this library; the warp map and coefficient amplitude are given
explicitly because the paper only shows its warped meshes as a figure (Fig. 4).
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream seeded with `seed`.

    Counter form: output_i = mix(seed + (i + 1) * gamma) (mod 2^64).
    """
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, start: int = 0) -> np.ndarray:
    """U(-1,1) doubles: 2 * (z >> 11) * 2^-53 - 1."""
    z = splitmix64(seed, count, start)
    return 2.0 * (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 1.0


def nodal_field(seed: int, n_nodes: int) -> np.ndarray:
    """Seeded nodal right-hand-side samples f ~ U(-1,1), one per global node."""
    return uniform_pm1(seed, n_nodes)


# ---------------------------------------------------------------------------
# Workload descriptions (plain parameters; both implementations read them).
# mu(x) = mu_a + mu_b * sum_i cos^2(mu_k * pi * x_i); warp x_i += amp * prod_j sin(pi x_j)
# ---------------------------------------------------------------------------

def problem(dim, nelem, order, *, warp_amp=0.0, mu_a=1.0, mu_b=0.0, mu_k=2.0,
            hier="h", n_hlevels=3, smoother="cheb", nu_pre=3, nu_post=3,
            omega=2.0 / 3.0, arnoldi_iters=10, cheb_lo_frac=0.25, cheb_safety=1.0):
    if isinstance(nelem, int):
        nelem = (nelem,) * dim
    return dict(dim=dim, nelem=tuple(nelem), order=order, warp_amp=warp_amp,
                mu_a=mu_a, mu_b=mu_b, mu_k=mu_k, hier=hier, n_hlevels=n_hlevels,
                smoother=smoother, nu_pre=nu_pre, nu_post=nu_post, omega=omega,
                arnoldi_iters=arnoldi_iters, cheb_lo_frac=cheb_lo_frac,
                cheb_safety=cheb_safety)


def mms2d_poisson(nelem=8, order=4, **kw):
    """2D unit square, mu = 1, Q_order on nelem^2 affine quads, h-MG V(2,2) Chebyshev:
    manufactured u = sin(pi x) sin(pi y), f = 2 pi^2 sin(pi x) sin(pi y)."""
    base = dict(hier="h", n_hlevels=3, smoother="cheb", nu_pre=2, nu_post=2)
    base.update(kw)
    return problem(2, nelem, order, **base)


def warped_var3d(nelem=16, order=4, hier="h", **kw):
    """3D warped cube (amp 0.1), mu = 1 + 1e3 sum cos^2(2 pi x_i), V(3,3) Chebyshev."""
    base = dict(warp_amp=0.1, mu_a=1.0, mu_b=1.0e3, mu_k=2.0, hier=hier,
                n_hlevels=3, smoother="cheb", nu_pre=3, nu_post=3)
    base.update(kw)
    return problem(3, nelem, order, **base)


def mesh_independence_problem(kind, E, order, smoother="cheb"):
    """Mesh-independence study (the paper's Sec. 4.4 setting): 2D fine mesh E x E (E a power of
    two >= 4), h-multigrid down to 2 x 2 elements at fixed order, V(3,3) point smoothing.
    kind "2d-const": unit square, mu = 1; "2d-var": warped square, mu = 1 + 1e6 sum cos^2(2 pi x_i)
    (the paper's amplitude for this study)."""
    levels = E.bit_length() - 1          # E = 2^(levels) -> levels-1 halvings reach 2 x 2
    base = dict(hier="h", n_hlevels=levels, smoother=smoother, nu_pre=3, nu_post=3)
    if kind == "2d-var":
        base.update(warp_amp=0.1, mu_a=1.0, mu_b=1e6, mu_k=2.0)
    return problem(2, E, order, **base)


def spectral_problem(kind, order, smoother="jacobi"):
    """Smoother / two-grid spectral study (the paper's Figs. 2-3 setting): 2D, 961 interior
    unknowns for every order (E = 32 / p elements per axis, p in {1, 2, 4, 8, 16}), two h-levels
    (the coarse grid solved exactly), V(3,3). kind "2d-const": unit square, mu = 1; "2d-var":
    warped square, mu = 1 + 1e6 sum cos^2(2 pi x_i)."""
    base = dict(hier="h", n_hlevels=2, smoother=smoother, nu_pre=3, nu_post=3)
    if kind == "2d-var":
        base.update(warp_amp=0.1, mu_a=1.0, mu_b=1e6, mu_k=2.0)
    return problem(2, 32 // order, order, **base)


def low_order_problem(prob, node_xyz, max_coarse=4000):
    """The low-order problem on the nodes of `prob` (Sec. 3.1.3): order 1 on order * nelem
    elements per axis, node coordinates node_xyz ([dim][N], prob's finest nodes), prob's
    coefficient; h-multigrid with Chebyshev V(3,3), halving the mesh while every axis stays even
    and the coarsest grid has more than max_coarse interior unknowns."""
    E = [e * prob["order"] for e in prob["nelem"]]
    cur, levels = list(E), 1
    while all(c % 2 == 0 and c >= 4 for c in cur) and int(np.prod([c - 1 for c in cur])) > max_coarse:
        cur = [c // 2 for c in cur]
        levels += 1
    out = problem(prob["dim"], tuple(E), 1, mu_a=prob.get("mu_a", 1.0), mu_b=prob.get("mu_b", 0.0),
                  mu_k=prob.get("mu_k", 2.0), hier="h", n_hlevels=levels, smoother="cheb")
    out["node_xyz"] = np.ascontiguousarray(node_xyz, dtype=np.float64)
    return out


# Seeds of the nodal right-hand sides for the 3D workloads.
SEED_WARPED_VAR3D = 2
SEED_PSWEEP3D = 3


def batched_problem(i, base_seed=4_000_000):
    """Solve i of the batched workload (parameters drawn from SplitMix64 with seed base+i):
    3D warped cube, elements per axis E in 2..12, order p in {2,4,6,8}, coefficient contrast
    10^k with k in 0..4: mu = 1 + (10^k - 1)/3 sum_i cos^2(2 pi x_i) (max/min = 10^k), p-multigrid
    down to p = 1 on the same mesh (whose dense coarsest system then has at most 11^3 unknowns),
    V(3,3) Chebyshev, FP32 V-cycle inside FP64 PCG. Returns (problem, rhs seed)."""
    z = splitmix64(base_seed + i, 3)
    E = 2 + int(z[0] % np.uint64(11))
    p = (2, 4, 6, 8)[int(z[1] % np.uint64(4))]
    k = int(z[2] % np.uint64(5))
    prob = problem(3, E, p, warp_amp=0.1, mu_a=1.0, mu_b=(10.0 ** k - 1.0) / 3.0, mu_k=2.0, hier="p",
                   n_hlevels=1, smoother="cheb", nu_pre=3, nu_post=3)
    prob["smooth_prec"] = "fp32"
    return prob, base_seed + i


def serving_request(i, base_seed=5):
    """Request i of the serving workload: Poisson arrivals (mean rate 2,000/s, exponential
    gaps from SplitMix64 seed base), dimension 2 or 3, target DOF log-uniform in [1e3, 2e6],
    order p uniform in 1..16; elements per axis E = round((N^(1/d) - 1)/p), moved to the nearest
    m * 2^k whose k halvings reach a p=1 grid of <= 729 nodes (m <= 8 in 3D, m <= 26 in 2D), which
    keeps the dense exact coarsest solve (O(n^3) FP64 setup) small,
    p-multigrid to p = 1 then those k h-levels; warped domain, mu = 1 + 1e3 sum cos^2(2 pi x_i),
    V(3,3) Chebyshev, FP32 V-cycle in FP64 PCG to 1e-8. Returns (problem, rhs seed, gap in s)."""
    u = uniform_pm1(base_seed, 5, start=5 * i)
    gap = -np.log(0.5 * (u[0] + 1.0) + 1e-300) / 2000.0
    d = 2 if u[1] < 0 else 3
    N = 10.0 ** (3.0 + (np.log10(2e6) - 3.0) * 0.5 * (u[2] + 1.0))
    p = 1 + min(15, int(8.0 * (u[3] + 1.0)))
    target = max(1.0, (N ** (1.0 / d) - 1.0) / p)
    mmax = 8 if d == 3 else 26
    best = None
    for k in range(0, 12):
        for m in range(1, mmax + 1):
            E = m << k
            if best is None or abs(E - target) < abs(best[0] - target):
                best = (E, k)
    E, k = best
    prob = problem(d, E, p, warp_amp=0.1, mu_a=1.0, mu_b=1e3, mu_k=2.0, hier="p", n_hlevels=k + 1,
                   smoother="cheb", nu_pre=3, nu_post=3)
    prob["smooth_prec"] = "fp32"
    return prob, base_seed * 1_000_000 + i, gap
