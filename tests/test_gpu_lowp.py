"""FP16 / BF16 V-cycle: the operator with 16-bit geometric factors against the FP64 oracle, and
FP64 PCG / MG-refinement solves whose V-cycle applies it (FP64 fine residual, inner products and
coarsest solve).

Tolerance of the 16-bit apply, from its arithmetic: the factors G are the only values rounded to
16 bits (unit roundoff u = 2^-11 for FP16, 2^-8 for BF16; the FP16 power-of-two scales are exact,
and a factor in FP16's subnormal range after scaling is off by at most 2^-25 of its element's
largest factor); x, the intermediates and the accumulation stay in FP32 (2^-24 per operation, a few
dozen operations per term). To first order |y16_i - y_i| <= u S_i + c 2^-24 S_i with
S = sum_e |K|^T |G| |K| |x| (absolute values of every factor), which the test evaluates with the
oracle's basis tables and geometry; it allows 2 u S_i + 64 2^-24 S_i."""
import numpy as np
import pytest

import synth
from oracle import fem

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U16 = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def hmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1402_5938_gb300 as pkg
    return pkg


def _t(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dt)


def abs_bound_scale(d, x_full, elem_max=False):
    """S = sum_e |K_e|^T |G_e| |K_e| |x_e| (all factors in absolute value), full-length. With
    elem_max, every |G_e| entry and every |x_e| entry is replaced by the element's largest one
    (the scale of errors that are absolute relative to an element's largest value)."""
    Phi, dPhi, W = d.basis_tables()
    el = np.arange(d.n_elem)
    xq, J, detJ = d.element_geometry(el, (Phi, dPhi, W))
    Jinv = np.linalg.inv(J)                                          # [e,q,k,i] = dxi_k / dx_i
    c = W[None, :] * np.abs(detJ) * d.mu(xq.reshape(-1, d.dim)).reshape(detJ.shape)
    G = c[:, :, None, None] * np.einsum("eqki,eqli->eqkl", Jinv, Jinv)
    nodes = d.element_nodes(el)
    X = np.abs(x_full)[nodes]                                        # (e, a)
    G = np.abs(G)
    if elem_max:
        X = np.broadcast_to(X.max(axis=1, keepdims=True), X.shape)
        G = np.broadcast_to(G.max(axis=(1, 2, 3), keepdims=True), G.shape)
    U = np.stack([X @ np.abs(dPhi[k]).T for k in range(d.dim)], axis=-1)   # (e, q, k)
    V = np.einsum("eqkl,eqk->eql", G, U)
    Se = sum(V[:, :, l] @ np.abs(dPhi[l]) for l in range(d.dim))    # (e, a)
    S = np.zeros(d.N)
    np.add.at(S, nodes.ravel(), Se.ravel())
    return S


CASES = [dict(dim=3, nelem=(3, 2, 2), order=p) for p in (1, 2, 3, 4, 5, 6, 7)] + [
    dict(dim=3, nelem=(5, 3, 2), order=4),      # ragged last warp group (EW = 3)
    dict(dim=3, nelem=(4, 4, 3), order=2),
    dict(dim=2, nelem=(7, 5), order=3),
    dict(dim=2, nelem=(9, 4), order=5),
    dict(dim=2, nelem=(3, 3), order=7),
    dict(dim=2, nelem=(6, 6), order=1),
]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-{c['nelem']}-p{c['order']}")
def test_lowp_apply_within_rounding_bound(hmg, case, prec):
    mu_b = 1e3
    prob = dict(synth.problem(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_b=mu_b, n_hlevels=1,
                              smoother="jacobi"), smooth_prec=prec)
    P = hmg.Problem(prob)
    d = fem.Discretization(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_b=mu_b)
    x = synth.uniform_pm1(21, d.N)
    y = torch.zeros(d.N, dtype=torch.float32, device=DEV)
    P.apply_f32(0, _t(x, torch.float32), y)
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    xr = x.astype(np.float32).astype(np.float64)
    xr[d.boundary] = 0.0
    ref = d.to_full(d.stiffness() @ xr[d.interior])
    S = abs_bound_scale(d, xr)
    err = np.abs(y - ref)[d.interior]
    bound = (2 * U16[prec] + 64 * 2.0 ** -24) * S[d.interior] + 1e-30
    assert np.all(err <= bound), float(np.max(err / S[d.interior]))
    # and it is a real 16-bit result, not an FP32 one in disguise: the error is well above FP32 rounding
    assert np.max(err / S[d.interior]) > 2.0 ** -20
    assert np.all(y[d.boundary] == 0.0)
    P.close()


def test_lowp_fp16_scaling_keeps_tiny_and_huge_inputs(hmg):
    """FP16 factors carry a power-of-two scale per element and the vectors stay FP32: y(c x) = c y(x)
    for c = 2^-40 and 2^40 (scaling by a power of two is exact in every operation), where a 16-bit
    vector operand would flush to zero or overflow."""
    prob = dict(synth.problem(3, (3, 2, 2), 4, warp_amp=0.1, mu_b=1e3, n_hlevels=1, smoother="jacobi"),
                smooth_prec="fp16")
    P = hmg.Problem(prob)
    N = P.ndof(0)
    x = _t(synth.uniform_pm1(22, N), torch.float32)
    ys = []
    for c in (1.0, 2.0 ** -40, 2.0 ** 40):
        y = torch.zeros(N, dtype=torch.float32, device=DEV)
        P.apply_f32(0, x * c, y)
        ys.append(y.double().cpu().numpy() / c)
    assert np.all(np.isfinite(ys[1])) and np.all(np.isfinite(ys[2]))
    top = np.abs(ys[0]).max()
    # exact scaling; only the FP32 atomic scatter order may differ between launches
    assert np.abs(ys[1] - ys[0]).max() <= 1e-6 * top and np.abs(ys[2] - ys[0]).max() <= 1e-6 * top
    P.close()


SOLVES = [
    (synth.warped_var3d(8, 4, hier="p"), "pcg"),
    (synth.warped_var3d(8, 2, hier="h"), "pcg"),
    (synth.warped_var3d(4, 4, hier="p"), "mg"),
    (synth.problem(2, 16, 6, warp_amp=0.1, mu_b=1e3, hier="p"), "pcg"),
    (synth.problem(3, 4, 8, warp_amp=0.1, mu_b=1e3, hier="p"), "pcg"),
]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("prob,mode", SOLVES, ids=lambda c: str(c)[:60])
def test_lowp_solve_reaches_fp64_accuracy(hmg, prob, mode, prec):
    """The 16-bit V-cycle inside FP64 PCG (flexible beta) or MG refinement reaches the FP64
    tolerance: true FP64 residual <= 1e-8 relative; iteration count within one of the FP64 solve's
    (FP16) or at most two more (BF16); and, where the oracle's interior system is small enough to
    factor, the solution within the bound the residual gives against the oracle's exact solution:
    ||u - u*||_2 <= ||b - A u||_2 / lambda_min(A), A symmetric positive definite."""
    import scipy.sparse.linalg as spla
    from oracle import fem
    P64 = hmg.Problem(prob)
    Pl = hmg.Problem(dict(prob, smooth_prec=prec))
    N = P64.ndof(0)
    fn = synth.nodal_field(31, N)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P64.rhs(_t(fn), b)
    u64 = torch.zeros_like(b)
    ul = torch.zeros_like(b)
    st64, it64, _ = P64.solve(mode, b, u64, rtol=1e-8, maxit=400)
    st, it, h = Pl.solve(mode, b, ul, rtol=1e-8, maxit=400)
    assert st64 == 0 and st == 0
    r = torch.zeros_like(b)
    P64.apply(0, ul, r)
    res = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
    assert res <= 1.05e-8
    assert it64 - 1 <= it <= it64 + (1 if prec == "fp16" else 2), (it, it64)
    d = fem.Discretization(prob["dim"], prob["nelem"], prob["order"], warp_amp=prob["warp_amp"],
                           mu_a=prob["mu_a"], mu_b=prob["mu_b"], mu_k=prob["mu_k"])
    if d.n_interior <= 12000:
        A = d.stiffness().tocsc()
        bi = d.rhs(fn)
        ustar = spla.spsolve(A, bi)
        lam_min = float(spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
        ui = ul.cpu().numpy()[d.interior]
        err = float(np.linalg.norm(ui - ustar))
        bound = float(np.linalg.norm(bi - A @ ui)) / lam_min
        assert err <= 1.0001 * bound + 1e-14 * np.linalg.norm(ustar), (err, bound)
        print(f"{prec} {mode}: |u - u*| {err:.2e} <= {bound:.2e}")
    print(f"{prec} {mode}: iterations {it} (FP64 {it64}), true residual {res:.2e}")
    P64.close()
    Pl.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_lowp_graph_and_batched_equal_host_loop(hmg, prec):
    """The flexible-beta PCG gives the same iterations through the device-side graph loop, the
    host loop and a lockstep batch."""
    prob = dict(synth.warped_var3d(8, 4, hier="p"), smooth_prec=prec)
    Pg = hmg.Problem(dict(prob, solve_graph=1))
    Ph = hmg.Problem(dict(prob, solve_graph=0))
    N = Pg.ndof(0)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    Pg.rhs(_t(synth.nodal_field(32, N)), b)
    ug, uh, ub = (torch.zeros_like(b) for _ in range(3))
    stg, itg, hg = Pg.solve("pcg", b, ug, rtol=1e-8, maxit=200)
    sth, ith, hh = Ph.solve("pcg", b, uh, rtol=1e-8, maxit=200)
    sts, its, _ = hmg.solve_batched([Pg], "pcg", [b], [ub], rtol=1e-8, maxit=200)
    assert stg == sth == sts[0] == 0
    assert abs(itg - ith) <= 1 and abs(its[0] - ith) <= 1
    assert float(torch.linalg.norm(ug - uh) / torch.linalg.norm(uh)) < 1e-6
    Pg.close()
    Ph.close()


def test_lowp_register_variant_within_rounding_bound(tmp_path):
    """The apply with each thread's 16-bit factors loaded into registers first (variant 1, small
    orders, picked by the autotuner where faster) passes the same rounding-bound parity: pinned for
    every case through the decision cache, in a fresh process."""
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path / "tune16.txt"
    lines = []
    for case in CASES:
        ne = int(np.prod(case["nelem"]))
        for kind in (2, 3):                      # HMG_PREC_FP16, HMG_PREC_BF16
            lines.append(f"0 {case['dim']} {case['order']} {ne} {kind} 1")
    cache.write_text("\n".join(lines) + "\n")
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(root, "tests", "test_gpu_lowp.py"), "-k", "apply_within_rounding_bound"],
                         env=env, cwd=root, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stdout[-3000:]
