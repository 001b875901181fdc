"""Parity at the full ~2M-DOF p-sweep sizes (3D warped cube, mu = 1 + 1e3 sum cos^2(2 pi x_i)):
(64^3, p=2), (32^3, p=4), (16^3, p=8), (8^3, p=16), all 129^3 = 2,146,689 nodes, in the
launch configuration the solver uses. The oracle cannot assemble these operators, so:

* the FP64 apply is compared on sampled rows that the oracle evaluates one by one from
  the weak form (tolerance 1e-12 relative, as for the small cases);
* the p-multigrid PCG solves (FP64, and FP32 / FP16 / BF16 V-cycles) are checked by
  properties that hold at any size: FP64 residual <= 1e-8 recomputed with the FP64 operator,
  the mixed solves within +1 iteration (FP32, FP16) or +3 (BF16) of the FP64 one, and the
  solutions agreeing."""
import numpy as np
import pytest

import synth
from oracle import fem

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SWEEP = [(64, 2), (32, 4), (16, 8), (8, 16)]


@pytest.fixture(scope="module")
def hmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1402_5938_gb300 as pkg
    return pkg


@pytest.mark.parametrize("E,p", SWEEP, ids=lambda v: str(v))
def test_fullsize_apply_sampled_rows(hmg, E, p):
    prob = synth.warped_var3d(E, p, hier="p", smoother="jacobi")
    P = hmg.Problem(prob)
    N = P.ndof(0)
    assert N == 129 ** 3
    x = synth.uniform_pm1(synth.SEED_PSWEEP3D, N)
    y = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.apply(0, torch.from_numpy(x).to(DEV), y)
    torch.cuda.synchronize()
    d = fem.Discretization(3, E, p, warp_amp=0.1, mu_b=1e3)
    rng = np.random.default_rng(E)
    # interior rows, plus rows on element vertices / edges / faces (shared by 8/4/2 elements)
    rows = list(d.interior[rng.choice(d.n_interior, 6, replace=False)])
    c = 1 + p * (E // 2)
    rows += [(c * 129 + c) * 129 + c, (c * 129 + c) * 129 + c + 1, (c * 129 + c + 1) * 129 + c + 1, N - 130 * 129 - 2]
    rows = np.array(rows)
    ref = d.apply_rows(x, rows)
    got = y.cpu().numpy()[rows]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    P.close()


@pytest.mark.parametrize("E,p", SWEEP, ids=lambda v: str(v))
def test_fullsize_pmg_pcg_fp64_and_mixed(hmg, E, p):
    """FP64 and every mixed-precision form reach the FP64 tolerance at the sweep's full size."""
    prob = synth.warped_var3d(E, p, hier="p")
    P64 = hmg.Problem(prob)
    P32 = hmg.Problem(dict(prob, smooth_prec="fp32"))
    N = P64.ndof(0)
    f = torch.from_numpy(synth.nodal_field(synth.SEED_PSWEEP3D, N)).to(DEV)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P64.rhs(f, b)
    u64, u32, r = torch.zeros_like(b), torch.zeros_like(b), torch.zeros_like(b)
    st64, it64, _ = P64.solve("pcg", b, u64, rtol=1e-8, maxit=500)
    st32, it32, _ = P32.solve("pcg", b, u32, rtol=1e-8, maxit=500)
    assert st64 == 0 and st32 == 0
    assert it32 <= it64 + 1, (it32, it64)
    for u in (u64, u32):
        P64.apply(0, u, r)
        assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.05e-8
    assert float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64)) <= 1e-5
    P32.close()
    # the V-cycles with 16-bit factors and flexible PCG: FP16 keeps the FP64 count (+1), BF16's
    # 8-bit mantissa may cost up to 2 more iterations
    for prec, extra in (("fp16", 1), ("bf16", 2)):
        Pl = hmg.Problem(dict(prob, smooth_prec=prec))
        ul = torch.zeros_like(b)
        stl, itl, _ = Pl.solve("pcg", b, ul, rtol=1e-8, maxit=500)
        assert stl == 0 and itl <= it64 + extra, (prec, itl, it64)
        P64.apply(0, ul, r)
        assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.05e-8
        assert float(torch.linalg.norm(ul - u64) / torch.linalg.norm(u64)) <= 1e-5
        Pl.close()
    P64.close()
