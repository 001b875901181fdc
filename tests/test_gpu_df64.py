"""GPU: the finest level's FP64 operator in double-float arithmetic (hmg_desc.fp64_arith =
HMG_ARITH_DF64), against the FP64 oracle.

Tolerance of the apply, derived from the arithmetic: every double-float operation rounds with a
unit of 2^-46 (about 1.4e-14) relative to the magnitudes it combines, and the FP64 inputs (x, the
geometric factors) are split with a relative error below 2^-48. The sum-factorized apply chains
12 line contractions of at most N <= 9 terms, a pointwise product and the element scatter, so the
accumulated error stays below a few hundred units relative to the largest entry: 1e-11 relative
(max-norm over interior nodes, relative to the largest reference entry), against about 1e-7 for
FP32 arithmetic. Solves: the same iteration count (+-1) as with the FP64 operator, and the true
FP64 residual of the solution (the native FP64 operator) within 1.1e-8 relative.
"""
import numpy as np
import pytest

import synth
from oracle import fem

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KDF = 7  # the double-float variant of the FP64 operator


@pytest.fixture(scope="module")
def hmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1402_5938_gb300 as pkg
    return pkg


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _z(n):
    return torch.zeros(n, dtype=torch.float64, device=DEV)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    dict(dim=3, nelem=(5, 3, 2), order=2),
    dict(dim=3, nelem=(3, 2, 2), order=4),
    dict(dim=3, nelem=(4, 4, 4), order=1),
    dict(dim=3, nelem=(2, 2, 1), order=8),
    dict(dim=3, nelem=(3, 2, 1), order=5),
    dict(dim=2, nelem=(7, 5), order=3),
    dict(dim=2, nelem=(13, 11), order=6),
    dict(dim=2, nelem=(5, 4), order=8),
]


def _prob(case):
    prob = synth.problem(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_a=1.0, mu_b=1e3, mu_k=2.0,
                         n_hlevels=1, smoother="jacobi")
    return dict(prob, fp64_arith="df64")


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-{c['nelem']}-p{c['order']}")
def test_df64_apply_matches_oracle(hmg, case):
    P = hmg.Problem(_prob(case))
    assert P.level_variants(0)[0] == KDF
    d = fem.Discretization(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_a=1.0, mu_b=1e3)
    x = synth.uniform_pm1(11, d.N)
    ys = []
    for _ in range(2):  # the same result on a second call (no state carried between calls)
        y = _z(d.N)
        P.apply(0, _t(x), y)
        torch.cuda.synchronize()
        ys.append(y.cpu().numpy())
    y = ys[0]
    assert np.array_equal(ys[0], ys[1]) or _rel(ys[1], ys[0]) < 1e-13  # atomics: summation order varies
    assert np.all(y[d.boundary] == 0.0)
    ref = d.stiffness() @ x[d.interior]
    err = _rel(y[d.interior], ref)
    assert err < 1e-11, err
    P.close()


def test_df64_falls_back_to_fp64_above_order_8(hmg):
    case = dict(dim=2, nelem=(3, 2), order=10)
    P = hmg.Problem(_prob(case))
    assert P.level_variants(0)[0] != KDF
    d = fem.Discretization(2, (3, 2), 10, warp_amp=0.1, mu_a=1.0, mu_b=1e3)
    x = synth.uniform_pm1(12, d.N)
    y = _z(d.N)
    P.apply(0, _t(x), y)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy()[d.interior], d.stiffness() @ x[d.interior]) < 1e-12
    P.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_df64_pcg_reaches_fp64_residual(hmg, prec):
    prob = dict(synth.warped_var3d(nelem=8, order=4, hier="p"), smooth_prec=prec)
    P64 = hmg.Problem(prob)
    Pdf = hmg.Problem(dict(prob, fp64_arith="df64"))
    assert Pdf.level_variants(0)[0] == KDF and P64.level_variants(0)[0] != KDF
    N = P64.ndof(0)
    b = _z(N)
    P64.rhs(_t(synth.nodal_field(synth.SEED_WARPED_VAR3D, N)), b)
    u64, udf = _z(N), _z(N)
    st64, it64, _ = P64.solve("pcg", b, u64, rtol=1e-8, maxit=200)
    stdf, itdf, _ = Pdf.solve("pcg", b, udf, rtol=1e-8, maxit=200)
    assert st64 == 0 and stdf == 0
    assert abs(itdf - it64) <= 1, (itdf, it64)
    r = _z(N)
    P64.apply(0, udf, r)  # native FP64 operator
    rel = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
    assert rel <= 1.1e-8, rel
    P64.close()
    Pdf.close()
