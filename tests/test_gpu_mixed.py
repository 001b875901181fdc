"""Mixed precision: the FP32 operator of the V-cycle against the FP64 oracle, and FP64
PCG / MG-refinement solves whose V-cycle runs in FP32 (FP64 fine residual, inner products
and coarsest solve).

FP32 tolerance: the apply evaluates each output through 4d contraction stages of N-term
sums plus the pointwise G product, each rounding with unit roundoff u = 2^-24 = 6e-8;
bounding the accumulated relative error by (4 d N + 16) u relative to the largest output
entry gives 1.0e-5 for d = 3, N = 17 and less for lower orders. The tests use 2e-5."""
import numpy as np
import pytest

import synth
from oracle import fem, multigrid

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


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


CASES = [
    dict(dim=3, nelem=(5, 3, 2), order=2),
    dict(dim=3, nelem=(3, 2, 2), order=4),
    dict(dim=3, nelem=(4, 4, 4), order=1),
    dict(dim=3, nelem=(2, 2, 1), order=8),
    dict(dim=3, nelem=(1, 1, 1), order=16),
    dict(dim=2, nelem=(7, 5), order=3),
    dict(dim=2, nelem=(3, 2), order=16),
    dict(dim=2, nelem=(20, 16), order=1),   # 64 elements per warp group in the warp-group form
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-{c['nelem']}-p{c['order']}")
def test_fp32_apply_matches_oracle(hmg, case):
    prob = dict(synth.problem(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_b=1e3, n_hlevels=1,
                              smoother="jacobi"), smooth_prec="fp32")
    P = hmg.Problem(prob)
    d = fem.Discretization(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_b=1e3)
    x = synth.uniform_pm1(12, d.N)
    y = torch.zeros(d.N, dtype=torch.float32, device=DEV)
    P.apply_f32(0, _t(x, torch.float32), y)
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    xr = x.astype(np.float32).astype(np.float64)          # the FP32 input the kernel saw
    if (case["order"] + 1) ** case["dim"] <= 1000:
        ref = d.stiffness() @ xr[d.interior]
        got = y[d.interior]
    else:
        rows = d.interior[np.random.default_rng(4).choice(d.n_interior, 16, replace=False)]
        ref = d.apply_rows(xr, rows)
        got = y[rows]
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    assert np.all(y[d.boundary] == 0.0)
    P.close()


SOLVES = [
    (synth.warped_var3d(4, 4, hier="h"), "pcg"),
    (synth.warped_var3d(4, 4, hier="p"), "pcg"),
    (synth.warped_var3d(4, 2, hier="p"), "mg"),
    (synth.mms2d_poisson(8, 4), "mg"),
    (synth.problem(2, 8, 8, warp_amp=0.1, mu_b=1e3, hier="p"), "pcg"),
]


@pytest.mark.parametrize("prob,mode", SOLVES, ids=lambda c: str(c)[:60])
def test_mixed_solve_reaches_fp64_accuracy(hmg, prob, mode):
    P64 = hmg.Problem(prob)
    P32 = hmg.Problem(dict(prob, smooth_prec="fp32"))
    N = P64.ndof(0)
    f = _t(synth.nodal_field(9, N))
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P64.rhs(f, b)
    u64 = torch.zeros_like(b)
    u32 = torch.zeros_like(b)
    st64, it64, h64 = P64.solve(mode, b, u64, rtol=1e-8, maxit=300)
    st32, it32, h32 = P32.solve(mode, b, u32, rtol=1e-8, maxit=300)
    assert st64 == 0 and st32 == 0
    assert it32 <= it64 + 1, (it32, it64)
    # FP64 residual of the mixed solution, by the FP64 operator, and agreement with the FP64
    # solution to the accuracy both reached
    r = torch.zeros_like(b)
    P64.apply(0, u32, r)
    res = torch.linalg.norm(b - r) / torch.linalg.norm(b)
    assert float(res) <= 1e-8
    err = float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64))
    assert err <= 1e-5, err
    P64.close()
    P32.close()


def test_mixed_vcycle_close_to_fp64_vcycle(hmg):
    prob = synth.warped_var3d(4, 4, hier="p")
    P64 = hmg.Problem(prob)
    P32 = hmg.Problem(dict(prob, smooth_prec="fp32"))
    H = multigrid.Hierarchy(prob)
    d = H.fine.disc
    r = synth.uniform_pm1(33, d.N)
    r[d.boundary] = 0
    z64 = torch.zeros(d.N, dtype=torch.float64, device=DEV)
    z32 = torch.zeros_like(z64)
    P64.vcycle(_t(r), z64)
    P32.vcycle(_t(r), z32)
    ref = H.vcycle(r[d.interior])
    e64 = np.abs(z64.cpu().numpy()[d.interior] - ref).max() / np.abs(ref).max()
    e32 = np.abs(z32.cpu().numpy()[d.interior] - ref).max() / np.abs(ref).max()
    assert e64 < 1e-10
    assert e32 < 1e-4          # FP32 V-cycle: rounding of ~30 operator applications
    P64.close()
    P32.close()


def test_fp32_register_variant_matches_oracle(tmp_path):
    """The FP32 apply with each thread's factors loaded into registers first (variant 1, small
    orders, picked by the autotuner where faster) passes the same parity as variant 0: pinned for
    every case through the decision cache, in a fresh process."""
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lines = []
    for case in CASES:
        ne = int(np.prod(case["nelem"]))
        lines.append(f"0 {case['dim']} {case['order']} {ne} 1 1")   # kind 1 = HMG_PREC_FP32
    cache = tmp_path / "tune32.txt"
    cache.write_text("\n".join(lines) + "\n")
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(root, "tests", "test_gpu_mixed.py"), "-k", "fp32_apply_matches_oracle"],
                         env=env, cwd=root, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stdout[-3000:]
