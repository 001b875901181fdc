"""The tensor-core form of the 16-bit V-cycle operator (3D, orders 1-4; variant 3 of the reduced-
precision apply, built when HMG_TC16=1) against the FP64 oracle, pinned through the autotuner's
decision cache in a fresh process so that it runs on every level of each hierarchy.

y = A_k x (Sec. 2.1, Sec. 2.3's matrix-free apply) computed as two FP16 tensor-core products per
tile of 128 elements (X Phi, then V Phi^T, FP32 accumulation) around the pointwise G grad u. Per
output the error is bounded by (u_G + 4 u_16 + 1024 2^-24) S_i + 2^-20 T_i: u_G = 2^-11 (FP16
factors) or 2^-8 (BF16 factors) for the stored factor, one FP16 rounding each of x, Phi (twice) and
v = G grad u (u_16 = 2^-11), FP32 accumulation of up to ~400 terms, with S = sum_e |Phi|^T |G|
|Phi| |x|; T is S with |x_e| and |G_e| replaced by the element's largest entries and covers the
values that fall into FP16's subnormal range relative to an element's power-of-two scale.
Meshes: several tiles with a ragged last one, a single partial tile, all orders 1-4. The FP64 PCG
with this V-cycle (flexible beta) converges to 1e-8 with at most two iterations more than the
oracle's FP64 count."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from paper_1402_5938_gb300 import Problem
ref = np.load({ref!r}, allow_pickle=True)
cases = {cases!r}
prec = {prec!r}
for ci, prob in enumerate(cases):
    P = Problem(dict(prob, smooth_prec=prec))
    worst = 0.0
    variants = []
    for k in range(P.nlevels() - 1):
        x = ref[f"x_{{ci}}_{{k}}"]
        interior = ref[f"interior_{{ci}}_{{k}}"]
        want = ref[f"want_{{ci}}_{{k}}"]
        N = x.size
        for rep in range(2):   # twice: the second call starts from the first call's state
            y = torch.zeros(N, dtype=torch.float32, device="cuda")
            P.apply_f32(k, torch.from_numpy(x).float().cuda(), y)
            got = y.double().cpu().numpy()
            bd = np.ones(N, dtype=bool)
            bd[interior] = False
            assert np.all(got[bd] == 0.0)
            err = np.abs(got[interior] - want)
            worst = max(worst, float(np.max(err / ref[f"bound_{{prec}}_{{ci}}_{{k}}"])))
        variants.append(P.level_variants(k)[1])
    f = ref[f"f_{{ci}}"]
    b = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    P.rhs(torch.from_numpy(f).cuda(), b)
    u = torch.zeros_like(b)
    st, it, hist = P.solve("pcg", b, u, rtol=1e-8, maxit=200)
    print("RESULT", ci, worst, st, it, int(ref[f"it_{{ci}}"]), float(hist[-1] / hist[0]), ",".join(map(str, variants)))
    P.close()
"""

CASES = [
    dict(dim=3, nelem=(9, 9, 9), order=4, hier="p", n_hlevels=1),    # 729 elements: 6 tiles, the last ragged
    dict(dim=3, nelem=(5, 3, 2), order=4, hier="p", n_hlevels=1),    # 30 elements: one partial tile
    dict(dim=3, nelem=(6, 4, 4), order=3, hier="h", n_hlevels=2),
    dict(dim=3, nelem=(8, 8, 6), order=2, hier="h", n_hlevels=2),
    dict(dim=3, nelem=(4, 4, 6), order=1, hier="h", n_hlevels=2),
]
U_G = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
U16 = 2.0 ** -11


def _problems():
    import synth
    return [synth.problem(c["dim"], c["nelem"], c["order"], warp_amp=0.1, mu_b=1e3, hier=c["hier"],
                          n_hlevels=c["n_hlevels"]) for c in CASES]


@pytest.fixture(scope="module")
def oracle_ref(tmp_path_factory):
    import synth
    from oracle import multigrid
    from test_gpu_lowp import abs_bound_scale
    out = {}
    for ci, prob in enumerate(_problems()):
        H = multigrid.Hierarchy(prob)
        for k in range(len(H.levels) - 1):
            d = H.levels[k].disc
            x = synth.uniform_pm1(80 + k, d.N).astype(np.float32).astype(np.float64)
            x[d.boundary] = 0.0
            out[f"x_{ci}_{k}"] = x
            out[f"interior_{ci}_{k}"] = d.interior
            out[f"want_{ci}_{k}"] = H.levels[k].A @ x[d.interior]
            S = abs_bound_scale(d, x)[d.interior]
            T = abs_bound_scale(d, x, elem_max=True)[d.interior]
            for prec, ug in U_G.items():
                out[f"bound_{prec}_{ci}_{k}"] = (ug + 4 * U16 + 1024 * 2.0 ** -24) * S + 2.0 ** -20 * T + 1e-30
        f = synth.nodal_field(81, H.fine.disc.N)
        out[f"f_{ci}"] = f
        _, it_ref, _, ok = H.solve_pcg(H.fine.disc.rhs(f))
        assert ok
        out[f"it_{ci}"] = it_ref
    path = tmp_path_factory.mktemp("tc16") / "oracle.npz"
    np.savez(path, **out)
    return str(path)


def _pin_file(path, probs, kind):
    """Decision-cache lines: the tensor-core variant (3) on every 16-bit level, FP64 levels at 0."""
    from oracle import multigrid
    lines = set()
    for prob in probs:
        for E, p in multigrid.level_shapes(prob):
            ne = int(np.prod(E))
            lines.add(f"0 {prob['dim']} {p} {ne} 0 0")
            lines.add(f"0 {prob['dim']} {p} {ne} {kind} 3")
    path.write_text("\n".join(sorted(lines)) + "\n")


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc16_within_rounding_bound_on_every_level(tmp_path, oracle_ref, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    probs = _problems()
    cache = tmp_path / "tune.txt"
    _pin_file(cache, probs, {"fp16": 2, "bf16": 3}[prec])
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache), HMG_TC16="1")   # the form is built on request
    out = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, ref=oracle_ref, cases=probs, prec=prec)],
                         env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    rows = [ln.split() for ln in out.stdout.splitlines() if ln.startswith("RESULT")]
    assert len(rows) == len(probs), out.stdout[-2000:]
    for r in rows:
        worst, st, it, it_ref, rel = float(r[2]), int(r[3]), int(r[4]), int(r[5]), float(r[6])
        used = set(r[7].split(","))
        assert used == {"3"}, r
        assert worst <= 1.0, r
        assert st == 0 and rel <= 1e-8, r
        assert it_ref - 1 <= it <= it_ref + 2, r
