"""The FP64 dense-element-matrix apply (variant 4, offered to the autotuner for orders 1 and 2)
against the FP64 oracle: pinned through the decision cache in a fresh process, every level's
operator (1e-12 relative, as for the sum-factorized apply) and PCG iteration counts (+-1)."""
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
import synth
from oracle import multigrid
from paper_1402_5938_gb300 import Problem
prob = {prob!r}
P = Problem(prob)
H = multigrid.Hierarchy(prob)
worst = 0.0
for k in range(P.nlevels() - 1):
    d = H.levels[k].disc
    x = synth.uniform_pm1(60 + k, d.N)
    x[d.boundary] = 0.0
    y = torch.zeros(d.N, dtype=torch.float64, device="cuda")
    P.apply(k, torch.from_numpy(x).cuda(), y)
    want = H.levels[k].A @ x[d.interior]
    worst = max(worst, float(np.abs(y.cpu().numpy()[d.interior] - want).max() / np.abs(want).max()))
d = H.fine.disc
f = synth.nodal_field(61, d.N)
b = torch.zeros(d.N, dtype=torch.float64, device="cuda")
P.rhs(torch.from_numpy(f).cuda(), b)
u = torch.zeros_like(b)
st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=200)
_, it_ref, _, ok = H.solve_pcg(d.rhs(f))
print("RESULT", worst, st, it, it_ref, ok)
"""

CASES = [dict(dim=3, nelem=(6, 4, 4), order=2, hier="p"), dict(dim=3, nelem=(8, 8, 4), order=1, hier="h"),
         dict(dim=2, nelem=(12, 8), order=2, hier="p"), dict(dim=2, nelem=(16, 16), order=1, hier="h")]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-p{c['order']}-{c['hier']}")
def test_dense_apply_matches_oracle(tmp_path, case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import synth
    prob = synth.problem(case["dim"], case["nelem"], case["order"], warp_amp=0.1, mu_b=1e3, hier=case["hier"],
                         n_hlevels=2)
    # pin variant 4 for every level shape of this hierarchy (kind 0 = FP64)
    from oracle import multigrid
    lines = []
    for E, p in multigrid.level_shapes(prob):
        lines.append(f"0 {case['dim']} {p} {int(np.prod(E))} 0 4")
    cache = tmp_path / "tune.txt"
    cache.write_text("\n".join(lines) + "\n")
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, prob=prob)], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = [ln for ln in out.stdout.splitlines() if ln.startswith("RESULT")][0].split()
    worst, st, it, it_ref, ok = float(res[1]), int(res[2]), int(res[3]), int(res[4]), res[5] == "True"
    assert worst <= 1e-12, worst
    assert st == 0 and ok and abs(it - it_ref) <= 1
