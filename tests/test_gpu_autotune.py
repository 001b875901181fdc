"""Autotuner decisions persist across processes through HMG_AUTOTUNE_CACHE: the first process
times the apply variants and appends its choices to the file (each level's own decision and the
first decision of its size class), a second process reads them and times nothing (no autotune trace
lines), and both solve to the same result; a level of another element count in the same size class
reuses the class's decision without timing."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = r"""
import sys, torch
sys.path.insert(0, {root!r})
import synth
from paper_1402_5938_gb300 import Problem
P = Problem(dict(synth.warped_var3d(16, 2, hier="p"), smooth_prec="fp16"))
N = P.ndof(0)
b = torch.zeros(N, dtype=torch.float64, device="cuda")
P.rhs(torch.from_numpy(synth.nodal_field(5, N)).cuda(), b)
u = torch.zeros_like(b)
st, it, h = P.solve("pcg", b, u, rtol=1e-8, maxit=100)
print("RESULT", st, it, float(u.norm()))
"""


def _run(env):
    out = subprocess.run([sys.executable, "-c", SNIPPET.format(root=ROOT)], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = [ln for ln in out.stdout.splitlines() if ln.startswith("RESULT")][0].split()
    return res, [ln for ln in out.stderr.splitlines() if ln.startswith("hmg autotune:")]


def test_autotune_cache_file_round_trip(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache), HMG_TRACE="1")
    r1, tuned1 = _run(env)
    lines = cache.read_text().split("\n")
    entries = [ln.split() for ln in lines if ln.strip()]
    own = [e for e in entries if int(e[3]) > 0]          # a level's own decision
    cls = [e for e in entries if int(e[3]) < 0]          # the first decision of its size class
    assert tuned1 and len(own) == len(tuned1) and 0 < len(cls) <= len(own)
    assert all(len(e) == 6 and all(x.lstrip("-").isdigit() for x in e) for e in entries)
    r2, tuned2 = _run(env)
    assert tuned2 == []                           # every decision came from the file
    assert r1[1] == r2[1] == "0" and r1[2] == r2[2]
    assert abs(float(r1[3]) - float(r2[3])) <= 1e-8 * float(r1[3])
    # a mesh of 20^3 elements: each timed level (20^3 Q2 and Q1, 8,000 elements) is in the size
    # class [4096, 8192) of the 16^3 problem's level of equal order and takes its decision untimed
    r3 = subprocess.run([sys.executable, "-c", SNIPPET.replace("warped_var3d(16, 2,", "warped_var3d(20, 2,").format(root=ROOT)],
                        env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r3.returncode == 0, r3.stderr[-2000:]
    assert [ln for ln in r3.stderr.splitlines() if ln.startswith("hmg autotune:")] == []


HIGH_ORDER = r"""
import sys, torch
sys.path.insert(0, {root!r})
import numpy as np, synth
from paper_1402_5938_gb300 import Problem
prob = synth.problem(3, (3, 2, 2), {order}, warp_amp=0.1, mu_b=1e3, hier="p", n_hlevels=1)
P = Problem(dict(prob, smooth_prec={prec!r}))
N = P.ndof(0)
x = torch.from_numpy(synth.uniform_pm1(9, N)).cuda()
y = torch.zeros_like(x)
P.apply(0, x, y)
print("RESULT", P.level_variants(0)[0], P.level_variants(0)[1], float(y.norm()))
"""


@pytest.mark.parametrize("order", [14, 15, 16])
def test_autotune_times_every_variant_at_high_3d_orders(order):
    """A 3D level of order 14-16 large enough to be timed (12 elements, >= 32,768 Gauss points): setup
    times every variant it can run and succeeds (FP64 and the mixed V-cycle's operator); the chosen
    FP64 variant's apply equals variant 0's (pinned by the decision cache) to rounding."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import tempfile
    import __graft_entry__
    __graft_entry__.build()
    out = {}
    for pin in (None, 0):
        env = dict(os.environ)
        env.pop("HMG_AUTOTUNE_CACHE", None)
        if pin is not None:
            f = tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False)
            f.write(f"0 3 {order} 12 0 {pin}\n0 3 {order} 12 2 0\n")
            f.close()
            env["HMG_AUTOTUNE_CACHE"] = f.name
        r = subprocess.run([sys.executable, "-c", HIGH_ORDER.format(root=ROOT, order=order, prec="fp16")], env=env,
                           cwd=ROOT, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][0].split()
        out[pin] = (int(res[1]), int(res[2]), float(res[3]))
    assert out[0][0] == 0
    assert abs(out[None][2] - out[0][2]) <= 1e-12 * out[0][2]
