"""Autotuner decisions persist across processes through HMG_AUTOTUNE_CACHE: the first process
times the apply variants and appends its choices to the file, a second process reads them and
times nothing (no autotune trace lines), and both solve to the same result."""
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
    assert tuned1 and len(entries) == len(tuned1)
    assert all(len(e) == 6 and all(x.lstrip("-").isdigit() for x in e) for e in entries)
    r2, tuned2 = _run(env)
    assert tuned2 == []                           # every decision came from the file
    assert r1[1] == r2[1] == "0" and r1[2] == r2[2]
    assert abs(float(r1[3]) - float(r2[3])) <= 1e-8 * float(r1[3])
