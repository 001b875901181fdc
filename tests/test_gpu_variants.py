"""Every block-shape variant of the operator apply against the FP64 oracle, pinned through the
autotuner's decision cache (HMG_AUTOTUNE_CACHE) in a fresh process so that the variant runs on
every level of the hierarchy, tiny levels included.

FP64 sum factorization, variants 0-3 (3 stages the geometric factors by TMA) and the FP64 pencil
form with even/odd line products, variants 5 (factors at their use) and 6 (one phase ahead), which
levels of order 7 and higher offer (6 up to order 8; variant 0 pinned below order 7, variant 5
above order 8): every level's operator within 1e-12 relative of the oracle's assembled A (Sec. 2.1,
Sec. 2.3's matrix-free apply), PCG iteration counts within +-1 of the oracle's (Algorithm 1); at the
16^3 Q4 size of the single-solve workload, variants 2 and 3 on sampled rows of the oracle's weak
form at element vertices, edges, faces and interiors. The V-cycle operator (pencil form) with FP32 factors, variants
0-2 (when a thread loads its factors): within 2e-5 of the oracle (the FP32 rounding bound of
the operator's chain of contractions), and the FP64 PCG with the FP32 V-cycle within +-1 iteration of
the oracle. With FP16 / BF16 factors, variants 0-2: every output within the rounding bound of the
16-bit factors."""
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
        if prec == "fp64":
            y = torch.zeros(N, dtype=torch.float64, device="cuda")
            P.apply(k, torch.from_numpy(x).cuda(), y)
        else:
            y = torch.zeros(N, dtype=torch.float32, device="cuda")
            P.apply_f32(k, torch.from_numpy(x).float().cuda(), y)
        got = y.double().cpu().numpy()
        bd = np.ones(N, dtype=bool)
        bd[interior] = False
        assert np.all(got[bd] == 0.0)
        err = np.abs(got[interior] - want)
        if prec in ("fp16", "bf16"):     # error over the rounding bound (k + 1) u S
            worst = max(worst, float(np.max(err / ref[f"bound_{{prec}}_{{ci}}_{{k}}"])))
        else:
            worst = max(worst, float(err.max() / np.abs(want).max()))
        variants.append(P.level_variants(k)[0 if prec == "fp64" else 1])
    f = ref[f"f_{{ci}}"]
    b = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    P.rhs(torch.from_numpy(f).cuda(), b)
    u = torch.zeros_like(b)
    st, it, hist = P.solve("pcg", b, u, rtol=1e-8, maxit=200)
    print("RESULT", ci, worst, st, it, int(ref[f"it_{{ci}}"]), float(hist[-1] / hist[0]), ",".join(map(str, variants)))
    P.close()
"""

# 2D and 3D, orders 2/4/8/16 on their hierarchies; the 3D 8^3 Q4 fine level (64,000 Gauss
# points) and the 2D 24^2 Q4 one are above the autotuner's size threshold
CASES = [
    dict(dim=3, nelem=(8, 8, 8), order=4, hier="p", n_hlevels=2),
    dict(dim=3, nelem=(4, 2, 2), order=2, hier="h", n_hlevels=2),
    dict(dim=3, nelem=(2, 2, 2), order=8, hier="p", n_hlevels=1),
    dict(dim=2, nelem=(24, 24), order=4, hier="p", n_hlevels=2),
    dict(dim=2, nelem=(3, 2), order=16, hier="p", n_hlevels=1),
    dict(dim=2, nelem=(6, 4), order=8, hier="h", n_hlevels=2),
]
U16 = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def _problems():
    import synth
    return [synth.problem(c["dim"], c["nelem"], c["order"], warp_amp=0.1, mu_b=1e3, hier=c["hier"],
                          n_hlevels=c["n_hlevels"]) for c in CASES]


@pytest.fixture(scope="module")
def oracle_ref(tmp_path_factory):
    """Oracle results of every case, computed once: per level a seeded x (boundary entries 0; in
    FP32-representable values), A x by the assembled oracle operator, and for the 16-bit
    operators the bound (2 u + 64 2^-24) S_i with S = sum_e |K|^T |G| |K| |x| (the bound of
    tests/test_gpu_lowp.py); the load vector's nodal f and the oracle's PCG iteration count."""
    import synth
    from oracle import multigrid
    from test_gpu_lowp import abs_bound_scale
    out = {}
    for ci, prob in enumerate(_problems()):
        H = multigrid.Hierarchy(prob)
        for k in range(len(H.levels) - 1):
            d = H.levels[k].disc
            x = synth.uniform_pm1(70 + k, d.N).astype(np.float32).astype(np.float64)
            x[d.boundary] = 0.0
            out[f"x_{ci}_{k}"] = x
            out[f"interior_{ci}_{k}"] = d.interior
            out[f"want_{ci}_{k}"] = H.levels[k].A @ x[d.interior]
            S = abs_bound_scale(d, x)[d.interior]
            for prec, u in U16.items():
                out[f"bound_{prec}_{ci}_{k}"] = (2 * u + 64 * 2.0 ** -24) * S + 1e-30
        f = synth.nodal_field(71, H.fine.disc.N)
        out[f"f_{ci}"] = f
        _, it_ref, _, ok = H.solve_pcg(H.fine.disc.rhs(f))
        assert ok
        out[f"it_{ci}"] = it_ref
    path = tmp_path_factory.mktemp("variants") / "oracle.npz"
    np.savez(path, **out)
    return str(path)


def _fp64_pin(variant, p, dim):
    """The FP64 variant pinned on a level of order p: the pencil variants exist from order 7 on
    (not at 3D orders 14-15, whose tile exceeds shared memory), variant 6 up to order 8."""
    n = p + 1
    if variant not in (5, 6):
        return variant
    if n < 8 or (dim == 3 and n in (15, 16)):
        return 0
    return 5 if variant == 6 and n > 9 else variant


def _pin_file(path, probs, kind, variant):
    """Cache lines 'device dim order elements kind variant' for every level of every problem;
    FP64 levels of mixed problems keep variant 0."""
    from oracle import multigrid
    lines = set()
    for prob in probs:
        for E, p in multigrid.level_shapes(prob):
            ne = int(np.prod(E))
            lines.add(f"0 {prob['dim']} {p} {ne} 0 {_fp64_pin(variant, p, prob['dim']) if kind == 0 else 0}")
            if kind:
                lines.add(f"0 {prob['dim']} {p} {ne} {kind} {variant}")
    path.write_text("\n".join(sorted(lines)) + "\n")


def _run(tmp_path, ref, prec, kind, variant):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    probs = _problems()
    cache = tmp_path / "tune.txt"
    _pin_file(cache, probs, kind, variant)
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, ref=ref, cases=probs, prec=prec)], env=env,
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    rows = [ln.split() for ln in out.stdout.splitlines() if ln.startswith("RESULT")]
    assert len(rows) == len(probs)
    res = []
    for r in rows:
        res.append(dict(ci=int(r[1]), worst=float(r[2]), st=int(r[3]), it=int(r[4]), it_ref=int(r[5]),
                        rel=float(r[6]), used=set(r[7].split(","))))
    return res


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 5, 6])
def test_fp64_variant_matches_oracle_on_every_level(tmp_path, oracle_ref, variant):
    from oracle import multigrid
    probs = _problems()
    for r in _run(tmp_path, oracle_ref, "fp64", 0, variant):
        shapes = multigrid.level_shapes(probs[r["ci"]])[:-1]
        assert r["used"] == {str(_fp64_pin(variant, p, probs[r["ci"]]["dim"])) for _, p in shapes}, r
        assert r["worst"] <= 1e-12, r
        assert r["st"] == 0 and r["rel"] <= 1e-8 and abs(r["it"] - r["it_ref"]) <= 1, r


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_fp32_variant_matches_oracle_on_every_level(tmp_path, oracle_ref, variant):
    for r in _run(tmp_path, oracle_ref, "fp32", 1, variant):
        assert r["used"] == {str(variant)}, r
        assert r["worst"] <= 2e-5, r
        assert r["st"] == 0 and r["rel"] <= 1e-8 and abs(r["it"] - r["it_ref"]) <= 1, r


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_variant_within_rounding_bound_on_every_level(tmp_path, oracle_ref, prec, variant):
    """The FP64 PCG with this V-cycle (flexible beta) converges to 1e-8 within one iteration of the
    oracle's FP64 count (FP16) or two (BF16)."""
    for r in _run(tmp_path, oracle_ref, prec, {"fp16": 2, "bf16": 3}[prec], variant):
        assert r["used"] == {str(variant)}, r
        assert r["worst"] <= 1.0, r
        assert r["st"] == 0 and r["rel"] <= 1e-8, r
        assert r["it_ref"] - 1 <= r["it"] <= r["it_ref"] + (1 if prec == "fp16" else 2), r


ROWS_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import synth
from oracle import fem
from paper_1402_5938_gb300 import Problem
prob = synth.warped_var3d(16, 4, hier="p")
P = Problem(prob)
d = fem.Discretization(3, 16, 4, warp_amp=prob["warp_amp"], mu_a=prob["mu_a"], mu_b=prob["mu_b"], mu_k=prob["mu_k"])
x = synth.uniform_pm1(72, d.N)
y = torch.zeros(d.N, dtype=torch.float64, device="cuda")
P.apply(0, torch.from_numpy(x).cuda(), y)
y = y.cpu().numpy()
# rows at element vertices, on element edges, on element faces and inside elements (node index
# along an axis: multiple of p = element boundary), near the domain boundary and in the middle
rng = np.random.default_rng(73)
idx = d.node_axis_index
on = [(idx[a] % 4 == 0) for a in range(3)]
nb = on[0].astype(int) + on[1] + on[2]
rows = []
for want in (3, 2, 1, 0):
    cand = np.flatnonzero((nb == want) & ~d.boundary)
    rows += list(rng.choice(cand, 8, replace=False))
rows += [int(np.ravel_multi_index((1, 1, 1), d.Nn[::-1])), int(np.ravel_multi_index((32, 32, 32), d.Nn[::-1]))]
rows = np.array(rows)
ref = d.apply_rows(x, rows)
print("RESULT", float(np.abs(y[rows] - ref).max() / np.abs(ref).max()), P.level_variants(0)[0])
"""


@pytest.mark.parametrize("variant", [2, 3])
def test_fp64_variant_at_16cube_q4_sampled_rows(tmp_path, variant):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    cache = tmp_path / "tune.txt"
    cache.write_text(f"0 3 4 4096 0 {variant}\n")
    env = dict(os.environ, HMG_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", ROWS_SCRIPT.format(root=ROOT)], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    r = [ln.split() for ln in out.stdout.splitlines() if ln.startswith("RESULT")][0]
    assert int(r[2]) == variant
    assert float(r[1]) <= 1e-12, r
