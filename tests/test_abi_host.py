"""CPU-only checks of the C ABI library: it loads, exports every function that
include/hmg.h declares, and its host-side logic (1D tables, Ritz-value eigen step,
descriptor defaults) is right. No device is touched."""
import os
import re

import numpy as np
import pytest

from oracle import basis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hmg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1402_5938_gb300 as pkg
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "hmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(hmg):
    lib = hmg.lib()
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("p", range(1, 17))
def test_host_tables_match_oracle(hmg, p):
    r, g, w = hmg.host_basis(p)
    assert np.abs(r - basis.gll_nodes(p)).max() < 1e-15
    gx, gw = basis.gauss_rule(p + 1)
    assert np.abs(g - gx).max() < 1e-15
    assert np.abs(w - gw).max() < 1e-15


def test_hessenberg_eigen_step(hmg):
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 5, 10):
        for _ in range(20):
            H = np.triu(rng.standard_normal((m, m)), -1)
            ref = np.linalg.eigvals(H).real.max()
            assert abs(hmg.host_hessenberg_max_real_eig(H) - ref) < 1e-10 * max(1, abs(ref))
    # a Ritz matrix of a symmetric positive operator (real spectrum)
    A = rng.standard_normal((10, 10))
    A = A @ A.T
    Q, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    import scipy.linalg as sla
    Hs, _ = sla.hessenberg(A, calc_q=True)
    assert abs(hmg.host_hessenberg_max_real_eig(Hs) - np.linalg.eigvalsh(A).max()) < 1e-9 * np.linalg.norm(A)


def test_descriptor_defaults_follow_the_paper(hmg):
    import ctypes
    d = hmg.Desc()
    assert hmg.lib().hmg_desc_default(ctypes.byref(d)) == 0
    assert d.nu_pre == 3 and d.nu_post == 3 and abs(d.omega - 2 / 3) < 1e-15
    assert d.arnoldi_iters == 10 and d.cheb_lo_frac == 0.25 and d.n_hlevels == 3


def test_descriptor_layout_matches_the_c_header(hmg, tmp_path):
    """The ctypes descriptor has the C struct's size and every field at the C offset (a field
    added on one side only would shift the ones after it), and the defaults leave the finest
    operator in native FP64 arithmetic."""
    import ctypes
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = [f[0] for f in hmg.Desc._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hmg.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(hmg_desc));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(hmg_desc, {n}));\n' for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(hmg.Desc)
    for n, off in zip(names, vals[1:]):
        assert getattr(hmg.Desc, n).offset == off, n
    d = hmg.Desc()
    assert hmg.lib().hmg_desc_default(ctypes.byref(d)) == 0
    assert d.fp64_arith == 0
    prob = dict(dim=3, nelem=(2, 2, 2), order=4)
    assert hmg.make_desc(prob).fp64_arith == 0
    assert hmg.make_desc(dict(prob, fp64_arith="df64")).fp64_arith == 1


def test_status_strings(hmg):
    lib = hmg.lib()
    for s in range(-7, 1):
        assert lib.hmg_status_string(s)


def test_workload_builders_for_the_paper_studies():
    """Host logic of the study workloads: the spectral problems have 961 interior unknowns at
    every order, and the low-order problem is order 1 on order * nelem elements with an h-hierarchy
    whose coarsest grid is small (or the finest grid itself when it cannot be halved)."""
    import numpy as np
    import synth
    for p in (1, 2, 4, 8, 16):
        pr = synth.spectral_problem("2d-var", p, "cheb")
        assert pr["n_hlevels"] == 2 and ((pr["nelem"][0] * p) - 1) ** 2 == 961
    for prob, levels in ((synth.problem(2, 32, 8), 3), (synth.problem(2, 32, 3), 2),
                         (synth.problem(3, 4, 4), 1), (synth.problem(2, (7, 5), 3), 1)):
        N = int(np.prod([e * prob["order"] + 1 for e in prob["nelem"]]))
        lo = synth.low_order_problem(prob, np.zeros((prob["dim"], N)))
        assert lo["order"] == 1 and list(lo["nelem"]) == [e * prob["order"] for e in prob["nelem"]]
        assert lo["n_hlevels"] == levels, (prob["nelem"], prob["order"], lo["n_hlevels"])
        assert lo["node_xyz"].shape == (prob["dim"], N)


def test_header_is_plain_c(tmp_path):
    """include/hmg.h is a C header: a C99 translation unit that uses every enum and the
    descriptor compiles with -pedantic -Werror (no C++ types cross the boundary)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use_hmg.c"
    src.write_text(
        '#include "hmg.h"\n'
        "int main(void) {\n"
        "  hmg_desc d;\n"
        "  hmg_problem* p = 0;\n"
        "  (void)d; (void)p;\n"
        "  return (int)HMG_OK + (int)HMG_HIER_P + (int)HMG_SMOOTH_BLOCKJACOBI + (int)HMG_MODE_PCG +\n"
        "         (int)HMG_PREC_BF16 + (int)HMG_ARITH_DF64 - 8;\n"
        "}\n")
    r = subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(root, "include"), "-c", str(src), "-o", str(tmp_path / "use_hmg.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
