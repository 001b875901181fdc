"""The paper's published iteration counts (Tables 1 and 4, point-smoother columns) recomputed by
the GPU solver: within +-2 of every printed count for p <= 8 (the paper's right-hand side is not
given; a seeded U(-1,1) load stands in for it)."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return True


def _cases():
    out = []
    for tab in ("table1_2d_const", "table4_3d_const"):
        for key in ("MG jacobi h", "MG cheb h", "PCG jacobi h", "PCG cheb h", "MG jacobi p", "MG cheb p",
                    "PCG jacobi p", "PCG cheb p"):
            for p in (1, 2, 3, 4, 5, 6, 7, 8):
                if str(p) in GOLD[tab][key]:
                    out.append((tab, key, p))
    return out


@pytest.mark.parametrize("tab,key,p", _cases())
def test_gpu_iteration_counts_match_paper(built, tab, key, p):
    import bench
    it = bench.paper_table_counts(tab, p, key)
    ref = GOLD[tab][key][str(p)]
    assert it is not None and abs(it - ref) <= 2, (it, ref)
