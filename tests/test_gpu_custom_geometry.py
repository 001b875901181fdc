"""User-given geometry (node_xyz) and coefficient (mu_fn) through hmg_setup, against the oracle
with the same inputs: the finest and a coarser level's operators (the coarser level's nodes are
the finest isoparametric map at its own reference nodes, computed on the GPU), the load vector,
and PCG iteration counts; plus the built-in warp reproduced by given coordinates and the error
paths (a bad coefficient, a folded mesh, the server refusing user callbacks)."""
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


def bumpy_map(X):
    """A non-polynomial smooth map of [0,1]^d fixing the boundary."""
    s = np.prod(np.sin(np.pi * X), axis=1)
    return X + 0.08 * s[:, None] * np.cos(np.pi * X[:, ::-1])


def mu_field(x):
    return 1.0 + 5.0 * x[0] ** 2 + 40.0 * np.exp(-10.0 * np.sum((x - 0.5) ** 2, axis=0))


CASES = [synth.problem(2, 8, 4, hier="p", n_hlevels=2, smoother="cheb"),
         synth.problem(3, 4, 4, hier="p", n_hlevels=2, smoother="cheb"),
         synth.problem(3, 4, 2, hier="h", n_hlevels=2, smoother="jacobi")]


@pytest.mark.parametrize("prob", CASES, ids=lambda c: f"{c['dim']}d-p{c['order']}-{c['hier']}")
def test_custom_geometry_and_coefficient_match_oracle(hmg, prob):
    ref = fem.Discretization(prob["dim"], prob["nelem"], prob["order"])
    prob = dict(prob, node_xyz=bumpy_map(ref.reference_coords()).T.copy(), mu_fn=mu_field)
    P = hmg.Problem(prob)
    H = multigrid.Hierarchy(prob)
    for k in range(min(2, P.nlevels())):
        d = H.levels[k].disc
        x = synth.uniform_pm1(40 + k, d.N)
        x[d.boundary] = 0.0
        y = torch.zeros(d.N, dtype=torch.float64, device=DEV)
        P.apply(k, _t(x), y)
        want = H.levels[k].A @ x[d.interior]
        got = y.cpu().numpy()[d.interior]
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max(), k
    for k in range(P.nlevels()):  # the coordinates the library reports are the ones it used
        d = H.levels[k].disc
        buf = torch.zeros(prob["dim"] * d.N, dtype=torch.float64, device=DEV)
        P.node_coords(k, buf)
        xyz = buf.cpu().numpy().reshape(prob["dim"], d.N)
        assert np.abs(xyz - d.node_coords().T).max() < 1e-13, k
    d = H.fine.disc
    f = synth.nodal_field(41, d.N)
    b = torch.zeros(d.N, dtype=torch.float64, device=DEV)
    P.rhs(_t(f), b)
    bref = d.rhs(f)
    assert np.abs(b.cpu().numpy()[d.interior] - bref).max() <= 1e-12 * np.abs(bref).max()
    u = torch.zeros_like(b)
    st, it, _ = P.solve("pcg", b, u, rtol=1e-8, maxit=200)
    _, it_ref, _, ok = H.solve_pcg(bref)
    assert st == 0 and ok and abs(it - it_ref) <= 1
    P.close()


def test_given_coordinates_reproduce_the_warp(hmg):
    """node_xyz = the built-in warp at the finest nodes: the finest operator is the built-in one."""
    prob = synth.warped_var3d(4, 4, hier="p")
    d = fem.Discretization(3, 4, 4, warp_amp=0.1)
    P0 = hmg.Problem(prob)
    P1 = hmg.Problem(dict(prob, warp_amp=0.0, node_xyz=d.node_coords().T.copy()))
    x = _t(synth.uniform_pm1(42, d.N))
    y0, y1 = torch.zeros_like(x), torch.zeros_like(x)
    P0.apply(0, x, y0)
    P1.apply(0, x, y1)
    assert float((y1 - y0).abs().max()) <= 1e-12 * float(y0.abs().max())
    P0.close()
    P1.close()


def test_custom_inputs_rejected_cleanly(hmg):
    base = synth.problem(2, 4, 2, hier="h", n_hlevels=1, smoother="jacobi")
    with pytest.raises(hmg.HmgError) as e:
        hmg.Problem(dict(base, mu_fn=lambda x: -np.ones(x.shape[1])))
    assert e.value.status == hmg.hmg.HMG_EINVAL
    with pytest.raises(hmg.HmgError):
        hmg.Problem(dict(base, mu_fn=lambda x: 1 / 0))            # a raising callback
    d = fem.Discretization(2, 4, 2)
    folded = d.reference_coords().T.copy()
    folded[0] = 1.0 - folded[0]                                   # mirrored: det J < 0
    with pytest.raises(hmg.HmgError):
        hmg.Problem(dict(base, node_xyz=folded))
    # the server caches hierarchies by descriptor values, so it refuses user inputs
    srv = hmg.Server(max_slots=1)
    with pytest.raises(hmg.HmgError):
        srv.submit(dict(base, mu_fn=mu_field), np.zeros(hmg.desc_ndof(base)))
    srv.close()
    # the library still works afterwards
    P = hmg.Problem(base)
    P.close()
