"""Host-buffer entry points and the measured peaks.

hmg_apply_host must give the device apply's result (same kernels: bit for bit up to the order of
the FP64 atomic scatter, so within 1e-14) and hmg_solve_host the solution of hmg_rhs + hmg_solve
(same iterations; solution within 1e-12), for page-locked and pageable host buffers, and the
solution must match the oracle's PCG iteration count (Algorithm 1) within +-1.
hmg_measure_peak: positive, finite rates in the range of a GB300 (FP64 FMA and MMA warps together no
faster than the faster alone; FP64 FMA 0.3-5 TFLOP/s, FP32 FMA
10-300, FP64 MMA 0.1-5)."""
import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_and_solve_host_equal_device_path(hmg, pinned):
    prob = synth.warped_var3d(4, 3, hier="p", n_hlevels=2)
    P = hmg.Problem(prob)
    N = P.ndof(0)
    x = torch.from_numpy(synth.uniform_pm1(51, N))
    f = torch.from_numpy(synth.nodal_field(52, N))
    if pinned:
        x, f = x.pin_memory(), f.pin_memory()
    for level in range(P.nlevels()):
        n = P.ndof(level)
        xl = x[:n].contiguous()
        yh = np.zeros(n)
        P.apply_host(level, xl.numpy() if not pinned else xl, yh if not pinned else torch.from_numpy(yh))
        yd = torch.zeros(n, dtype=torch.float64, device=DEV)
        P.apply(level, xl.to(DEV), yd)
        yd = yd.cpu().numpy()
        assert np.abs(yh - yd).max() <= 1e-14 * np.abs(yd).max(), level
    uh = torch.zeros(N, dtype=torch.float64)
    st, it, hist = P.solve_host("pcg", f, uh, rtol=1e-8, maxit=100)
    b = torch.zeros(N, dtype=torch.float64, device=DEV)
    P.rhs(f.to(DEV), b)
    ud = torch.zeros_like(b)
    st2, it2, hist2 = P.solve("pcg", b, ud, rtol=1e-8, maxit=100)
    assert st == st2 == 0 and it == it2
    assert hist[-1] <= 1e-8 * hist[0]
    assert float((uh - ud.cpu()).abs().max() / ud.abs().max()) <= 1e-12
    from oracle import multigrid
    H = multigrid.Hierarchy(prob)
    _, it_ref, _, ok = H.solve_pcg(H.fine.disc.rhs(f.numpy()))
    assert ok and abs(it - it_ref) <= 1
    with pytest.raises(ValueError):
        P.apply_host(0, np.zeros(N - 1), np.zeros(N))
    P.close()


def test_measure_peak_in_range(hmg):
    fp64 = hmg.measure_peak("fp64")
    fp32 = hmg.measure_peak("fp32")
    mma = hmg.measure_peak("fp64_mma")
    both = hmg.measure_peak("fp64_both")
    assert 0.3 < fp64 < 5.0, fp64
    assert 10.0 < fp32 < 300.0, fp32
    assert 0.1 < mma < 5.0, mma
    # FMA and MMA warps together: no faster than the faster of the two alone (one set of FP64
    # units), so the FP64 FMA rate is the FP64 operator's roof
    assert 0.1 < both < 1.2 * max(fp64, mma), (both, fp64, mma)
    print(f"measured TFLOP/s: FP64 FMA {fp64:.3f}, FP32 FMA {fp32:.2f}, FP64 MMA {mma:.3f}, both {both:.3f}")
