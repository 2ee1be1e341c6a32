"""The paper's Schwarz method as a stationary iteration on the GPU (Section
3.2, Eq. schwarz; grid option schwarz = 1) against the oracle's exact-solve
iteration (orc_schwarz) on the 64x48 blobs pair, 2x2 subdomains.

The GPU's local solves are symmetric block-SOR sweeps; with enough sweeps
(600 at omega = 1.8: the error of a local solve on these tiles falls below
1e-12 after about 410) they are exact to rounding, so the iterates must
follow the oracle's iterate by iterate."""
import numpy as np
import pytest

from paper_1508_02977_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EXACT = dict(sweeps=600, omega=1.8)


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1508_02977_gb300 import ofsolve
    return ofsolve


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def ras(S, p, iters, overlap=4, rtol=1e-30, precision=0, dtype=torch.float64, **kw):
    """Runs `iters` stationary Schwarz iterations from U = 0 on a 2x2
    partition (tiles W/2 x H/2); returns (U, history, info)."""
    opts = dict(EXACT)
    opts.update(kw)
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(p.W, p.H)], tile=(p.W // 2, p.H // 2), overlap=overlap, precision=precision,
                        schwarz=1, **opts)
        S.of_set_frames(h, 0, dev(p.f1, dtype), dev(p.f2, dtype))
        S.of_set_alpha(h, 0, None, p.alpha0)
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        st, info = S.of_solve(h, [U], rtol=rtol, max_inner=iters, raise_on=False)
        hist = S.of_get_schwarz_history(h, 0)
        return U.cpu().numpy(), hist, info[0]
    finally:
        S.of_destroy(h)


def test_iterates_match_the_oracle(S, oracle):
    """Iterates 1..6 and the history ||U^k - U^{k-1}||_2 equal the oracle's
    exact-solve Schwarz iteration (2x2 parts, 4-node overlap)."""
    p = synth.blobs()
    sysm = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam)
    Uo, ho = sysm.schwarz(2, 2, 4, 6)
    U, hist, info = ras(S, p, 6)
    assert info["inner_iters"] == 6 and len(hist) == 6
    assert np.linalg.norm(U - Uo) <= 1e-8 * np.linalg.norm(Uo)
    assert np.allclose(hist, ho, rtol=1e-8, atol=0), (hist, ho)
    for k in (1, 3):
        Uk, _, _ = ras(S, p, k)
        Ok, _ = sysm.schwarz(2, 2, 4, k)
        assert np.linalg.norm(Uk - Ok) <= 1e-8 * np.linalg.norm(Ok)


def test_fixed_point_is_the_direct_solution(S, oracle):
    """Iterated to a residual of 1e-13 the method reaches the global
    solution (banded Cholesky) to 1e-10; the residual check stops it."""
    p = synth.blobs()
    Ud = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam).solve_direct()
    U, hist, info = ras(S, p, 200, rtol=1e-13)
    assert info["status"] == S.OF_OK, info
    assert info["inner_iters"] < 200 and info["rel_residual"] <= 1e-13
    assert np.linalg.norm(U - Ud) <= 1e-10 * np.linalg.norm(Ud)
    assert hist[-1] < 1e-9 * hist[0]


def test_more_overlap_converges_faster(S, oracle):
    """Section 4 (Schwarz convergence against the overlap): the iterations
    to reach 1e-8 of the direct solution do not increase with the overlap."""
    p = synth.blobs()
    Ud = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam).solve_direct()
    counts = []
    for ov in (1, 2, 4, 8):
        U, hist, info = ras(S, p, 200, overlap=ov, rtol=1e-9)
        assert np.linalg.norm(U - Ud) <= 1e-7 * np.linalg.norm(Ud), (ov, info)
        counts.append(info["inner_iters"])
    assert all(a >= b for a, b in zip(counts, counts[1:])), counts
    assert counts[0] > counts[-1], counts


def test_mixed_precision_iteration_reaches_the_tolerance(S, oracle):
    """FP32 local solves with the double-float residual: the iteration is a
    refinement, so it still reaches a 1e-8 residual (recomputed by the
    oracle) with a few sweeps per local solve, and the residual decreases
    monotonically in the history."""
    p = synth.texture(160, 120, seed=77)
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(p.W, p.H)], tile=(40, 40), overlap=4, sweeps=24, omega=1.7,
                        precision=S.OF_PREC_MIXED, schwarz=1)
        S.of_set_frames(h, 0, dev(p.f1, torch.float32), dev(p.f2, torch.float32))
        S.of_set_alpha(h, 0, None, p.alpha0)
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        st, info = S.of_solve(h, [U], rtol=1e-8, max_inner=2000)
        hist = S.of_get_schwarz_history(h, 0)
        U = U.cpu().numpy()
    finally:
        S.of_destroy(h)
    f1 = p.f1.astype(np.float32).astype(np.float64)
    f2 = p.f2.astype(np.float32).astype(np.float64)
    rr = oracle.rel_residual_frames(f1, f2, p.alpha0, p.lam, U)
    assert rr <= 1.5e-8, (rr, info)
    assert len(hist) == info[0]["inner_iters"]
    assert hist[-1] < 1e-3 * hist[0]


def test_history_state_and_arguments(S):
    p = synth.blobs()
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(p.W, p.H)], tile=(32, 24), overlap=4, precision=0)
        S.of_set_frames(h, 0, dev(p.f1), dev(p.f2))
        S.of_set_alpha(h, 0, None, p.alpha0)
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-8)
        with pytest.raises(S.OFError) as e:
            S.of_get_schwarz_history(h, 0)
        assert e.value.status == S.OF_ERR_STATE
        with pytest.raises(S.OFError) as e:
            S.of_setup_grid(h, [(p.W, p.H)], tile=(32, 24), overlap=4, precision=0, schwarz=1, coarse=8)
        assert e.value.status == S.OF_ERR_ARG
        with pytest.raises(S.OFError) as e:
            S.of_setup_grid(h, [(p.W, p.H)], tile=(32, 24), overlap=4, precision=0, schwarz=2)
        assert e.value.status == S.OF_ERR_ARG
    finally:
        S.of_destroy(h)
