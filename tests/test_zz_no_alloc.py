"""of_residual_noalloc, the entry point for callers that cannot allocate
device memory (for instance code inside a frame-budgeted loop, or a plug-in
whose host owns every allocation): it must give the same residual as the
handle-based entry points, call after call, using only its static scratch.

Kept in its own file so that pytest collects it last."""
import numpy as np
import pytest

from paper_1508_02977_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1508_02977_gb300 import ofsolve
    return ofsolve


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def handle_reference(S, f1, f2, alpha, lam, U):
    """Relative residual (of_residual) and b - A U (of_apply) from an FP64
    handle: the existing entry points."""
    H, W = f1.shape
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(W, H)], precision=S.OF_PREC_FP64, lam=lam)
        S.of_set_frames(h, 0, dev(f1), dev(f2))
        S.of_set_alpha(h, 0, dev(alpha))
        rel = S.of_residual(h, 0, dev(U))
        q = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
        b = torch.zeros_like(q)
        S.of_apply(h, 0, dev(U), q, b)
        return rel, (b - q).cpu().numpy(), (b.abs() + q.abs()).cpu().numpy()
    finally:
        S.of_destroy(h)


def test_noalloc_residual_matches_handle_path_twice(S):
    lam = 0.9
    # two calls in a row on different frames and sizes: the shared scratch
    # (partials and counter) must not carry anything over
    for k, (W, H) in enumerate([(300, 200), (131, 67)]):
        f1, f2 = synth.random_frames(W, H, 900 + k)
        alpha = synth.random_alpha(W, H, 910 + k)
        U = np.random.default_rng(920 + k).standard_normal((3, H, W)) * 0.1
        rel_ref, r_ref, scale = handle_reference(S, f1, f2, alpha, lam, U)
        r = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
        norms = torch.zeros(3, dtype=torch.float64, device="cuda")
        st = S.of_residual_noalloc(dev(f1), dev(f2), dev(alpha), lam, dev(U), r, norms)
        assert st == S.OF_OK
        torch.cuda.synchronize()
        n = norms.cpu().numpy()
        assert abs(n[0] - rel_ref) <= 1e-12 * rel_ref
        assert np.sqrt(n[1] / n[2]) == pytest.approx(n[0], rel=1e-14)
        assert np.all(np.abs(r.cpu().numpy() - r_ref) <= 1e-13 * (scale + 1e-300))


def test_noalloc_norms_without_r_match_handle_and_oracle(S, oracle):
    """With r = NULL only the norms are written: the same relative residual
    as of_residual and as the FP64 oracle's CSR residual, on two calls in a
    row (a solve-like U, so that the residual is small against b)."""
    lam = 1.0
    for k, (W, H) in enumerate([(96, 80), (250, 31)]):
        p = synth.texture(W, H, seed=930 + k)
        alpha = np.full((H - 1, W - 1, 2), p.alpha0)
        sysm = oracle.System.from_frames(p.f1, p.f2, alpha, lam)
        U, _, _ = sysm.solve_pcg(tol=1e-4)
        rel_o = sysm.rel_residual(U)
        rel_ref, _, _ = handle_reference(S, p.f1, p.f2, alpha, lam, U)
        norms = torch.zeros(3, dtype=torch.float64, device="cuda")
        st = S.of_residual_noalloc(dev(p.f1), dev(p.f2), dev(alpha), lam, dev(U), None, norms)
        assert st == S.OF_OK
        torch.cuda.synchronize()
        n = norms.cpu().numpy()
        assert abs(n[0] - rel_ref) <= 1e-12 * rel_ref
        assert abs(n[0] - rel_o) <= 1e-9 * rel_o
        assert n[2] == pytest.approx(np.dot(sysm.b, sysm.b), rel=1e-12)


def test_noalloc_rejects_frames_beyond_the_scratch(S):
    W, H = 20000, 8192  # ceil(20000/124) * ceil(8192/32) = 162 * 256 > 32768
    tiny = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = S._lib.of_residual_noalloc(W, H, S._vp(tiny.data_ptr()), S._vp(tiny.data_ptr()), S._vp(tiny.data_ptr()),
                                    1.0, S._vp(tiny.data_ptr()), None, S._vp(tiny.data_ptr()), None)
    assert st == S.OF_ERR_ARG
