"""Per-element lambda (grid option lambda_min > 0; Section 1: Lambda =
(alpha_K, alpha_K, lambda_K) piecewise constant; Section 2.3: adapted here by
the rule of alpha) on the GPU against the FP64 oracle with the same field."""
import numpy as np
import pytest

from paper_1508_02977_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")

EPS32 = np.finfo(np.float32).eps


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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def abs_matvec(sysm, x):
    A = sp.csr_matrix((np.abs(sysm.val), sysm.col, sysm.rowptr), shape=(sysm.n, sysm.n))
    return (A @ np.abs(np.asarray(x).ravel())).reshape(3, sysm.H, sysm.W)


def lam_field(W, H, seed):
    return 0.3 + np.random.default_rng(seed).random((H - 1, W - 1, 2)) * 2.0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("W,H", [(64, 48), (7, 5), (130, 67), (2, 9)])
def test_apply_with_lambda_field_matches_oracle(S, oracle, prec, W, H):
    f1, f2 = synth.random_frames(W, H, 700 + W)
    alpha = synth.random_alpha(W, H, 710 + H)
    lamel = lam_field(W, H, 720 + W * H)
    if prec == 1:
        f1, f2, alpha, lamel = f32(f1), f32(f2), f32(alpha), f32(lamel)
    dt = torch.float64 if prec == 0 else torch.float32
    sysm = oracle.System.from_frames(f1, f2, alpha, 1.0, lamel=lamel)
    p = np.random.default_rng(730).standard_normal((3, H, W))
    if prec == 1:
        p = f32(p)
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(W, H)], precision=prec, lambda_min=0.01)
        S.of_set_frames(h, 0, dev(f1, dt), dev(f2, dt))
        S.of_set_alpha(h, 0, dev(alpha, dt))
        S.of_set_lambda(h, 0, dev(lamel, dt))
        q = torch.zeros(3, H, W, dtype=dt, device="cuda")
        S.of_apply(h, 0, dev(p, dt), q)
        back = torch.zeros(H - 1, W - 1, 2, dtype=torch.float64, device="cuda")
        S.of_get_lambda(h, 0, back)
        q, back = q.cpu().numpy().astype(np.float64), back.cpu().numpy()
    finally:
        S.of_destroy(h)
    assert np.array_equal(back, lamel)
    tol = 1e-13 if prec == 0 else 64 * EPS32
    assert np.all(np.abs(q - sysm.matvec(p)) <= tol * abs_matvec(sysm, p) + 1e-300)


def test_solves_with_lambda_field_match_oracle(S, oracle):
    """FP64 path: the direct solution to 1e-10; mixed path (FP16 sweeps, whose
    preconditioner keeps the constant lambda): residual <= 1e-6 with the field
    and flow within 1e-4 px of the oracle's solution."""
    p = synth.blobs()
    lamel = lam_field(p.W, p.H, 740)
    Ud = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam, lamel=lamel).solve_direct()
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(p.W, p.H)], tile=(32, 24), overlap=4, precision=0, lambda_min=0.01)
        S.of_set_frames(h, 0, dev(p.f1), dev(p.f2))
        S.of_set_alpha(h, 0, None, p.alpha0)
        S.of_set_lambda(h, 0, dev(lamel))
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-14, max_inner=20000)
        U = U.cpu().numpy()
    finally:
        S.of_destroy(h)
    assert np.linalg.norm(U - Ud) <= 1e-10 * np.linalg.norm(Ud)

    t = synth.texture(240, 192, seed=741)
    lamel = f32(lam_field(t.W, t.H, 742))
    f1, f2 = f32(t.f1), f32(t.f2)
    sysm = oracle.System.from_frames(f1, f2, t.alpha0, t.lam, lamel=lamel)
    Uo, _, _ = sysm.solve_pcg(tol=1e-12)
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(t.W, t.H)], tile=(48, 48), sweeps=4, omega=1.6, precision=1, lambda_min=0.01)
        S.of_set_frames(h, 0, dev(t.f1, torch.float32), dev(t.f2, torch.float32))
        S.of_set_alpha(h, 0, None, t.alpha0)
        S.of_set_lambda(h, 0, dev(lamel, torch.float32))
        U = torch.zeros(3, t.H, t.W, dtype=torch.float64, device="cuda")
        st, info = S.of_solve(h, [U], rtol=1e-6)
        U = U.cpu().numpy()
    finally:
        S.of_destroy(h)
    assert sysm.rel_residual(U) <= 1e-6, info
    assert np.abs(U[:2] - Uo[:2]).max() <= 1e-4


def test_adaptation_pass_updates_lambda_like_the_oracle(S, oracle):
    """One adaptation pass (Section 2.3) on the FP64 path with a per-element
    lambda: the indicator with Lambda_K = (alpha_K, alpha_K, lambda_K) and
    Lambda_e the max of the two sides, then alpha and lambda by the same rule
    (thresholds alpha_th and lambda_min)."""
    p = synth.blobs()
    alpha = synth.random_alpha(p.W, p.H, 750, 0.02, 0.08)
    lamel = lam_field(p.W, p.H, 751)
    lam_min = 0.05
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(p.W, p.H)], tile=(32, 24), precision=0, lambda_min=lam_min, lam=2.5)
        S.of_set_frames(h, 0, dev(p.f1), dev(p.f2))
        S.of_set_alpha(h, 0, dev(alpha))
        S.of_set_lambda(h, 0, dev(lamel))
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-12, max_inner=20000)
        eta = torch.zeros(p.H - 1, p.W - 1, 2, dtype=torch.float64, device="cuda")
        S.of_adapt_alpha(h, 4.0, 0.25, 1e-3, [eta])
        a_new, l_new = torch.zeros_like(eta), torch.zeros_like(eta)
        S.of_get_alpha(h, 0, a_new)
        S.of_get_lambda(h, 0, l_new)
        U, eta, a_new, l_new = U.cpu().numpy(), eta.cpu().numpy(), a_new.cpu().numpy(), l_new.cpu().numpy()
        with pytest.raises(S.OFError) as e:
            z = np.zeros_like(a_new)
            S.of_adapt_alpha_vjp(h, 4.0, 0.25, 1e-3, [dev(z)], [dev(z)], [dev(np.zeros((3, p.H, p.W)))])
        assert e.value.status == S.OF_ERR_STATE
    finally:
        S.of_destroy(h)
    sysm = oracle.System.from_frames(p.f1, p.f2, alpha, 2.5, lamel=lamel)
    eta_o = sysm.indicator(U)
    assert np.abs(eta - eta_o).max() <= 1e-12 * eta_o.max()
    a_o = oracle.alpha_update(eta_o, alpha, 4.0, 0.25, 1e-3)
    l_o = oracle.alpha_update(eta_o, lamel, 4.0, 0.25, lam_min)
    assert np.abs(a_new - a_o).max() <= 1e-12 * a_o.max()
    assert np.abs(l_new - l_o).max() <= 1e-12 * l_o.max()
    assert (l_new < lamel).any() and (l_new == lamel).any()


def test_lambda_field_arguments(S):
    h = S.of_create(0)
    try:
        S.of_setup_grid(h, [(20, 16)], precision=0)
        with pytest.raises(S.OFError) as e:
            S.of_set_lambda(h, 0, None, 1.0)
        assert e.value.status == S.OF_ERR_STATE
        for kw in (dict(lambda_min=2.0, lam=1.0), dict(lambda_min=0.1, rho=1.0), dict(lambda_min=-1.0)):
            with pytest.raises(S.OFError) as e:
                S.of_setup_grid(h, [(20, 16)], precision=0, **kw)
            assert e.value.status == S.OF_ERR_ARG
    finally:
        S.of_destroy(h)
