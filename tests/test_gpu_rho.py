"""GPU parity of the K_rho data term (Section 1: the matrix A_rho and the
vector F): element data, operator, load, solves, indicator and the alpha
gradient, through the C ABI against the FP64 oracle."""
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


def handle(S, sizes, **kw):
    h = S.of_create(0)
    S.of_setup_grid(h, sizes, **kw)
    return h


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def csr_abs_matvec(sysm, x):
    A = sp.csr_matrix((np.abs(sysm.val), sysm.col, sysm.rowptr), shape=(sysm.n, sysm.n))
    return (A @ np.abs(np.asarray(x).ravel())).reshape(3, sysm.H, sysm.W)


def oracle_planes(oracle, f1, f2, rho, model):
    """The oracle's element data in the [18][H-1][W-1] plane order."""
    Ael, Fel = oracle.element_data(f1, f2, rho, model)
    out = []
    for t in range(2):
        out += [Ael[:, :, t, k] for k in range(6)] + [Fel[:, :, t, k] for k in range(3)]
    return np.stack(out)


@pytest.mark.parametrize("prec,model,rho", [(0, 0, 1.5), (0, 1, 2.5), (1, 0, 1.5), (0, 0, 9.0)])
def test_element_data_matches_oracle(S, oracle, prec, model, rho):
    """Products of the element data, K_rho over each triangle family's
    lattice (rho = 9: taps reach past the 53-node height)."""
    W, H = 75, 53
    f1, f2 = synth.random_frames(W, H, 81)
    dt = torch.float64 if prec == 0 else torch.float32
    if prec == 1:
        f1, f2 = f32(f1), f32(f2)
    h = handle(S, [(W, H)], precision=prec, model=model, rho=rho)
    try:
        S.of_set_frames(h, 0, dev(f1, dt), dev(f2, dt))
        out = torch.zeros(18, H - 1, W - 1, dtype=dt, device="cuda")
        S.of_get_element_data(h, 0, out)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        S.of_destroy(h)
    want = oracle_planes(oracle, f1, f2, rho, model)
    for q in range(18):
        scale = max(np.abs(want[q]).max(), 1e-300)
        err = np.abs(got[q] - want[q]).max() / scale
        assert err <= (1e-13 if prec == 0 else 2e-6), (q, err)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("W,H", [(64, 48), (7, 5), (130, 67), (2, 2)])
def test_apply_rho_matches_oracle(S, oracle, prec, W, H):
    rho, lam = 1.3, 0.8
    f1, f2 = synth.random_frames(W, H, 3 * W + H)
    alpha = synth.random_alpha(W, H, W + 2 * H)
    p = np.random.default_rng(W * H + 5).standard_normal((3, H, W))
    dt = torch.float64 if prec == 0 else torch.float32
    if prec == 1:
        f1, f2, alpha, p = f32(f1), f32(f2), f32(alpha), f32(p)
    sysm = oracle.System.from_frames(f1, f2, alpha, lam, rho=rho)
    h = handle(S, [(W, H)], precision=prec, lam=lam, rho=rho)
    try:
        S.of_set_frames(h, 0, dev(f1, dt), dev(f2, dt))
        S.of_set_alpha(h, 0, dev(alpha, dt))
        q = torch.zeros(3, H, W, dtype=dt, device="cuda")
        b = torch.zeros_like(q)
        S.of_apply(h, 0, dev(p, dt), q, b)
        q, b = q.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    finally:
        S.of_destroy(h)
    scale = csr_abs_matvec(sysm, p)
    tol = 1e-13 if prec == 0 else 128 * EPS32
    assert np.all(np.abs(q - sysm.matvec(p)) <= tol * scale + 1e-300)
    bw = sysm.b.reshape(3, H, W)
    assert np.abs(b - bw).max() <= (1e-13 if prec == 0 else 1e-5) * max(np.abs(bw).max(), 1e-300)


def test_rho_preconditioner_is_the_unsmoothed_one(S, oracle):
    """With rho > 0 the Schwarz sweeps still use the element records of
    g g^T: z = M r equals the oracle's sweeps on the unsmoothed system."""
    W, H = 75, 53
    f1, f2 = synth.random_frames(W, H, 83)
    alpha = synth.random_alpha(W, H, 84)
    sysm = oracle.System.from_frames(f1, f2, alpha, 1.0, rho=2.0)
    r = np.random.default_rng(85).standard_normal((3, H, W))
    h = handle(S, [(W, H)], precision=0, tile=(16, 12), sweeps=2, omega=1.6, rho=2.0)
    try:
        S.of_set_frames(h, 0, dev(f1), dev(f2))
        S.of_set_alpha(h, 0, dev(alpha))
        z = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
        S.of_precondition(h, 0, dev(r), z)
        z = z.cpu().numpy()
    finally:
        S.of_destroy(h)
    want = sysm.precond_system().schwarz_sweeps(r, (16, 12), 0, 2, 1.6)
    assert np.abs(z - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("coarse", [0, 12])
def test_rho_fp64_solve_matches_direct(S, oracle, coarse):
    p = synth.blobs()
    sysm = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam, rho=1.5)
    Ud = sysm.solve_direct()
    h = handle(S, [(p.W, p.H)], precision=0, tile=(16, 16), sweeps=2, omega=1.5, rho=1.5, coarse=coarse)
    try:
        S.of_set_frames(h, 0, dev(p.f1), dev(p.f2))
        S.of_set_alpha(h, 0, None, p.alpha0)
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-14, max_inner=20000)
        U = U.cpu().numpy()
    finally:
        S.of_destroy(h)
    assert np.linalg.norm(U - Ud) <= 1e-10 * np.linalg.norm(Ud)


def test_rho_mixed_solve_texture(S, oracle):
    """640x480 texture, mixed precision, rho = 1.5: the oracle's FP64
    residual of the returned flow (oracle operator from the FP32 frames)."""
    t = synth.texture()
    f1, f2 = f32(t.f1), f32(t.f2)
    h = handle(S, [(t.W, t.H)], tile=(48, 48), sweeps=4, omega=1.6, precision=1, rho=1.5)
    try:
        S.of_set_frames(h, 0, dev(t.f1, torch.float32), dev(t.f2, torch.float32))
        S.of_set_alpha(h, 0, None, t.alpha0)
        U = torch.zeros(3, t.H, t.W, dtype=torch.float64, device="cuda")
        st, info = S.of_solve(h, [U], rtol=1e-6)
        U = U.cpu().numpy()
    finally:
        S.of_destroy(h)
    sysm = oracle.System.from_frames(f1, f2, np.float32(t.alpha0), t.lam, rho=1.5)
    assert sysm.rel_residual(U) <= 1e-6


def test_rho_indicator_matches_oracle(S, oracle):
    p = synth.blobs()
    alpha = synth.random_alpha(p.W, p.H, 86, 0.02, 0.08)
    h = handle(S, [(p.W, p.H)], precision=0, tile=(32, 24), rho=1.5)
    try:
        S.of_set_frames(h, 0, dev(p.f1), dev(p.f2))
        S.of_set_alpha(h, 0, dev(alpha))
        U = torch.zeros(3, p.H, p.W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-12)
        eta = torch.zeros(p.H - 1, p.W - 1, 2, dtype=torch.float64, device="cuda")
        S.of_adapt_alpha(h, 4.0, 0.25, 1e-3, [eta])
        U, eta = U.cpu().numpy(), eta.cpu().numpy()
    finally:
        S.of_destroy(h)
    eta_o = oracle.System.from_frames(p.f1, p.f2, alpha, p.lam, rho=1.5).indicator(U)
    assert np.abs(eta - eta_o).max() <= 1e-12 * eta_o.max()


def test_rho_adjoint_gradients_match_oracle(S, oracle):
    """dL/dalpha and dL/df2, dL/df1 through the adjoint solve with the K_rho
    operator (L = mean EPE): against the oracle's adjoint gradient (pinned by
    central differences) on the same U and adjoint state, and dL/dalpha
    against central differences of oracle direct solves."""
    W, H, rho, lam = 24, 20, 1.2, 1.0
    f1, f2 = synth.random_frames(W, H, 87)
    alpha = synth.random_alpha(W, H, 88)
    gt = np.random.default_rng(89).uniform(-1, 1, (2, H, W))
    sysm = oracle.System.from_frames(f1, f2, alpha, lam, rho=rho)
    Ud = sysm.solve_direct()
    g = oracle.mean_epe_grad(Ud, gt)
    h = handle(S, [(W, H)], precision=0, tile=(8, 8), sweeps=2, rho=rho)
    try:
        S.of_set_frames(h, 0, dev(f1), dev(f2))
        S.of_set_alpha(h, 0, dev(alpha))
        U = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-14, max_inner=20000)
        da = torch.zeros(H - 1, W - 1, 2, dtype=torch.float64, device="cuda")
        d2 = torch.zeros(H, W, dtype=torch.float64, device="cuda")
        d1 = torch.zeros(H, W, dtype=torch.float64, device="cuda")
        S.of_adjoint(h, [dev(g)], [da], [d2], [d1])
        da, d2, d1 = da.cpu().numpy(), d2.cpu().numpy(), d1.cpu().numpy()
    finally:
        S.of_destroy(h)
    Lam = sysm.solve_with(g)
    wa, w2, w1 = oracle.adjoint_grad(f1, f2, alpha, lam, Ud, Lam, rho=rho)
    for got, want in ((da, wa), (d2, w2), (d1, w1)):
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    hstep = 1e-5
    for (y, x, t) in [(0, 0, 0), (5, 7, 1), (18, 22, 0), (3, 2, 1)]:
        vals = []
        for sgn in (1, -1):
            a = alpha.copy()
            a[y, x, t] += sgn * hstep
            Us = oracle.System.from_frames(f1, f2, a, lam, rho=rho).solve_direct()
            vals.append(oracle.mean_epe(Us, gt))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        assert abs(da[y, x, t] - fd) <= 1e-5 * np.abs(da).max(), (y, x, t, da[y, x, t], fd)


def test_rho_adjoint_mixed_with_presmoothing(S, oracle):
    """FP32 path with K_sigma and K_rho together: frame gradients w.r.t. the
    unsmoothed images against the oracle (its chain rule through
    smooth_transpose of the K_sigma step) to 1e-3 of the largest entry."""
    W, H, rho, sig, lam = 40, 30, 1.5, 1.0, 1.0
    I1, I2 = synth.random_frames(W, H, 90)
    I1, I2 = f32(I1), f32(I2)
    alpha = f32(synth.random_alpha(W, H, 91))
    f1, f2 = oracle.smooth(I1, sig), oracle.smooth(I2, sig)
    c = np.random.default_rng(92).standard_normal((3, H, W))
    h = handle(S, [(W, H)], precision=1, tile=(16, 16), sweeps=2, rho=rho, sigma=sig)
    try:
        S.of_set_frames(h, 0, dev(I1, torch.float32), dev(I2, torch.float32))
        S.of_set_alpha(h, 0, dev(alpha, torch.float32))
        U = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-10)
        d2 = torch.zeros(H, W, dtype=torch.float64, device="cuda")
        S.of_adjoint(h, [dev(c)], None, [d2])
        d2 = d2.cpu().numpy()
        fs1, fs2 = (torch.zeros(H, W, dtype=torch.float64, device="cuda") for _ in range(2))
        S.of_get_frames(h, 0, fs1, fs2)
        fs1, fs2 = fs1.cpu().numpy(), fs2.cpu().numpy()
    finally:
        S.of_destroy(h)
    sysm = oracle.System.from_frames(fs1, fs2, alpha, lam, rho=rho)
    Ud = sysm.solve_direct()
    Lam = sysm.solve_with(c)
    _, w2, _ = oracle.adjoint_grad(fs1, fs2, alpha, lam, Ud, Lam, rho=rho)
    want = oracle.smooth_transpose(w2, sig)
    assert np.abs(d2 - want).max() <= 1e-3 * np.abs(want).max()


def test_rho_batch_of_two_pairs(S, oracle):
    """K_rho element data, operator and adjoint frame gradients of a batch of
    two pairs of different sizes (per-pair plane offsets) against the oracle
    pair by pair (FP64)."""
    sizes = [(33, 21), (20, 28)]
    rho, lam = 1.3, 1.0
    data = []
    for i, (W, H) in enumerate(sizes):
        f1, f2 = synth.random_frames(W, H, 93 + i)
        data.append((f1, f2, synth.random_alpha(W, H, 95 + i)))
    h = handle(S, sizes, precision=0, tile=(8, 8), sweeps=2, rho=rho, lam=lam)
    try:
        Us, planes, qs = [], [], []
        for i, (f1, f2, a) in enumerate(data):
            W, H = sizes[i]
            S.of_set_frames(h, i, dev(f1), dev(f2))
            S.of_set_alpha(h, i, dev(a))
            out = torch.zeros(18, H - 1, W - 1, dtype=torch.float64, device="cuda")
            S.of_get_element_data(h, i, out)
            planes.append(out.cpu().numpy())
            p = np.random.default_rng(97 + i).standard_normal((3, H, W))
            q = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
            S.of_apply(h, i, dev(p), q)
            qs.append((p, q.cpu().numpy()))
            Us.append(torch.zeros(3, H, W, dtype=torch.float64, device="cuda"))
        S.of_solve(h, Us, rtol=1e-14, max_inner=20000)
        cs = [np.random.default_rng(99 + i).standard_normal((3, H, W)) for i, (W, H) in enumerate(sizes)]
        d2 = [torch.zeros(H, W, dtype=torch.float64, device="cuda") for W, H in sizes]
        S.of_adjoint(h, [dev(c) for c in cs], None, d2)
    finally:
        S.of_destroy(h)
    for i, (f1, f2, a) in enumerate(data):
        want = oracle_planes(oracle, f1, f2, rho, 0)
        assert np.abs(planes[i] - want).max() <= 1e-13 * np.abs(want).max()
        sysm = oracle.System.from_frames(f1, f2, a, lam, rho=rho)
        p, q = qs[i]
        assert np.all(np.abs(q - sysm.matvec(p)) <= 1e-13 * csr_abs_matvec(sysm, p) + 1e-300)
        U = sysm.solve_direct()
        Lam = sysm.solve_with(cs[i])
        _, w2, _ = oracle.adjoint_grad(f1, f2, a, lam, U, Lam, rho=rho)
        assert np.abs(d2[i].cpu().numpy() - w2).max() <= 1e-8 * np.abs(w2).max()


def test_rho_adapt_alpha_vjp_batch_matches_oracle(S, oracle):
    """of_adapt_alpha_vjp with the K_rho data term (interior residual
    F - A_rho U_h; frame derivatives through K_rho^T) on a batch of two
    pairs of different sizes, one spanning several blocks in x and several
    K_rho strips in y (FP64): dL/dalpha, dL/dU, dL/df2, dL/df1 equal the
    oracle's update and indicator VJPs at the GPU's solution."""
    sizes = [(150, 70), (17, 26)]
    rho, lam, kappa, thr, ath = 1.3, 1.0, 4.0, 0.25, 1e-4
    data = []
    for i, (W, H) in enumerate(sizes):
        f1, f2 = synth.random_frames(W, H, 350 + i)
        data.append((f1, f2, synth.random_alpha(W, H, 360 + i),
                     np.random.default_rng(370 + i).standard_normal((H - 1, W - 1, 2))))
    h = handle(S, sizes, precision=0, tile=(8, 8), sweeps=2, rho=rho, lam=lam)
    try:
        Us = []
        for i, (f1, f2, a, _) in enumerate(data):
            S.of_set_frames(h, i, dev(f1), dev(f2))
            S.of_set_alpha(h, i, dev(a))
            Us.append(torch.zeros(3, sizes[i][1], sizes[i][0], dtype=torch.float64, device="cuda"))
        S.of_solve(h, Us, rtol=1e-14, max_inner=20000)
        v = [dev(d[3]) for d in data]
        da = [torch.zeros_like(x) for x in v]
        dU = [torch.zeros_like(u) for u in Us]
        d2 = [torch.zeros(hh, w, dtype=torch.float64, device="cuda") for w, hh in sizes]
        d1 = [torch.zeros_like(x) for x in d2]
        S.of_adapt_alpha_vjp(h, kappa, thr, ath, v, da, dU, d2, d1)
    finally:
        S.of_destroy(h)
    for i, (f1, f2, a, vv) in enumerate(data):
        U = Us[i].cpu().numpy()
        eta = oracle.System.from_frames(f1, f2, a, lam, rho=rho).indicator(U)
        wa, w = oracle.alpha_update_vjp(eta, a, kappa, thr, ath, vv)
        wU, wa2, w2, w1 = oracle.indicator_vjp(f1, f2, a, lam, U, w, rho=rho)
        for got, want in ((da[i], wa + wa2), (dU[i], wU), (d2[i], w2), (d1[i], w1)):
            got = got.cpu().numpy()
            assert np.abs(got - want).max() <= 1e-9 * max(np.abs(want).max(), 1e-300), i


def test_rho_adaptation_pass_gradients_match_oracle(S, oracle):
    """Differentiating through one adaptation pass with K_rho (FP64 handle):
    the autograd chain of of_adjoint and of_adapt_alpha_vjp against the
    oracle's reverse chain (pinned by central differences of direct
    solves)."""
    from paper_1508_02977_gb300.autograd import Solver, adapt_solve_fn
    W, H, lam, rho = 24, 18, 1.0, 1.1
    f1, f2 = synth.random_frames(W, H, 380)
    a0 = synth.random_alpha(W, H, 381)
    kappa, thr, ath = 4.0, 0.25, 1e-4
    c = np.random.default_rng(382).standard_normal((3, H, W))
    solver = Solver(W, H, precision=0, tile=(8, 8), sweeps=2, rtol=1e-14, lam=lam, rho=rho)
    try:
        t1 = dev(f1).requires_grad_(True)
        t2 = dev(f2).requires_grad_(True)
        ta = dev(a0).requires_grad_(True)
        U = adapt_solve_fn(t1, t2, ta, solver, 1, kappa, thr, ath)
        (U * dev(c)).sum().backward()
    finally:
        solver.close()
    da, d2, d1 = oracle.adaptation_grad(f1, f2, a0, lam, 1, kappa, thr, ath, c, rho=rho)
    for got, want in ((ta.grad, da), (t2.grad, d2), (t1.grad, d1)):
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-7 * np.abs(want).max()


def test_rho_constant_model_adjoint_and_vjp_match_oracle(S, oracle):
    """Brightness constancy (OF_MODEL_CONSTANT: g = (d/dx f2, d/dy f2, 0))
    with K_rho, FP64 path: flow = the oracle's flow-block direct solve, m
    stays 0, and the adjoint gradients and the one-pass adaptation VJP equal
    the oracle's."""
    W, H, rho, lam, kappa, thr, ath = 30, 22, 1.3, 1.0, 4.0, 0.25, 1e-4
    f1, f2 = synth.random_frames(W, H, 420)
    a = synth.random_alpha(W, H, 421)
    gt = np.random.default_rng(422).uniform(-1, 1, (2, H, W))
    v = np.random.default_rng(423).standard_normal((H - 1, W - 1, 2))
    sysm = oracle.System.from_frames(f1, f2, a, lam, model=1, rho=rho)
    Ud = sysm.solve_direct()
    h = handle(S, [(W, H)], precision=0, tile=(8, 8), sweeps=2, rho=rho, lam=lam, model=S.OF_MODEL_CONSTANT)
    try:
        S.of_set_frames(h, 0, dev(f1), dev(f2))
        S.of_set_alpha(h, 0, dev(a))
        U = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
        S.of_solve(h, [U], rtol=1e-14, max_inner=20000)
        Un = U.cpu().numpy()
        ga = torch.zeros(H - 1, W - 1, 2, dtype=torch.float64, device="cuda")
        g2 = torch.zeros(H, W, dtype=torch.float64, device="cuda")
        g1 = torch.zeros_like(g2)
        S.of_adjoint(h, [dev(oracle.mean_epe_grad(Un, gt))], [ga], [g2], [g1])
        # the adjoint solve left the pass's solution in place: re-solve, then the VJP
        S.of_solve(h, [U], rtol=1e-14, max_inner=20000)
        da = torch.zeros_like(ga)
        dU = torch.zeros_like(U)
        d2 = torch.zeros_like(g2)
        d1 = torch.zeros_like(g2)
        S.of_adapt_alpha_vjp(h, kappa, thr, ath, [dev(v)], [da], [dU], [d2], [d1])
        U2 = U.cpu().numpy()
    finally:
        S.of_destroy(h)
    assert np.abs(Un[2]).max() == 0.0
    assert np.linalg.norm(Un - Ud) <= 1e-10 * np.linalg.norm(Ud)
    Lo = sysm.solve_with(oracle.mean_epe_grad(Ud, gt))
    wa, w2, w1 = oracle.adjoint_grad(f1, f2, a, lam, Ud, Lo, model=1, rho=rho)
    for got, want in ((ga, wa), (g2, w2), (g1, w1)):
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    eta = sysm.indicator(U2)
    ua, w = oracle.alpha_update_vjp(eta, a, kappa, thr, ath, v)
    wU, wa2, v2, v1 = oracle.indicator_vjp(f1, f2, a, lam, U2, w, model=1, rho=rho)
    for got, want in ((da, ua + wa2), (dU, wU), (d2, v2), (d1, v1)):
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-9 * max(np.abs(want).max(), 1e-300)
