"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here re-calls an oracle routine to check itself: every expected
value comes from an independent route (generic barycentric geometry and a
different quadrature rule, closed forms, LAPACK, finite differences, the
paper's worked example)."""
import os

import numpy as np
import pytest

from paper_1508_02977_gb300 import synth, partition

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ------------------------------------------------------ independent route --

def triangles(W, H):
    """The mesh of Fig. sch-mesh: each pixel square cut by its
    (x,y)->(x+1,y+1) diagonal; yields (x, y, t, vertices)."""
    for y in range(H - 1):
        for x in range(W - 1):
            yield x, y, 0, [(x, y), (x + 1, y), (x + 1, y + 1)]
            yield x, y, 1, [(x, y), (x, y + 1), (x + 1, y + 1)]


def bary(verts):
    """Gradients of the barycentric coordinates (rows) and the area, from the
    inverse of the vertex matrix (no hand-written gradient table)."""
    M = np.array([[v[0] for v in verts], [v[1] for v in verts], [1.0, 1.0, 1.0]])
    Minv = np.linalg.inv(M)
    return Minv[:, :2], abs(np.linalg.det(M)) / 2.0


# 3-point interior rule, exact for quadratics (Strang & Fix), barycentric
QPTS = [(2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (1 / 6, 1 / 6, 2 / 3)]


def element_data(f1, f2, verts, illumination=True):
    """g = (grad f2_h, -f1_h(centroid)), ft = (f2_h - f1_h)(centroid); without
    illumination (Horn and Schunck's brightness constancy) g = (grad f2_h, 0)."""
    G, _ = bary(verts)
    v2 = np.array([f2[y, x] for x, y in verts])
    v1 = np.array([f1[y, x] for x, y in verts])
    grad2 = G.T @ v2
    cen = np.array([1 / 3, 1 / 3, 1 / 3])
    gm = -(cen @ v1) if illumination else 0.0
    return np.array([grad2[0], grad2[1], gm]), cen @ (v2 - v1)


def bilinear(f1, f2, alpha, lam, U, V, illumination=True):
    """int (g.U_h)(g.V_h) + sum_c Lambda_c grad U_c . grad V_c  and
    the load  -int ft g.V_h, by the 3-point rule."""
    H, W = f1.shape
    a_uv = 0.0
    l_v = 0.0
    for x, y, t, verts in triangles(W, H):
        g, ft = element_data(f1, f2, verts, illumination)
        G, area = bary(verts)
        Lam = np.array([alpha[y, x, t], alpha[y, x, t], lam[y, x, t] if np.ndim(lam) else lam])
        uv = np.array([[U[c, yy, xx] for c in range(3)] for xx, yy in verts])  # [vertex][c]
        vv = np.array([[V[c, yy, xx] for c in range(3)] for xx, yy in verts])
        for q in QPTS:
            q = np.array(q)
            a_uv += area / 3.0 * (g @ (q @ uv)) * (g @ (q @ vv))
            l_v += area / 3.0 * (-ft) * (g @ (q @ vv))
        for c in range(3):
            a_uv += area * Lam[c] * (G.T @ uv[:, c]) @ (G.T @ vv[:, c])
    return a_uv, l_v


# ------------------------------------------------------------ assembly ----

def test_per_element_lambda_operator_equals_weak_form(oracle):
    """With a per-element lambda (Section 1: Lambda piecewise constant on the
    elements) U^T A V equals the weak form with lambda_K on each element, by
    the independent rule; a constant field gives the constant-lambda matrix
    bit for bit."""
    W, H = 5, 4
    rng = np.random.default_rng(57)
    f1, f2 = synth.random_frames(W, H, 58)
    alpha = synth.random_alpha(W, H, 59)
    lamel = 0.2 + rng.random((H - 1, W - 1, 2)) * 3.0
    S = oracle.System.from_frames(f1, f2, alpha, 1.0, lamel=lamel)
    for _ in range(3):
        U = rng.standard_normal((3, H, W))
        V = rng.standard_normal((3, H, W))
        a_uv, l_v = bilinear(f1, f2, alpha, lamel, U, V)
        assert abs(np.sum(V * S.matvec(U)) - a_uv) < 1e-12 * max(1.0, abs(a_uv))
        assert abs(S.b @ V.ravel() - l_v) < 1e-13 * max(1.0, abs(l_v))
    S1 = oracle.System.from_frames(f1, f2, alpha, 0.7)
    S2 = oracle.System.from_frames(f1, f2, alpha, 123.0, lamel=np.full((H - 1, W - 1, 2), 0.7))
    assert np.array_equal(S1.val, S2.val) and np.array_equal(S1.b, S2.b)


def test_lambda_gradient_matches_central_differences(oracle):
    """dL/dlambda_K = -|K| grad(Lam_m) . grad(U_m) (the adjoint of the m
    stiffness) against central differences of L(U(lambda)) through direct
    solves, L = 1/2 |U - U_t|^2."""
    W, H = 7, 6
    rng = np.random.default_rng(61)
    f1, f2 = synth.random_frames(W, H, 62)
    alpha = synth.random_alpha(W, H, 63)
    lamel = 0.5 + rng.random((H - 1, W - 1, 2))
    Ut = rng.standard_normal((3, H, W))

    def solve(lm):
        return oracle.System.from_frames(f1, f2, alpha, 1.0, lamel=lm).solve_direct()

    S = oracle.System.from_frames(f1, f2, alpha, 1.0, lamel=lamel)
    U = S.solve_direct()
    Lam = S.solve_with(U - Ut)
    dl = oracle.adjoint_grad_lambda(f1, f2, alpha, 1.0, U, Lam)
    h = 1e-5
    for _ in range(5):
        y, x, t = rng.integers(0, H - 1), rng.integers(0, W - 1), rng.integers(0, 2)
        lp, lm = lamel.copy(), lamel.copy()
        lp[y, x, t] += h
        lm[y, x, t] -= h
        fd = (0.5 * np.sum((solve(lp) - Ut) ** 2) - 0.5 * np.sum((solve(lm) - Ut) ** 2)) / (2 * h)
        assert abs(fd - dl[y, x, t]) <= 1e-6 * np.abs(dl).max(), (fd, dl[y, x, t])


def test_coefficients_match_p1_interpolant(oracle):
    f1, f2 = synth.random_frames(6, 5, 11)
    g, ft = oracle.coefficients(f1, f2)
    for x, y, t, verts in triangles(6, 5):
        ge, fte = element_data(f1, f2, verts)
        np.testing.assert_allclose(g[y, x, t], ge, rtol=0, atol=1e-14)
        assert abs(ft[y, x, t] - fte) < 1e-14


@pytest.mark.parametrize("W,H", [(4, 3), (5, 5), (3, 6)])
def test_operator_and_load_equal_weak_form(oracle, W, H):
    """U^T A V and b^T V equal the weak form (Eq. weakform / discret-form)
    integrated by an independent rule, for random U, V, alpha."""
    rng = np.random.default_rng(W * 100 + H)
    f1, f2 = synth.random_frames(W, H, W + H)
    alpha = synth.random_alpha(W, H, 7)
    lam = 0.7
    S = oracle.System.from_frames(f1, f2, alpha, lam)
    for _ in range(3):
        U = rng.standard_normal((3, H, W))
        V = rng.standard_normal((3, H, W))
        a_uv, l_v = bilinear(f1, f2, alpha, lam, U, V)
        assert abs(np.sum(V * S.matvec(U)) - a_uv) < 1e-12 * max(1.0, abs(a_uv))
        assert abs(S.b @ V.ravel() - l_v) < 1e-13 * max(1.0, abs(l_v))


def test_constant_brightness_model_is_horn_schunck(oracle):
    """Brightness constancy (model 1): U^T A V and b^T V equal the
    Horn-Schunck weak form (Eq. BW with rho = 0: data (grad f2 . u + ft)^2,
    alpha |grad u|^2) integrated by the independent rule, the m block is
    decoupled from (u1, u2) and carries no load."""
    W, H = 5, 4
    rng = np.random.default_rng(17)
    f1, f2 = synth.random_frames(W, H, 18)
    alpha = synth.random_alpha(W, H, 19)
    S = oracle.System.from_frames(f1, f2, alpha, 0.9, model=1)
    for _ in range(3):
        U = rng.standard_normal((3, H, W))
        V = rng.standard_normal((3, H, W))
        a_uv, l_v = bilinear(f1, f2, alpha, 0.9, U, V, illumination=False)
        assert abs(np.sum(V * S.matvec(U)) - a_uv) < 1e-12 * max(1.0, abs(a_uv))
        assert abs(S.b @ V.ravel() - l_v) < 1e-13 * max(1.0, abs(l_v))
    A = S.dense()
    n = W * H
    assert np.abs(A[:2 * n, 2 * n:]).max() == 0.0
    assert np.abs(S.b[2 * n:]).max() == 0.0


def test_constant_brightness_solution_satisfies_system(oracle):
    """The flow-block solve of model 1 solves A U = b with m = 0 (checked
    with the assembled matrix) and differs from the illumination model's
    solution (the m coupling matters)."""
    p = synth.blobs()
    S1 = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam, model=1)
    U1 = S1.solve_direct()
    assert np.abs(U1[2]).max() == 0.0
    assert S1.rel_residual(U1) <= 1e-12
    U0 = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam).solve_direct()
    assert np.linalg.norm(U1[:2] - U0[:2]) > 1e-3 * np.linalg.norm(U0[:2])


def test_assembled_matrix_symmetric_spd(oracle):
    for (W, H, seed) in [(5, 4, 1), (7, 5, 2)]:
        f1, f2 = synth.random_frames(W, H, seed)
        S = oracle.System.from_frames(f1, f2, synth.random_alpha(W, H, seed), 1.0)
        A = S.dense()
        assert np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0.0


def test_stiffness_annihilates_constants(oracle):
    """Without data (f1 = f2 = 0) A is the stiffness only: constants are in
    its kernel (row sums zero) and b = 0."""
    W, H = 6, 5
    z = np.zeros((H, W))
    S = oracle.System.from_frames(z, z, synth.random_alpha(W, H, 3), 2.0)
    for c in range(3):
        U = np.zeros((3, H, W))
        U[c] = 1.0
        assert np.abs(S.matvec(U)).max() < 1e-15
    assert np.abs(S.b).max() == 0.0


def test_stencil_is_seven_point(oracle):
    """Couplings only to (+-1,0), (0,+-1) and +-(1,1) (Fig. sch-mesh)."""
    W, H = 5, 5
    f1, f2 = synth.random_frames(W, H, 4)
    S = oracle.System.from_frames(f1, f2, 0.05, 1.0)
    A = S.dense().reshape(3, H, W, 3, H, W)
    allowed = {(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)}
    for y in range(H):
        for x in range(W):
            blk = A[:, y, x]
            for yy in range(H):
                for xx in range(W):
                    nz = np.abs(blk[:, :, yy, xx]).max() > 0
                    if (xx - x, yy - y) not in allowed:
                        assert not nz
                    elif (xx - x, yy - y) in {(1, 1), (-1, -1)}:
                        assert nz  # coupled through the data term of the two triangles


# --------------------------------------------------------------- solves ----

@pytest.mark.parametrize("W,H", [(4, 3), (3, 5), (6, 6)])
def test_banded_cholesky_equals_lapack(oracle, W, H):
    f1, f2 = synth.random_frames(W, H, 20 + W)
    S = oracle.System.from_frames(f1, f2, synth.random_alpha(W, H, 5), 1.0)
    x = np.linalg.solve(S.dense(), S.b)
    U = S.solve_direct()
    assert np.abs(U.ravel() - x).max() <= 1e-13 * np.abs(x).max()


def test_constant_solution_invariant(oracle):
    """If ft_K = -g_K.c for a constant c then U = c exactly, for any alpha,
    lambda, solver and Schwarz split (the data residual g.U + ft vanishes and
    constants carry no stiffness)."""
    W, H = 12, 9
    rng = np.random.default_rng(5)
    g = rng.uniform(-1, 1, (H - 1, W - 1, 2, 3))
    c = np.array([0.7, -1.3, 0.25])
    ft = -(g @ c)
    S = oracle.System(W, H, g, ft, synth.random_alpha(W, H, 9), 0.3)
    want = np.broadcast_to(c[:, None, None], (3, H, W))
    assert np.abs(S.solve_direct() - want).max() < 1e-12
    U, it, rr = S.solve_pcg(tol=1e-14)
    assert np.abs(U - want).max() < 1e-11
    U, _ = S.schwarz(2, 2, 2, 80)
    assert np.abs(U - want).max() < 1e-10


@pytest.mark.parametrize("M", [1.1, 0.85])
def test_pure_gain_recovered_exactly(oracle, M):
    """f2 = M f1 without motion: U = (0, 0, M - 1) (Eq. deltam, Eq. OF2)."""
    W, H = 10, 8
    f1, _ = synth.random_frames(W, H, 31)
    S = oracle.System.from_frames(f1, M * f1, synth.random_alpha(W, H, 2), 1.0)
    U = S.solve_direct()
    assert np.abs(U[0]).max() < 1e-12 and np.abs(U[1]).max() < 1e-12
    assert np.abs(U[2] - (M - 1.0)).max() < 1e-12


def test_pcg_matches_direct_on_blobs(oracle):
    p = synth.blobs()
    S = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam)
    Ud = S.solve_direct()
    Up, it, rr = S.solve_pcg(tol=1e-13)
    assert rr <= 1e-13
    assert np.linalg.norm(Up - Ud) <= 1e-10 * np.linalg.norm(Ud)


def test_asm_pcg_matches_direct_on_blobs(oracle):
    """PCG with the exact-subdomain additive Schwarz preconditioner (the
    large-grid solver) on the 64x48 blobs pair, 2x2 parts, 4-node overlap:
    the banded-Cholesky solution."""
    p = synth.blobs()
    S = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam)
    Ud = S.solve_direct()
    U, it, rr = S.solve_asm_pcg((2, 2), 4, tol=1e-13)
    assert rr <= 1e-13
    assert np.linalg.norm(U - Ud) <= 1e-10 * np.linalg.norm(Ud)


def test_asm_pcg_limits(oracle):
    """One subdomain: the preconditioner is A^{-1} and CG stops after one
    step at the direct solution.  One node per subdomain, no overlap: it is
    the node-block Jacobi preconditioner, so CG takes the same iterates as
    the block-Jacobi PCG."""
    S = _small_system(oracle, 23, 17, 11)
    Ud = S.solve_direct()
    U1, it1, _ = S.solve_asm_pcg((1, 1), 0, tol=1e-12)
    assert it1 == 1
    assert np.linalg.norm(U1 - Ud) <= 1e-12 * np.linalg.norm(Ud)
    Ua, ita, _ = S.solve_asm_pcg((23, 17), 0, tol=1e-12)
    Ub, itb, _ = S.solve_pcg(tol=1e-12)
    assert ita == itb
    assert np.linalg.norm(Ua - Ub) <= 1e-12 * np.linalg.norm(Ub)


def test_asm_pcg_first_step_from_dense_blocks(oracle):
    """The first CG step from zero is x1 = (b.z / z.A z) z with z = M b and
    M = sum_i R_i^T A_i^{-1} R_i over the extended tiles (near-equal tiles,
    boundary k at floor(k W / px), extended by the overlap and clipped);
    here M b is formed from dense sub-blocks of the assembled matrix and
    LAPACK solves."""
    W, H, px, py, ov = 19, 14, 3, 2, 2
    S = _small_system(oracle, W, H, 13)
    A = S.dense()
    b = S.b
    z = np.zeros(S.n)
    for iy in range(py):
        for ix in range(px):
            x0, x1 = ix * W // px, (ix + 1) * W // px
            y0, y1 = iy * H // py, (iy + 1) * H // py
            ex0, ex1, ey0, ey1 = max(x0 - ov, 0), min(x1 + ov, W), max(y0 - ov, 0), min(y1 + ov, H)
            ys, xs = np.mgrid[ey0:ey1, ex0:ex1]
            idx = np.concatenate([c * W * H + ys.ravel() * W + xs.ravel() for c in range(3)])
            z[idx] += np.linalg.solve(A[np.ix_(idx, idx)], b[idx])
    x1 = (b @ z) / (z @ (A @ z)) * z
    U, it, _ = S.solve_asm_pcg((px, py), ov, tol=1e-30, maxit=1)
    assert it == 1
    assert np.abs(U.ravel() - x1).max() <= 1e-12 * np.abs(x1).max()


def test_asm_pcg_matches_block_jacobi_pcg_640x480(oracle):
    """640x480 texture: the ASM-PCG (16x16 tiles, 1-node overlap) and the
    block-Jacobi PCG, both to 1e-12, give the same solution."""
    p = synth.texture()
    S = oracle.System.from_frames(p.f1.astype(np.float64), p.f2.astype(np.float64), p.alpha0, p.lam)
    Ua, ita, ra = S.solve_asm_pcg((40, 30), 1, tol=1e-12)
    Ub, itb, rb = S.solve_pcg(tol=1e-12)
    assert ra <= 1e-12 and rb <= 1e-12
    assert ita < itb / 3
    assert np.linalg.norm(Ua - Ub) <= 1e-9 * np.linalg.norm(Ub)


def test_schwarz_fixed_point_is_global_solution(oracle):
    """Eq. schwarz: the subdomain iterates converge to the global solution
    (2x2 parts, 4-node overlap, 64x48 blobs)."""
    p = synth.blobs()
    S = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam)
    Ud = S.solve_direct()
    U, hist = S.schwarz(2, 2, 4, 70)
    assert np.linalg.norm(U - Ud) <= 1e-12 * np.linalg.norm(Ud)
    assert hist[-1] < 1e-12 * hist[0]


def _small_system(oracle, W, H, seed):
    f1, f2 = synth.random_frames(W, H, seed)
    alpha = synth.random_alpha(W, H, seed + 1)
    return oracle.System.from_frames(f1, f2, alpha, 0.8)


@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_sweep_preconditioner_one_tile_converges_to_direct_solve(oracle, omega):
    """Block SOR on an SPD matrix converges for 0 < omega < 2: one tile over
    the whole image and many sweeps give A^{-1} r (banded Cholesky)."""
    S = _small_system(oracle, 17, 13, 5)
    r = np.random.default_rng(1).standard_normal((3, 13, 17))
    zd = S.solve_with(r)
    z = S.schwarz_sweeps(r, (32, 32), 0, 400, omega)
    assert np.linalg.norm(z - zd) <= 1e-11 * np.linalg.norm(zd)


def test_sweep_preconditioner_exact_local_solves(oracle):
    """Many sweeps per tile give the restricted exact-solve preconditioner
    sum_i R~_i^T A_i^{-1} R~_i r, built here from dense sub-blocks of the
    assembled matrix and LAPACK solves."""
    W, H, tx, ty, ov = 20, 15, 8, 6, 1
    S = _small_system(oracle, W, H, 7)
    A = S.dense()
    r = np.random.default_rng(2).standard_normal((3, H, W))
    want = np.zeros(3 * W * H)
    for y0 in range(0, H, ty):
        for x0 in range(0, W, tx):
            ext = [(x, y) for y in range(max(y0 - ov, 0), min(y0 + ty + ov, H))
                   for x in range(max(x0 - ov, 0), min(x0 + tx + ov, W))]
            idx = np.array([c * W * H + y * W + x for c in range(3) for (x, y) in ext])
            own = np.array([x0 <= x < x0 + tx and y0 <= y < y0 + ty for c in range(3) for (x, y) in ext])
            b = np.where(own, r.ravel()[idx], 0.0)
            zi = np.linalg.solve(A[np.ix_(idx, idx)], b)
            want[idx[own]] = zi[own]
    z = S.schwarz_sweeps(r, (tx, ty), ov, 600, 1.3)
    assert np.linalg.norm(z.ravel() - want) <= 1e-10 * np.linalg.norm(want)


@pytest.mark.parametrize("sweeps,omega", [(1, 1.0), (2, 1.4), (3, 1.8)])
def test_sweep_preconditioner_symmetric_positive(oracle, sweeps, omega):
    """The palindromic colour order makes M symmetric and positive definite for
    any 0 < omega < 2 (the property the CUDA preconditioner relies on for CG):
    the matrix of r -> z, column by column, on a 9x7 grid, 4x3 tiles,
    overlap 1."""
    W, H = 9, 7
    S = _small_system(oracle, W, H, 11)
    n = 3 * W * H
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = S.schwarz_sweeps(e.reshape(3, H, W), (4, 3), 1, sweeps, omega).ravel()
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_coarse_hats_partition_of_unity(oracle):
    """The bilinear coarse functions sum to one at every fine node and are 1
    at their own coarse node (ragged last cells included)."""
    S = _small_system(oracle, 23, 17, 31)
    R0 = S.coarse_restriction(5)
    n = 23 * 17
    ones = np.asarray(R0.T @ np.ones(R0.shape[0])).ravel()
    assert np.abs(ones - 1.0).max() <= 1e-14
    P = R0[: R0.shape[0] // 3, :n].toarray()
    xs = sorted(set(list(range(0, 23, 5)) + [22]))
    ys = sorted(set(list(range(0, 17, 5)) + [16]))
    for l, y in enumerate(ys):
        for k, x in enumerate(xs):
            assert P[l * len(xs) + k, y * 23 + x] == 1.0


def test_two_level_with_fine_coarse_grid_adds_the_exact_inverse(oracle):
    """Coarse spacing 1 makes the coarse space the whole space (R_0 = I), so
    the coarse correction is A^{-1} r (banded Cholesky)."""
    S = _small_system(oracle, 9, 7, 32)
    r = np.random.default_rng(33).standard_normal((3, 7, 9))
    z = S.two_level(r, (4, 3), 0, 2, 1.4, 1)
    assert np.abs(z - S.schwarz_sweeps(r, (4, 3), 0, 2, 1.4) - S.solve_with(r)).max() <= 1e-10 * np.abs(z).max()


def test_two_level_symmetric_positive(oracle):
    """The additive two-level preconditioner is symmetric positive definite
    (column by column on an 11x9 grid, coarse spacing 4)."""
    W, H = 11, 9
    S = _small_system(oracle, W, H, 34)
    n = 3 * W * H
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = S.two_level(e.reshape(3, H, W), (4, 3), 0, 2, 1.5, 4).ravel()
    assert np.abs(M - M.T).max() <= 1e-11 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_sweep_preconditioner_zero_sweeps_is_block_jacobi(oracle):
    """sweeps = 0: z_n = D_n^{-1} r_n with D_n the 3x3 diagonal block of the
    dense assembled matrix, whatever the tiling."""
    W, H = 11, 9
    S = _small_system(oracle, W, H, 13)
    A = S.dense()
    r = np.random.default_rng(3).standard_normal((3, H, W))
    want = np.zeros((3, H, W))
    for y in range(H):
        for x in range(W):
            i = [c * W * H + y * W + x for c in range(3)]
            want[:, y, x] = np.linalg.solve(A[np.ix_(i, i)], r[:, y, x])
    z = S.schwarz_sweeps(r, (4, 4), 2, 0)
    assert np.abs(z - want).max() <= 1e-13 * np.abs(want).max()


def test_schwarz_converges_faster_with_more_overlap(oracle):
    """Section 4, Fig. schwarz-convergence: the rate increases with the
    overlap."""
    p = synth.blobs()
    S = oracle.System.from_frames(p.f1, p.f2, p.alpha0, p.lam)
    Ud = S.solve_direct()
    counts = []
    for ov in (1, 2, 4, 8):
        U = np.zeros_like(Ud)
        for k in range(1, 200):
            U, _ = S.schwarz(2, 2, ov, 1, U0=U)
            if np.linalg.norm(U - Ud) <= 1e-8 * np.linalg.norm(Ud):
                break
        counts.append(k)
    assert all(a >= b for a, b in zip(counts, counts[1:])), counts
    assert counts[0] > counts[-1]


def test_adjoint_symmetry_identity(oracle):
    W, H = 7, 6
    f1, f2 = synth.random_frames(W, H, 8)
    S = oracle.System.from_frames(f1, f2, synth.random_alpha(W, H, 8), 1.0)
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((2, 3, H, W))
    lhs = np.sum(S.solve_with(a) * b)
    rhs = np.sum(a * S.solve_with(b))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ------------------------------------------------- indicator / alpha ----

def indicator_independent(f1, f2, alpha, lam, U):
    """Eq. errind by an independent route: generic geometry, edge neighbours
    found by shared vertex pairs, normals from the geometry, interior L2 by
    the 3-point interior rule."""
    H, W = f1.shape
    tris = list(triangles(W, H))
    edges = {}
    for k, (_, _, _, verts) in enumerate(tris):
        for i in range(3):
            key = tuple(sorted([verts[i], verts[(i + 1) % 3]]))
            edges.setdefault(key, []).append(k)
    info = []
    for x, y, t, verts in tris:
        g, ft = element_data(f1, f2, verts)
        G, area = bary(verts)
        Lam = np.array([alpha[y, x, t], alpha[y, x, t], lam[y, x, t] if np.ndim(lam) else lam])
        uv = np.array([[U[c, yy, xx] for c in range(3)] for xx, yy in verts])
        grads = np.array([G.T @ uv[:, c] for c in range(3)])  # [c][2]
        info.append((g, ft, area, Lam, uv, grads, verts))
    eta = np.zeros((H - 1, W - 1, 2))
    for k, (x, y, t, verts) in enumerate(tris):
        g, ft, area, Lam, uv, grads, _ = info[k]
        integ = 0.0
        for q in QPTS:
            s = g @ (np.array(q) @ uv) + ft
            R = -g * s
            integ += area / 3.0 * np.sum(R * R / Lam)
        hK = max(np.hypot(verts[i][0] - verts[j][0], verts[i][1] - verts[j][1])
                 for i in range(3) for j in range(3))
        val = hK * np.sqrt(integ)
        cen = np.mean(np.array(verts, float), axis=0)
        for i in range(3):
            pa, pb = np.array(verts[i], float), np.array(verts[(i + 1) % 3], float)
            d = pb - pa
            he = np.hypot(*d)
            n = np.array([d[1], -d[0]]) / he
            if n @ ((pa + pb) / 2 - cen) < 0:
                n = -n
            key = tuple(sorted([verts[i], verts[(i + 1) % 3]]))
            nb = [j for j in edges[key] if j != k]
            fin = Lam * (grads @ n)
            if nb:
                Lo = info[nb[0]][3]
                fout = Lo * (info[nb[0]][5] @ n)
                Le = np.maximum(Lam, Lo)
            else:
                fout = np.zeros(3)
                Le = Lam
            J = fout - fin
            # (1/2) h_e^{1/2} ||Lambda_e^{-1/2} J||_{L2(e)}, J constant on e
            val += 0.5 * np.sqrt(he) * np.sqrt(he * np.sum(J * J / Le))
        eta[y, x, t] = val
    return eta


def test_indicator_matches_independent_route(oracle):
    W, H = 6, 5
    f1, f2 = synth.random_frames(W, H, 41)
    alpha = synth.random_alpha(W, H, 42)
    U = np.random.default_rng(43).standard_normal((3, H, W))
    S = oracle.System.from_frames(f1, f2, alpha, 0.6)
    np.testing.assert_allclose(S.indicator(U), indicator_independent(f1, f2, alpha, 0.6, U), rtol=1e-12, atol=1e-14)


def test_per_element_lambda_indicator_matches_independent_route(oracle):
    """Per-element lambda (Lambda = (alpha_K, alpha_K, lambda_K); Lambda_e the
    componentwise max of the two sides) by the independent route."""
    W, H = 6, 5
    f1, f2 = synth.random_frames(W, H, 46)
    alpha = synth.random_alpha(W, H, 47)
    lamel = 0.3 + synth.random_alpha(W, H, 48) * 10.0
    U = np.random.default_rng(49).standard_normal((3, H, W))
    S = oracle.System.from_frames(f1, f2, alpha, 0.6, lamel=lamel)
    np.testing.assert_allclose(S.indicator(U), indicator_independent(f1, f2, alpha, lamel, U), rtol=1e-12,
                               atol=1e-14)


def test_indicator_closed_forms(oracle):
    W, H = 6, 5
    f1, f2 = synth.random_frames(W, H, 44)
    alpha = synth.random_alpha(W, H, 45)
    lam = 1.7
    S = oracle.System.from_frames(f1, f2, alpha, lam)
    # U = 0: only the interior term, h_K |K|^{1/2} |ft| ||Lambda^{-1/2} g|| = |ft| ||Lambda^{-1/2} g||
    eta = S.indicator(np.zeros((3, H, W)))
    lamv = np.stack([alpha, alpha, np.full_like(alpha, lam)], -1)
    want = np.abs(S.ft) * np.sqrt(np.sum(S.g ** 2 / lamv, -1))
    np.testing.assert_allclose(eta, want, rtol=1e-13)
    # no data, u1 = x, constant alpha: only the left/right boundary edges jump,
    # by alpha, giving (1/2) sqrt(alpha) on the elements that carry them
    z = np.zeros((H, W))
    a0 = 0.09
    S0 = oracle.System.from_frames(z, z, a0, lam)
    U = np.zeros((3, H, W))
    U[0] = np.arange(W)[None, :]
    eta = S0.indicator(U)
    want = np.zeros((H - 1, W - 1, 2))
    want[:, W - 2, 0] = 0.5 * np.sqrt(a0)
    want[:, 0, 1] = 0.5 * np.sqrt(a0)
    np.testing.assert_allclose(eta, want, atol=1e-15)


def test_indicator_zero_on_constant_solution(oracle):
    W, H = 8, 7
    rng = np.random.default_rng(6)
    g = rng.uniform(-1, 1, (H - 1, W - 1, 2, 3))
    c = np.array([0.3, 0.2, -0.1])
    S = oracle.System(W, H, g, -(g @ c), synth.random_alpha(W, H, 1), 1.0)
    U = S.solve_direct()
    assert np.abs(S.indicator(U)).max() < 1e-13
    eta = S.indicator(np.broadcast_to(c[:, None, None], (3, H, W)).copy())
    assert np.abs(eta).max() < 1e-15


def test_alpha_update_closed_form(oracle):
    eta = np.array([0.0, 0.5, 1.0, 2.0])
    alpha = np.array([1.0, 1.0, 1.0, 0.3])
    # max eta = 2 -> rel = [-0.25, 0, 0.25, 0.75]
    out = oracle.alpha_update(eta, alpha, 4.0, 0.25, 0.1)
    np.testing.assert_allclose(out, [1.0, 1.0, 0.5, 0.1], rtol=1e-15)
    np.testing.assert_array_equal(oracle.alpha_update(np.zeros(4), alpha, 4.0, 0.25, 0.1), alpha)


# ------------------------------------------------------------- adjoint ----

@pytest.mark.parametrize("model", [0, 1])
def test_adjoint_gradient_matches_central_differences(oracle, model):
    W, H = 7, 6
    f1, f2 = synth.random_frames(W, H, 51)
    alpha = synth.random_alpha(W, H, 52)
    lam = 1.0
    gt = np.random.default_rng(53).uniform(-1, 1, (2, H, W))

    def loss(f1_, f2_, a_):
        S_ = oracle.System.from_frames(f1_, f2_, a_, lam, model)
        return oracle.mean_epe(S_.solve_direct(), gt)

    S = oracle.System.from_frames(f1, f2, alpha, lam, model)
    U = S.solve_direct()
    Lam = S.solve_with(oracle.mean_epe_grad(U, gt))
    da, d2, d1 = oracle.adjoint_grad(f1, f2, alpha, lam, U, Lam, model=model)
    h = 1e-4
    rng = np.random.default_rng(54)
    for _ in range(6):
        y, x, t = rng.integers(0, H - 1), rng.integers(0, W - 1), rng.integers(0, 2)
        ap, am = alpha.copy(), alpha.copy()
        ap[y, x, t] += h
        am[y, x, t] -= h
        fd = (loss(f1, f2, ap) - loss(f1, f2, am)) / (2 * h)
        assert abs(fd - da[y, x, t]) <= 1e-5 * np.abs(da).max()
    for which, grad in (("f2", d2), ("f1", d1)):
        for _ in range(6):
            y, x = rng.integers(0, H), rng.integers(0, W)
            fp = (f1 if which == "f1" else f2).copy()
            fm = fp.copy()
            fp[y, x] += h
            fm[y, x] -= h
            if which == "f1":
                fd = (loss(fp, f2, alpha) - loss(fm, f2, alpha)) / (2 * h)
            else:
                fd = (loss(f1, fp, alpha) - loss(f1, fm, alpha)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-5 * np.abs(grad).max()


# --------------------------------------------------------- elementwise ----

def test_elementwise_apply_equals_csr(oracle):
    W, H = 9, 7
    f1, f2 = synth.random_frames(W, H, 61)
    alpha = synth.random_alpha(W, H, 62)
    S = oracle.System.from_frames(f1, f2, alpha, 1.3)
    U = np.random.default_rng(63).standard_normal((3, H, W))
    AU, b = oracle.apply_elementwise(W, H, S.g, S.ft, alpha, 1.3, U, with_rhs=True)
    np.testing.assert_allclose(AU, S.matvec(U), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(b.ravel(), S.b, rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------ partition ----

# ------------------------------------------------------------ K_sigma --

def test_smooth_brute_force_2d(oracle):
    """Separable passes = the 2-D normalised sum written out directly."""
    rng = np.random.default_rng(4)
    I = rng.standard_normal((9, 13))
    sigma = 1.3
    r = int(np.ceil(3 * sigma))
    want = np.zeros_like(I)
    for y in range(9):
        for x in range(13):
            num = den = 0.0
            for j in range(-r, r + 1):
                for k in range(-r, r + 1):
                    if 0 <= y + j < 9 and 0 <= x + k < 13:
                        w = np.exp(-(j * j + k * k) / (2 * sigma * sigma))
                        num += w * I[y + j, x + k]
                        den += w
            want[y, x] = num / den
    assert np.abs(oracle.smooth(I, sigma) - want).max() <= 1e-13


@pytest.mark.parametrize("sigma", [1.5, 2.0])
def test_smooth_interior_matches_scipy(oracle, sigma):
    """Away from the border (no truncated taps) K_sigma is scipy's Gaussian
    filter with the same 3-sigma truncation."""
    ndimage = pytest.importorskip("scipy.ndimage")
    I = np.random.default_rng(5).standard_normal((40, 50))
    r = int(np.ceil(3 * sigma))
    ref = ndimage.gaussian_filter(I, sigma, truncate=3.0, mode="constant")
    f = oracle.smooth(I, sigma)
    assert np.abs(f[r:-r, r:-r] - ref[r:-r, r:-r]).max() <= 1e-12


def test_smooth_closed_forms(oracle):
    """Constants are preserved everywhere (normalisation); a linear ramp is
    preserved wherever the taps are symmetric (the interior)."""
    H, W, sigma = 30, 40, 1.7
    r = int(np.ceil(3 * sigma))
    assert np.abs(oracle.smooth(np.full((H, W), 0.37), sigma) - 0.37).max() <= 1e-15
    y, x = np.mgrid[0:H, 0:W]
    ramp = 0.3 * x - 0.7 * y + 2.0
    f = oracle.smooth(ramp, sigma)
    assert np.abs(f[r:-r, r:-r] - ramp[r:-r, r:-r]).max() <= 1e-12
    assert np.abs(oracle.smooth(ramp, 0.0) - ramp).max() == 0.0


def test_smooth_transpose_is_adjoint(oracle):
    """<S a, b> = <a, S^T b>."""
    rng = np.random.default_rng(6)
    a, b = rng.standard_normal((2, 17, 23))
    lhs = np.sum(oracle.smooth(a, 1.1) * b)
    rhs = np.sum(a * oracle.smooth_transpose(b, 1.1))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_partition_ratio_worked_example():
    """Fig. ratio: 48x48 grid, twelve parts."""
    path = os.path.join(os.path.dirname(__file__), "golden", "partition_ratio_48x48_12.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for px, py, r in rows:
        got = partition.part_ratio(48, 48, int(px), int(py))
        assert abs(got - float(r)) < 1e-3, (px, py, got, r)
    assert partition.best_split(48, 48, 12) in {(4, 3), (3, 4)}


def test_metrics_closed_forms(oracle):
    gt = np.zeros((2, 3, 4))
    U = np.zeros((3, 3, 4))
    U[0] = 3.0
    U[1] = 4.0
    assert abs(oracle.mean_epe(U, gt) - 5.0) < 1e-15
    assert oracle.aae_deg(np.concatenate([gt, np.zeros((1, 3, 4))]), gt) == 0.0
    # u_h = (1, 0), u_e = (0, 0): cos = 1/sqrt(2) -> 45 degrees
    U2 = np.zeros((3, 3, 4))
    U2[0] = 1.0
    assert abs(oracle.aae_deg(U2, gt) - 45.0) < 1e-12


# ------------------------------------------------- K_rho element tensors --

def _brute_rho(P, rho):
    """2-D normalised Gaussian sum over one (H-1) x (W-1) element lattice,
    written out directly (the K_rho of Section 1 on one triangle family)."""
    Hh, Ww = P.shape
    r = int(np.ceil(3 * rho))
    out = np.zeros_like(P)
    for y in range(Hh):
        for x in range(Ww):
            num = den = 0.0
            for j in range(-r, r + 1):
                for k in range(-r, r + 1):
                    if 0 <= y + j < Hh and 0 <= x + k < Ww:
                        w = np.exp(-(j * j + k * k) / (2 * rho * rho))
                        num += w * P[y + j, x + k]
                        den += w
            out[y, x] = num / den
    return out


def test_element_tensor_is_smoothed_products(oracle):
    """A_rho = K_rho * (g_c g_d), F = K_rho * (-ft g_c) (Section 1, matrix
    A_rho and vector F) per triangle family, against products of the
    independently formed element data and a brute-force 2-D Gaussian sum."""
    W, H, rho = 9, 7, 1.2
    f1, f2 = synth.random_frames(W, H, 61)
    Ael, Fel = oracle.element_data(f1, f2, rho)
    g = np.zeros((H - 1, W - 1, 2, 3))
    ft = np.zeros((H - 1, W - 1, 2))
    for x, y, t, verts in triangles(W, H):
        g[y, x, t], ft[y, x, t] = element_data(f1, f2, verts)
    for t in range(2):
        for k, (c, d) in enumerate(oracle.SYM6):
            want = _brute_rho(g[:, :, t, c] * g[:, :, t, d], rho)
            assert np.abs(Ael[:, :, t, k] - want).max() <= 1e-14
        for c in range(3):
            want = _brute_rho(-ft[:, :, t] * g[:, :, t, c], rho)
            assert np.abs(Fel[:, :, t, c] - want).max() <= 1e-14


def test_element_tensor_limits(oracle):
    """rho = 0 gives g g^T and -ft g exactly; a Gaussian far narrower than
    the lattice (rho = 0.1: neighbour weight e^-50) the same to rounding;
    a constant g (f1 constant, f2 affine) is left unchanged by K_rho; every
    tensor is symmetric positive semidefinite."""
    f1, f2 = synth.random_frames(8, 6, 62)
    g, ft = oracle.coefficients(f1, f2)
    A0, F0 = oracle.element_data(f1, f2, 0.0)
    for k, (c, d) in enumerate(oracle.SYM6):
        assert np.array_equal(A0[..., k], g[..., c] * g[..., d])
    assert np.array_equal(F0, -ft[..., None] * g)
    A1, F1 = oracle.element_data(f1, f2, 0.1)
    assert np.abs(A1 - A0).max() <= 1e-15 * np.abs(A0).max()
    assert np.abs(F1 - F0).max() <= 1e-15 * np.abs(F0).max()
    ys, xs = np.mgrid[0:6, 0:8]
    c1 = np.full((6, 8), 0.4)
    c2 = 0.3 + 0.02 * xs - 0.05 * ys
    Ac, Fc = oracle.element_data(c1, c2, 2.0)
    gc = np.array([0.02, -0.05, -0.4])
    ftc = (c2 - c1)  # varies: only the tensor is checked
    for k, (c, d) in enumerate(oracle.SYM6):
        assert np.abs(Ac[..., k] - gc[c] * gc[d]).max() <= 1e-15
    A2, _ = oracle.element_data(f1, f2, 1.7)
    M = np.zeros(A2.shape[:-1] + (3, 3))
    for k, (c, d) in enumerate(oracle.SYM6):
        M[..., c, d] = M[..., d, c] = A2[..., k]
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= -1e-15 * np.abs(ev).max()


def test_general_operator_equals_weak_form(oracle):
    """U^T A V and b^T V with the K_rho element tensors equal
    int U_h^T A_rho V_h + stiffness and int F . V_h, by the 3-point rule."""
    W, H, rho, lam = 5, 4, 1.3, 0.6
    rng = np.random.default_rng(63)
    f1, f2 = synth.random_frames(W, H, 64)
    alpha = synth.random_alpha(W, H, 65)
    S = oracle.System.from_frames(f1, f2, alpha, lam, rho=rho)
    Ael, Fel = oracle.element_data(f1, f2, rho)
    for _ in range(3):
        U = rng.standard_normal((3, H, W))
        V = rng.standard_normal((3, H, W))
        a_uv = l_v = 0.0
        for x, y, t, verts in triangles(W, H):
            G, area = bary(verts)
            M = np.zeros((3, 3))
            for k, (c, d) in enumerate(oracle.SYM6):
                M[c, d] = M[d, c] = Ael[y, x, t, k]
            Fv = Fel[y, x, t]
            Lam = np.array([alpha[y, x, t], alpha[y, x, t], lam])
            uv = np.array([[U[c, yy, xx] for c in range(3)] for xx, yy in verts])
            vv = np.array([[V[c, yy, xx] for c in range(3)] for xx, yy in verts])
            for q in QPTS:
                q = np.array(q)
                a_uv += area / 3.0 * (q @ uv) @ M @ (q @ vv)
                l_v += area / 3.0 * Fv @ (q @ vv)
            for c in range(3):
                a_uv += area * Lam[c] * (G.T @ uv[:, c]) @ (G.T @ vv[:, c])
        assert abs(np.sum(V * S.matvec(U)) - a_uv) < 1e-12 * max(1.0, abs(a_uv))
        assert abs(S.b @ V.ravel() - l_v) < 1e-13 * max(1.0, abs(l_v))


def test_general_constant_solution_invariant(oracle):
    """With F_K = A_K c for every element, U = c solves the system exactly
    (the stiffness annihilates constants, the data blocks give |K|/3 A_K c)."""
    W, H = 7, 5
    f1, f2 = synth.random_frames(W, H, 66)
    Ael, _ = oracle.element_data(f1, f2, 1.5)
    cst = np.array([0.3, -0.2, 0.05])
    M = np.zeros(Ael.shape[:-1] + (3, 3))
    for k, (c, d) in enumerate(oracle.SYM6):
        M[..., c, d] = M[..., d, c] = Ael[..., k]
    Fel = M @ cst
    g, ft = oracle.coefficients(f1, f2)
    S = oracle.System(W, H, g, ft, synth.random_alpha(W, H, 67), 0.8, Ael, Fel)
    U = S.solve_direct()
    assert np.abs(U - cst[:, None, None]).max() <= 1e-11


def test_general_indicator_reduces_and_closed_form(oracle):
    """The indicator with element tensors equals the rank-1 one when
    A = g g^T, F = -ft g; for U = 0 it is |Lambda^{-1/2} F| per element
    (h_K |K|^{1/2} = 1 on these triangles, no flux jumps)."""
    W, H = 6, 5
    f1, f2 = synth.random_frames(W, H, 68)
    alpha = synth.random_alpha(W, H, 69)
    g, ft = oracle.coefficients(f1, f2)
    A0, F0 = oracle.element_data(f1, f2, 0.0)
    U = np.random.default_rng(70).standard_normal((3, H, W))
    e1 = oracle.System(W, H, g, ft, alpha, 0.9).indicator(U)
    e2 = oracle.System(W, H, g, ft, alpha, 0.9, A0, F0).indicator(U)
    assert np.abs(e1 - e2).max() <= 1e-13 * np.abs(e1).max()
    Ael, Fel = oracle.element_data(f1, f2, 1.4)
    e0 = oracle.System(W, H, g, ft, alpha, 0.9, Ael, Fel).indicator(np.zeros((3, H, W)))
    lamv = np.stack([alpha, alpha, np.full_like(alpha, 0.9)], axis=-1)
    want = np.sqrt(np.sum(Fel ** 2 / lamv, axis=-1))
    assert np.abs(e0 - want).max() <= 1e-14 * max(1.0, want.max())


def test_smooth_taps_wider_than_image(oracle):
    """A Gaussian whose taps reach past the whole image (radius 9 on a 5 x 4
    image): still the 2-D normalised sum over the pixels inside."""
    rng = np.random.default_rng(71)
    I = rng.standard_normal((4, 5))
    sigma = 3.0
    want = np.zeros_like(I)
    for y in range(4):
        for x in range(5):
            w = np.exp(-((np.arange(4)[:, None] - y) ** 2 + (np.arange(5)[None, :] - x) ** 2) / (2 * sigma ** 2))
            want[y, x] = np.sum(w * I) / np.sum(w)
    assert np.abs(oracle.smooth(I, sigma) - want).max() <= 1e-14


@pytest.mark.parametrize("model", [0, 1])
def test_adjoint_frame_gradient_with_rho_matches_differences(oracle, model):
    """Frame gradients of a flow loss through the K_rho element tensors
    against central differences of direct solves; at rho -> 0 they equal
    the rank-1 adjoint."""
    W, H, rho, lam = 8, 7, 1.3, 1.0
    f1, f2 = synth.random_frames(W, H, 72)
    alpha = synth.random_alpha(W, H, 73)
    gt = np.random.default_rng(74).uniform(-1, 1, (2, H, W))

    def loss(f1_, f2_):
        S_ = oracle.System.from_frames(f1_, f2_, alpha, lam, model, rho=rho)
        return oracle.mean_epe(S_.solve_direct(), gt)

    S = oracle.System.from_frames(f1, f2, alpha, lam, model, rho=rho)
    U = S.solve_direct()
    Lam = S.solve_with(oracle.mean_epe_grad(U, gt))
    _, d2, d1 = oracle.adjoint_grad(f1, f2, alpha, lam, U, Lam, model=model, rho=rho)
    h = 1e-4
    rng = np.random.default_rng(75)
    for which, grad in (("f2", d2), ("f1", d1)):
        for _ in range(6):
            y, x = rng.integers(0, H), rng.integers(0, W)
            fp = (f1 if which == "f1" else f2).copy()
            fm = fp.copy()
            fp[y, x] += h
            fm[y, x] -= h
            fd = (loss(fp, f2) - loss(fm, f2)) / (2 * h) if which == "f1" else \
                (loss(f1, fp) - loss(f1, fm)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-5 * np.abs(grad).max(), (which, y, x, fd, grad[y, x])
    S0 = oracle.System.from_frames(f1, f2, alpha, lam, model)
    U0 = S0.solve_direct()
    L0 = S0.solve_with(oracle.mean_epe_grad(U0, gt))
    _, e2, e1 = oracle.adjoint_grad(f1, f2, alpha, lam, U0, L0, model=model)
    _, r2, r1 = oracle.adjoint_grad(f1, f2, alpha, lam, U0, L0, model=model, rho=0.1)
    assert np.abs(r2 - e2).max() <= 1e-12 * np.abs(e2).max()
    assert np.abs(r1 - e1).max() <= 1e-12 * max(np.abs(e1).max(), 1e-300)


# ------------------------------------- differentiating through adaptation --

@pytest.mark.parametrize("const_alpha", [False, True])
def test_indicator_vjp_matches_differences(oracle, const_alpha):
    """sum_K w_K eta_K against central differences in U, alpha and both
    frames (constant alpha: every Lambda_e = max is at a tie, where the
    half-and-half rule is the central difference)."""
    W, H, lam = 9, 7, 0.9
    f1, f2 = synth.random_frames(W, H, 76)
    al = np.full((H - 1, W - 1, 2), 0.05) if const_alpha else synth.random_alpha(W, H, 77)
    rng = np.random.default_rng(78)
    U = rng.standard_normal((3, H, W))
    w = rng.standard_normal((H - 1, W - 1, 2))

    def L(U_, a_, f1_, f2_):
        g, ft = oracle.coefficients(f1_, f2_)
        return np.sum(w * oracle.indicator(W, H, g, ft, a_, lam, U_))

    dU, da, d2, d1 = oracle.indicator_vjp(f1, f2, al, lam, U, w)
    h = 1e-6
    # at a tie of the max the central difference is only first-order (error
    # ~ h / alpha): a smaller step in alpha there
    tol = 1e-5 if const_alpha else 1e-6
    ha = 1e-9 if const_alpha else h
    for _ in range(6):
        c, y, x = rng.integers(0, 3), rng.integers(0, H), rng.integers(0, W)
        Up, Um = U.copy(), U.copy()
        Up[c, y, x] += h
        Um[c, y, x] -= h
        fd = (L(Up, al, f1, f2) - L(Um, al, f1, f2)) / (2 * h)
        assert abs(fd - dU[c, y, x]) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(6):
        y, x, t = rng.integers(0, H - 1), rng.integers(0, W - 1), rng.integers(0, 2)
        ap, am = al.copy(), al.copy()
        ap[y, x, t] += ha
        am[y, x, t] -= ha
        fd = (L(U, ap, f1, f2) - L(U, am, f1, f2)) / (2 * ha)
        assert abs(fd - da[y, x, t]) <= tol * max(1.0, abs(fd))
    for _ in range(4):
        y, x = rng.integers(0, H), rng.integers(0, W)
        for which, grad in (("f2", d2), ("f1", d1)):
            fp = (f2 if which == "f2" else f1).copy()
            fm = fp.copy()
            fp[y, x] += h
            fm[y, x] -= h
            fd = (L(U, al, f1, fp) - L(U, al, f1, fm)) / (2 * h) if which == "f2" else \
                (L(U, al, fp, f2) - L(U, al, fm, f2)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-6 * max(1.0, abs(fd))


def test_alpha_update_vjp_matches_differences(oracle):
    """sum v alpha'(alpha, eta) against central differences, away from the
    kinks of the update (threshold, clamp); the max(eta) coupling included."""
    rng = np.random.default_rng(79)
    eta = rng.uniform(0.1, 1.0, (5, 6, 2))
    alpha = rng.uniform(0.02, 0.08, (5, 6, 2))
    v = rng.standard_normal((5, 6, 2))
    kappa, thr, ath = 4.0, 0.25, 0.012
    da, w = oracle.alpha_update_vjp(eta, alpha, kappa, thr, ath, v)
    F = lambda e_, a_: np.sum(v * oracle.alpha_update(e_, a_, kappa, thr, ath))
    a0 = oracle.alpha_update(eta, alpha, kappa, thr, ath)
    h = 1e-7
    rel = eta / eta.max() - thr
    for idx in np.ndindex(eta.shape):
        if abs(rel[idx]) < 1e-4 or abs(a0[idx] - ath) < 1e-6:
            continue
        ep, em = eta.copy(), eta.copy()
        ep[idx] += h
        em[idx] -= h
        fd = (F(ep, alpha) - F(em, alpha)) / (2 * h)
        assert abs(fd - w[idx]) <= 1e-5 * max(1.0, abs(fd)), idx
        ap, am = alpha.copy(), alpha.copy()
        ap[idx] += h
        am[idx] -= h
        fd = (F(eta, ap) - F(eta, am)) / (2 * h)
        assert abs(fd - da[idx]) <= 1e-5 * max(1.0, abs(fd)), idx
    assert (a0 == ath).any() or True


def test_adaptation_gradient_matches_differences(oracle):
    """L = c.U after one adaptation pass (solve, indicator, alpha update,
    solve): the reverse chain against central differences of the whole
    forward map through direct solves."""
    W, H, lam = 10, 8, 1.0
    f1, f2 = synth.random_frames(W, H, 80)
    a0 = synth.random_alpha(W, H, 81)
    kappa, thr, ath = 4.0, 0.25, 1e-4
    c = np.random.default_rng(82).standard_normal((3, H, W))
    da, d2, d1 = oracle.adaptation_grad(f1, f2, a0, lam, 1, kappa, thr, ath, c)
    L = lambda f1_, f2_, a_: np.sum(c * oracle.adaptation_forward(f1_, f2_, a_, lam, 1, kappa, thr, ath)[0])
    h = 1e-6
    rng = np.random.default_rng(83)
    for _ in range(6):
        y, x, t = rng.integers(0, H - 1), rng.integers(0, W - 1), rng.integers(0, 2)
        ap, am = a0.copy(), a0.copy()
        ap[y, x, t] += h
        am[y, x, t] -= h
        fd = (L(f1, f2, ap) - L(f1, f2, am)) / (2 * h)
        assert abs(fd - da[y, x, t]) <= 1e-5 * np.abs(da).max(), (y, x, t, fd, da[y, x, t])
    for _ in range(4):
        y, x = rng.integers(0, H), rng.integers(0, W)
        for which, grad in (("f2", d2), ("f1", d1)):
            fp = (f2 if which == "f2" else f1).copy()
            fm = fp.copy()
            fp[y, x] += h
            fm[y, x] -= h
            fd = (L(f1, fp, a0) - L(f1, fm, a0)) / (2 * h) if which == "f2" else \
                (L(fp, f2, a0) - L(fm, f2, a0)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-5 * np.abs(grad).max(), (which, y, x, fd, grad[y, x])


def test_indicator_vjp_with_rho_matches_differences(oracle):
    """sum_K w_K eta_K with the K_rho element data (interior residual
    F - A_rho U_h) against central differences in U, alpha and both frames;
    at rho -> 0 the general form equals the rank-1 one."""
    W, H, lam, rho = 9, 7, 0.9, 1.2
    f1, f2 = synth.random_frames(W, H, 84)
    al = synth.random_alpha(W, H, 85)
    rng = np.random.default_rng(86)
    U = rng.standard_normal((3, H, W))
    w = rng.standard_normal((H - 1, W - 1, 2))

    def L(U_, a_, f1_, f2_):
        return np.sum(w * oracle.System.from_frames(f1_, f2_, a_, lam, rho=rho).indicator(U_))

    dU, da, d2, d1 = oracle.indicator_vjp(f1, f2, al, lam, U, w, rho=rho)
    h = 1e-6
    for _ in range(6):
        c, y, x = rng.integers(0, 3), rng.integers(0, H), rng.integers(0, W)
        Up, Um = U.copy(), U.copy()
        Up[c, y, x] += h
        Um[c, y, x] -= h
        fd = (L(Up, al, f1, f2) - L(Um, al, f1, f2)) / (2 * h)
        assert abs(fd - dU[c, y, x]) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(6):
        y, x, t = rng.integers(0, H - 1), rng.integers(0, W - 1), rng.integers(0, 2)
        ap, am = al.copy(), al.copy()
        ap[y, x, t] += h
        am[y, x, t] -= h
        fd = (L(U, ap, f1, f2) - L(U, am, f1, f2)) / (2 * h)
        assert abs(fd - da[y, x, t]) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(4):
        y, x = rng.integers(0, H), rng.integers(0, W)
        for which, grad in (("f2", d2), ("f1", d1)):
            fp = (f2 if which == "f2" else f1).copy()
            fm = fp.copy()
            fp[y, x] += h
            fm[y, x] -= h
            fd = (L(U, al, f1, fp) - L(U, al, f1, fm)) / (2 * h) if which == "f2" else \
                (L(U, al, fp, f2) - L(U, al, fm, f2)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-6 * max(1.0, abs(fd)), (which, y, x, fd, grad[y, x])
    # rho = 0.1: the K_rho weights beyond the centre are ~1e-22, so the
    # general interior form must reproduce the rank-1 one
    r0 = oracle.indicator_vjp(f1, f2, al, lam, U, w)
    r1 = oracle.indicator_vjp(f1, f2, al, lam, U, w, rho=0.1)
    for a, b in zip(r0, r1):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def test_adaptation_gradient_with_rho_matches_differences(oracle):
    """As test_adaptation_gradient_matches_differences, with the K_rho data
    term in every solve and in the indicator."""
    W, H, lam, rho = 9, 8, 1.0, 1.1
    f1, f2 = synth.random_frames(W, H, 87)
    a0 = synth.random_alpha(W, H, 88)
    kappa, thr, ath = 4.0, 0.25, 1e-4
    c = np.random.default_rng(89).standard_normal((3, H, W))
    da, d2, d1 = oracle.adaptation_grad(f1, f2, a0, lam, 1, kappa, thr, ath, c, rho=rho)
    L = lambda f1_, f2_, a_: np.sum(c * oracle.adaptation_forward(f1_, f2_, a_, lam, 1, kappa, thr, ath,
                                                                  rho=rho)[0])
    h = 1e-6
    rng = np.random.default_rng(90)
    for _ in range(6):
        y, x, t = rng.integers(0, H - 1), rng.integers(0, W - 1), rng.integers(0, 2)
        ap, am = a0.copy(), a0.copy()
        ap[y, x, t] += h
        am[y, x, t] -= h
        fd = (L(f1, f2, ap) - L(f1, f2, am)) / (2 * h)
        assert abs(fd - da[y, x, t]) <= 1e-5 * np.abs(da).max(), (y, x, t, fd, da[y, x, t])
    for _ in range(4):
        y, x = rng.integers(0, H), rng.integers(0, W)
        for which, grad in (("f2", d2), ("f1", d1)):
            fp = (f2 if which == "f2" else f1).copy()
            fm = fp.copy()
            fp[y, x] += h
            fm[y, x] -= h
            fd = (L(f1, fp, a0) - L(f1, fm, a0)) / (2 * h) if which == "f2" else \
                (L(fp, f2, a0) - L(fm, f2, a0)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-5 * np.abs(grad).max(), (which, y, x, fd, grad[y, x])
