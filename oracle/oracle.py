"""ctypes shim of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle defines what the CUDA library must
compute; it shares no code with it.  Only the tests, the package's smoke
check and the CPU-baseline leg of the benchmark may import this module.

Layouts: frames [H][W]; per-element arrays [H-1][W-1][2] (two triangles per
pixel square, t=0 below the (x,y)->(x+1,y+1) diagonal); vectors [3][H][W]
(u1, u2, m).  Everything is float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = ctypes.CDLL(_LIB)
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.orc_coefficients.argtypes = [i32, i32, _f64p, _f64p, _f64p, _f64p]
        L.orc_csr_nnz.argtypes = [i32, i32]
        L.orc_csr_nnz.restype = i64
        L.orc_csr_pattern.argtypes = [i32, i32, _i64p, _i64p]
        vp = ctypes.c_void_p
        L.orc_assemble.argtypes = [i32, i32, _f64p, _f64p, _f64p, f64, vp, _i64p, _i64p, _f64p, _f64p]
        L.orc_assemble_el.argtypes = [i32, i32, _f64p, _f64p, _f64p, f64, vp, _i64p, _i64p, _f64p, _f64p]
        L.orc_csr_matvec.argtypes = [i64, _i64p, _i64p, _f64p, _f64p, _f64p]
        L.orc_csr_matvec.restype = None
        L.orc_apply_elementwise.argtypes = [i32, i32, _f64p, _f64p, _f64p, f64, vp, _f64p, _f64p, ctypes.c_void_p]
        L.orc_band_cholesky_solve.argtypes = [i32, i32, _i64p, _i64p, _f64p, _f64p, _f64p]
        L.orc_pcg.argtypes = [i32, i32, _i64p, _i64p, _f64p, _f64p, _f64p, f64, i32, ctypes.POINTER(f64)]
        L.orc_asm_pcg.argtypes = [i32, i32, _i64p, _i64p, _f64p, _f64p, _f64p, i32, i32, i32, f64, i32,
                                  ctypes.POINTER(f64)]
        L.orc_schwarz.argtypes = [i32, i32, _i64p, _i64p, _f64p, _f64p, i32, i32, i32, i32, _f64p, ctypes.c_void_p]
        L.orc_indicator.argtypes = [i32, i32, _f64p, _f64p, _f64p, f64, vp, _f64p, _f64p]
        L.orc_indicator_el.argtypes = [i32, i32, _f64p, _f64p, _f64p, f64, vp, _f64p, _f64p]
        L.orc_alpha_update.argtypes = [i64, _f64p, _f64p, f64, f64, f64]
        L.orc_adjoint_grad.argtypes = [i32, i32, _f64p, _f64p, _f64p, f64, _f64p, _f64p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, i32]
        L.orc_num_threads.restype = i32
        _lib = L
        return L


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def coefficients(f1, f2, model=0):
    """(g [H-1][W-1][2][3], ft [H-1][W-1][2]) of every element.  model 1 is
    brightness constancy (Horn and Schunck, Eq. BW without m): the
    illumination column g_m of the data term is dropped."""
    L = _load()
    f1, f2 = _c(f1), _c(f2)
    H, W = f1.shape
    g = np.zeros((H - 1, W - 1, 2, 3))
    ft = np.zeros((H - 1, W - 1, 2))
    if L.orc_coefficients(W, H, f1, f2, g, ft):
        raise ValueError("grid must be at least 2x2")
    if model == 1:
        g[..., 2] = 0.0
    return g, ft


# index pairs (c, d) of the 6 stored entries of a symmetric 3x3 element tensor
SYM6 = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def element_data(f1, f2, rho, model=0):
    """Element tensor A_rho and load vector F of every element (Section 1:
    the matrix A_rho and the vector F, whose entries are K_rho applied to
    the products f_x^2, f_x f_y, -f_x f, ... and -f_x f_t, -f_y f_t, f f_t).
    With g = (f_x, f_y, -f) this is A_rho = K_rho * (g g^T), F = K_rho * (-ft g).
    K_rho is the normalised sampled Gaussian of `smooth` applied to each
    product over the (W-1) x (H-1) lattice of one triangle family (t = 0 and
    t = 1 separately).  Returns Ael [H-1][W-1][2][6] (entries SYM6) and
    Fel [H-1][W-1][2][3]; rho = 0 gives g g^T and -ft g exactly."""
    g, ft = coefficients(f1, f2, model)
    Ael = np.stack([g[..., c] * g[..., d] for c, d in SYM6], axis=-1)
    Fel = -ft[..., None] * g
    if rho > 0:
        for t in range(2):
            for k in range(6):
                Ael[:, :, t, k] = smooth(Ael[:, :, t, k], rho)
            for k in range(3):
                Fel[:, :, t, k] = smooth(Fel[:, :, t, k], rho)
    return Ael, Fel


class System:
    """The assembled FP64 system A U = b of one frame pair (CSR, [3][H][W]
    unknown ordering).  With element tensors Ael, Fel (K_rho > 0) the data
    term uses them in place of g g^T and -ft g; g, ft are still kept (the
    preconditioner of the CUDA path is built from them)."""

    def __init__(self, W, H, g, ft, alpha, lam, Ael=None, Fel=None, lamel=None):
        L = _load()
        self.W, self.H, self.lam = int(W), int(H), float(lam)
        self.g, self.ft, self.alpha = _c(g), _c(ft), _c(alpha)
        # per-element lambda [H-1][W-1][2] (None: the constant lam everywhere)
        self.lamel = None if lamel is None else _c(np.broadcast_to(np.asarray(lamel, dtype=np.float64),
                                                                    (H - 1, W - 1, 2)))
        self.Ael = None if Ael is None else _c(Ael)
        self.Fel = None if Fel is None else _c(Fel)
        n = 3 * W * H
        nnz = int(L.orc_csr_nnz(W, H))
        self.rowptr = np.zeros(n + 1, dtype=np.int64)
        self.col = np.zeros(nnz, dtype=np.int64)
        self.val = np.zeros(nnz)
        self.b = np.zeros(n)
        L.orc_csr_pattern(W, H, self.rowptr, self.col)
        if self.Ael is None:
            rc = L.orc_assemble(W, H, self.g, self.ft, self.alpha, self.lam, _ptr(self.lamel), self.rowptr,
                                self.col, self.val, self.b)
        else:
            rc = L.orc_assemble_el(W, H, self.Ael, self.Fel, self.alpha, self.lam, _ptr(self.lamel), self.rowptr,
                                   self.col, self.val, self.b)
        if rc:
            raise RuntimeError(f"oracle assembly failed ({rc})")

    @classmethod
    def from_frames(cls, f1, f2, alpha, lam, model=0, rho=0.0, lamel=None):
        f1 = _c(f1)
        H, W = f1.shape
        alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (H - 1, W - 1, 2))
        g, ft = coefficients(f1, f2, model)
        if rho > 0:
            Ael, Fel = element_data(f1, f2, rho, model)
            S = cls(W, H, g, ft, alpha, lam, Ael, Fel, lamel=lamel)
        else:
            S = cls(W, H, g, ft, alpha, lam, lamel=lamel)
        S.model = int(model)
        S.rho = float(rho)
        return S

    def precond_system(self):
        """The system whose Schwarz sweeps precondition this one on the CUDA
        path: for K_rho > 0 the same stiffness with the unsmoothed data term
        g g^T (an SPD operator close to A_rho; A_rho itself enters through
        the operator only)."""
        if self.Ael is None:
            return self
        return System(self.W, self.H, self.g, self.ft, self.alpha, self.lam, lamel=self.lamel)

    @property
    def n(self) -> int:
        return 3 * self.W * self.H

    def shape3(self, v):
        return np.asarray(v).reshape(3, self.H, self.W)

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for r in range(self.n):
            s, e = self.rowptr[r], self.rowptr[r + 1]
            A[r, self.col[s:e]] = self.val[s:e]
        return A

    def matvec(self, x):
        L = _load()
        x = _c(x).ravel()
        y = np.zeros(self.n)
        L.orc_csr_matvec(self.n, self.rowptr, self.col, self.val, x, y)
        return y.reshape(3, self.H, self.W)

    def residual(self, U):
        return self.b.reshape(3, self.H, self.W) - self.matvec(U)

    def rel_residual(self, U) -> float:
        return float(np.linalg.norm(self.residual(U)) / np.linalg.norm(self.b))

    def _solve_flow_block(self, rhs):
        """Brightness constancy: the m block is the pure-Neumann lambda
        Laplacian (singular, constants in its kernel), decoupled from (u1, u2)
        and without load.  Solve the (u1, u2) block with a sparse direct
        solver; m = 0 (the minimum-norm solution)."""
        import scipy.sparse.linalg as spla
        n2 = 2 * self.W * self.H
        rhs = _c(rhs).ravel()
        if np.abs(rhs[n2:]).max() > 0.0:
            raise ValueError("the m equations carry no data in this model: their right-hand side must be 0")
        A = self._sparse()[:n2, :n2].tocsc()
        x = np.zeros(self.n)
        x[:n2] = spla.spsolve(A, rhs[:n2])
        return x.reshape(3, self.H, self.W)

    def solve_direct(self):
        """Banded Cholesky (small grids: cost ~ 27 W H min(W,H)^2)."""
        if getattr(self, "model", 0) == 1:
            return self._solve_flow_block(self.b)
        L = _load()
        x = np.zeros(self.n)
        rc = L.orc_band_cholesky_solve(self.W, self.H, self.rowptr, self.col, self.val, self.b, x)
        if rc == 3:
            raise np.linalg.LinAlgError("matrix not positive definite")
        if rc:
            raise RuntimeError(f"banded Cholesky failed ({rc})")
        return x.reshape(3, self.H, self.W)

    def solve_pcg(self, tol=1e-12, maxit=100000, x0=None, rhs=None):
        """Block-Jacobi PCG; returns (U, iterations, final relative residual)."""
        L = _load()
        x = np.zeros(self.n) if x0 is None else _c(x0).ravel().copy()
        b = self.b if rhs is None else _c(rhs).ravel()
        rr = ctypes.c_double(0.0)
        it = L.orc_pcg(self.W, self.H, self.rowptr, self.col, self.val, b, x, tol, maxit, ctypes.byref(rr))
        if it < 0:
            raise RuntimeError("oracle PCG breakdown")
        return x.reshape(3, self.H, self.W), int(it), float(rr.value)

    def solve_asm_pcg(self, parts, overlap, tol=1e-12, maxit=100000, x0=None, rhs=None):
        """PCG with the exact-subdomain additive Schwarz preconditioner on a
        parts = (px, py) partition extended by `overlap` node layers (the
        solver for grids too large for banded Cholesky); returns (U,
        iterations, final relative residual recomputed as b - A U)."""
        L = _load()
        x = np.zeros(self.n) if x0 is None else _c(x0).ravel().copy()
        b = self.b if rhs is None else _c(rhs).ravel()
        rr = ctypes.c_double(0.0)
        it = L.orc_asm_pcg(self.W, self.H, self.rowptr, self.col, self.val, b, x, int(parts[0]), int(parts[1]),
                           int(overlap), tol, maxit, ctypes.byref(rr))
        if it == -2:
            raise MemoryError("oracle ASM-PCG: allocation failed")
        if it < 0:
            raise RuntimeError("oracle ASM-PCG breakdown (a subdomain matrix is not positive definite)")
        return x.reshape(3, self.H, self.W), int(it), float(rr.value)

    def solve_with(self, rhs, direct=True, tol=1e-13):
        if getattr(self, "model", 0) == 1 and direct:
            return self._solve_flow_block(rhs)
        L = _load()
        rhs = _c(rhs).ravel()
        x = np.zeros(self.n)
        if direct:
            rc = L.orc_band_cholesky_solve(self.W, self.H, self.rowptr, self.col, self.val, rhs, x)
            if rc:
                raise RuntimeError(f"banded Cholesky failed ({rc})")
            return x.reshape(3, self.H, self.W)
        U, _, _ = self.solve_pcg(tol=tol, rhs=rhs)
        return U

    def schwarz(self, px, py, overlap, iters, U0=None):
        """The paper's Schwarz iteration (Eq. schwarz) with exact subdomain
        solves; returns (U, history of ||U^k - U^{k-1}||)."""
        L = _load()
        U = np.zeros(self.n) if U0 is None else _c(U0).ravel().copy()
        hist = np.zeros(iters)
        rc = L.orc_schwarz(self.W, self.H, self.rowptr, self.col, self.val, self.b, px, py, overlap,
                           iters, U, hist.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise RuntimeError(f"oracle Schwarz failed ({rc})")
        return U.reshape(3, self.H, self.W), hist

    def _sparse(self):
        import scipy.sparse as sp
        if getattr(self, "_A", None) is None:
            self._A = sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))
        return self._A

    def schwarz_sweeps(self, r, tile, overlap, sweeps, omega=1.0):
        """The symmetric restricted Schwarz preconditioner z = M r with
        approximate local solves, written out plainly (the CUDA path's
        subdomain solver; the paper solves each subdomain exactly, Section 3.2).

        Owned tiles T_i of tile[0] x tile[1] nodes from the origin, clipped at
        the image edge; extended tiles E_i = T_i plus `overlap` node layers,
        clipped.  Local problem: A restricted to E_i (zero Dirichlet values
        outside E_i), right-hand side r on T_i and 0 on the rest of E_i.  It is
        solved from z = 0 by symmetric 3-colour block SOR: colour (i + j) mod 3
        in the coordinates of the unclipped extended tile (nodes of one colour
        are not coupled), colours visited 0,1,2,1 `sweeps` times and then 0;
        a visit sets z_n <- z_n + omega (D_n^{-1} (b_n - sum_{m != n} A_nm z_m)
        - z_n) for every node n of the colour, D_n the 3x3 diagonal block.
        sweeps = 0 is block Jacobi, z_n = D_n^{-1} b_n.  z is the sum over i
        of the owned part of each local solution."""
        A = self._sparse()
        W, H, HW = self.W, self.H, self.W * self.H
        r = _c(r).ravel()
        z = np.zeros(self.n)
        tx, ty = int(tile[0]), int(tile[1])
        seq = [0, 1, 2, 1] * int(sweeps) + [0]
        for y0 in range(0, H, ty):
            for x0 in range(0, W, tx):
                ox1, oy1 = min(x0 + tx, W), min(y0 + ty, H)
                ex0, ey0 = max(x0 - overlap, 0), max(y0 - overlap, 0)
                ex1, ey1 = min(ox1 + overlap, W), min(oy1 + overlap, H)
                ys, xs = np.mgrid[ey0:ey1, ex0:ex1]
                ys, xs = ys.ravel(), xs.ravel()
                m = xs.size
                idx = np.concatenate([ys * W + xs + c * HW for c in range(3)])
                Ai = A[idx][:, idx].tocsr()
                owned = (xs >= x0) & (xs < ox1) & (ys >= y0) & (ys < oy1)
                own3 = np.tile(owned, 3)
                b = np.where(own3, r[idx], 0.0)
                colour = ((xs - (x0 - overlap)) + (ys - (y0 - overlap))) % 3
                D = np.empty((m, 3, 3))
                dense_diag = {}
                for c in range(3):
                    for d in range(3):
                        dense_diag[c, d] = np.asarray(Ai[c * m + np.arange(m), d * m + np.arange(m)]).ravel()
                        D[:, c, d] = dense_diag[c, d]
                zi = np.zeros((3, m))
                bi = b.reshape(3, m)
                if sweeps == 0:
                    zi = np.linalg.solve(D, bi.T[..., None])[..., 0].T
                else:
                    for c in seq:
                        sel = np.nonzero(colour == c)[0]
                        y = (Ai @ zi.ravel()).reshape(3, m)
                        zn = zi[:, sel].T
                        rhs = bi[:, sel].T - y[:, sel].T + np.einsum("kij,kj->ki", D[sel], zn)
                        x = np.linalg.solve(D[sel], rhs[..., None])[..., 0]
                        zi[:, sel] = (zn + omega * (x - zn)).T
                z[idx[own3]] = zi.ravel()[own3]
        return z.reshape(3, H, W)

    def coarse_restriction(self, spacing):
        """R_0: bilinear hat functions of a coarse grid with nodes at
        x = 0, s, 2s, ... and x = W - 1 (likewise in y), one per component;
        rows ordered (component, coarse y, coarse x).  Returns a sparse
        [3 nc, 3 W H] matrix."""
        import scipy.sparse as sp
        def hats(n):
            xs = sorted(set(list(range(0, n, spacing)) + [n - 1]))
            Hm = np.zeros((len(xs), n))
            for k, c in enumerate(xs):
                for x in range(n):
                    if x == c:
                        Hm[k, x] = 1.0
                    elif k > 0 and xs[k - 1] < x < c:
                        Hm[k, x] = (x - xs[k - 1]) / (c - xs[k - 1])
                    elif k < len(xs) - 1 and c < x < xs[k + 1]:
                        Hm[k, x] = (xs[k + 1] - x) / (xs[k + 1] - c)
            return Hm
        P = sp.csr_matrix(np.kron(hats(self.H), hats(self.W)))
        return sp.block_diag([P, P, P]).tocsr()

    def two_level(self, r, tile, overlap, sweeps, omega, spacing):
        """Additive two-level preconditioner: the restricted Schwarz sweeps
        (schwarz_sweeps) plus the coarse correction R_0^T A_0^{-1} R_0 r with
        the Galerkin coarse operator A_0 = R_0 A R_0^T of the bilinear coarse
        space (coarse_restriction)."""
        R0 = self.coarse_restriction(spacing)
        A0 = (R0 @ self._sparse() @ R0.T).toarray()
        r = _c(r).ravel()
        zc = R0.T @ np.linalg.solve(A0, R0 @ r)
        return self.schwarz_sweeps(r, tile, overlap, sweeps, omega) + zc.reshape(3, self.H, self.W)

    def indicator(self, U):
        L = _load()
        eta = np.zeros((self.H - 1, self.W - 1, 2))
        if self.Ael is None:
            L.orc_indicator(self.W, self.H, self.g, self.ft, self.alpha, self.lam, _ptr(self.lamel), _c(U).ravel(),
                            eta)
        else:
            L.orc_indicator_el(self.W, self.H, self.Ael, self.Fel, self.alpha, self.lam, _ptr(self.lamel),
                               _c(U).ravel(), eta)
        return eta


def _gauss_taps(sigma):
    r = int(np.ceil(3.0 * sigma))
    k = np.arange(-r, r + 1)
    return k, np.exp(-(k.astype(np.float64) ** 2) / (2.0 * sigma * sigma))


def _smooth_axis(A, axis, sigma, transpose=False):
    """One normalised pass of K_sigma along `axis`: out(x) = sum over the taps
    k with 0 <= x+k < n of w_k A(x+k), divided by the sum of those w_k; the
    transposed pass divides each input by the normaliser of the position it
    comes from instead."""
    A = np.moveaxis(np.asarray(A, dtype=np.float64), axis, -1)
    n = A.shape[-1]
    k, w = _gauss_taps(sigma)
    norm = np.zeros(n)
    for kk, wk in zip(k, w):
        lo, hi = max(0, -kk), min(n, n - kk)
        if hi > lo:  # a tap that reaches past the whole axis adds nothing
            norm[lo:hi] += wk
    src = A / norm if transpose else A
    out = np.zeros_like(A)
    for kk, wk in zip(k, w):
        lo, hi = max(0, -kk), min(n, n - kk)
        if hi > lo:
            out[..., lo:hi] += wk * src[..., lo + kk:hi + kk]
    if not transpose:
        out = out / norm
    return np.moveaxis(out, -1, axis)


def smooth(I, sigma):
    """f = K_sigma * I (Section 1): sampled Gaussian w_k = exp(-k^2/(2 sigma^2)),
    |k| <= ceil(3 sigma), along x then along y, each pass normalised over the
    taps inside the image.  sigma = 0 returns I."""
    if sigma <= 0:
        return np.array(I, dtype=np.float64)
    return _smooth_axis(_smooth_axis(I, 1, sigma), 0, sigma)


def smooth_transpose(G, sigma):
    """The transpose of `smooth` (x-pass then y-pass, so S^T = S_x^T S_y^T)."""
    if sigma <= 0:
        return np.array(G, dtype=np.float64)
    return _smooth_axis(_smooth_axis(G, 0, sigma, True), 1, sigma, True)


def _lamel(lamel, W, H):
    return None if lamel is None else _c(np.broadcast_to(np.asarray(lamel, dtype=np.float64), (H - 1, W - 1, 2)))


def apply_elementwise(W, H, g, ft, alpha, lam, U, with_rhs=False, lamel=None):
    """A U (and b) without storing A, for grids too large for the CSR
    (lamel: per-element lambda, None for the constant lam)."""
    L = _load()
    lamel = _lamel(lamel, W, H)
    y = np.zeros(3 * W * H)
    b = np.zeros(3 * W * H) if with_rhs else None
    alpha = _c(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (H - 1, W - 1, 2)))
    L.orc_apply_elementwise(W, H, _c(g), _c(ft), alpha, float(lam), _ptr(lamel), _c(U).ravel(), y, _ptr(b))
    y = y.reshape(3, H, W)
    return (y, b.reshape(3, H, W)) if with_rhs else y


def rel_residual_frames(f1, f2, alpha, lam, U, model=0, lamel=None) -> float:
    """||b - A U||_2 / ||b||_2 of a frame pair, formed element by element."""
    f1 = _c(f1)
    H, W = f1.shape
    g, ft = coefficients(f1, f2, model)
    AU, b = apply_elementwise(W, H, g, ft, alpha, lam, U, with_rhs=True, lamel=lamel)
    return float(np.linalg.norm(b - AU) / np.linalg.norm(b))


def indicator(W, H, g, ft, alpha, lam, U, lamel=None):
    L = _load()
    lamel = _lamel(lamel, W, H)
    eta = np.zeros((H - 1, W - 1, 2))
    alpha = _c(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (H - 1, W - 1, 2)))
    L.orc_indicator(W, H, _c(g), _c(ft), alpha, float(lam), _ptr(lamel), _c(U).ravel(), eta)
    return eta


def adjoint_grad_lambda(f1, f2, alpha, lam, U, Lam):
    """dL/dlambda_K = -|K| grad(Lam_m) . grad(U_m) per element (the derivative
    of the m stiffness w.r.t. a per-element lambda), given U and the adjoint
    state Lam."""
    L = _load()
    f1, f2 = _c(f1), _c(f2)
    H, W = f1.shape
    alpha = _c(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (H - 1, W - 1, 2)))
    dl = np.zeros((H - 1, W - 1, 2))
    L.orc_adjoint_grad(W, H, f1, f2, alpha, float(lam), _c(U).ravel(), _c(Lam).ravel(), None, None, None, _ptr(dl), 0)
    return dl


def alpha_update(eta, alpha, kappa, eta_thr, alpha_th):
    L = _load()
    a = _c(alpha).copy()
    L.orc_alpha_update(a.size, _c(eta), a, kappa, eta_thr, alpha_th)
    return a


def adjoint_grad(f1, f2, alpha, lam, U, Lam, want_f1=True, model=0, rho=0.0):
    """(dL/dalpha, dL/df2, dL/df1) given U and the adjoint state Lam.  With
    rho > 0 the frame gradients go through the K_rho element tensors
    (_adjoint_frames_rho); dL/dalpha only involves the stiffness."""
    L = _load()
    f1, f2 = _c(f1), _c(f2)
    H, W = f1.shape
    alpha = _c(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (H - 1, W - 1, 2)))
    da = np.zeros((H - 1, W - 1, 2))
    d2 = np.zeros((H, W))
    d1 = np.zeros((H, W)) if want_f1 else None
    L.orc_adjoint_grad(W, H, f1, f2, alpha, float(lam), _c(U).ravel(), _c(Lam).ravel(),
                       _ptr(da), _ptr(d2), _ptr(d1), None, int(model))
    if rho > 0:
        d2, d1r = _adjoint_frames_rho(f1, f2, U, Lam, model, rho)
        d1 = d1r if want_f1 else None
    return da, d2, d1


def _tri_vertex_index(W, H):
    """[H-1][W-1][2][3] (y, x) vertex coordinates of every element (Section
    2.2 mesh: t = 0 -> (x,y), (x+1,y), (x+1,y+1); t = 1 -> (x,y), (x,y+1),
    (x+1,y+1))."""
    ys, xs = np.mgrid[0:H - 1, 0:W - 1]
    vy = np.zeros((H - 1, W - 1, 2, 3), dtype=np.int64)
    vx = np.zeros_like(vy)
    vy[..., 0, :] = np.stack([ys, ys, ys + 1], -1)
    vx[..., 0, :] = np.stack([xs, xs + 1, xs + 1], -1)
    vy[..., 1, :] = np.stack([ys, ys + 1, ys + 1], -1)
    vx[..., 1, :] = np.stack([xs, xs, xs + 1], -1)
    return vy, vx


def _adjoint_frames_rho(f1, f2, U, Lam, model, rho):
    """Frame gradients with the K_rho data term.  With E = Lam^T (A U - b)
    assembled from the element tensors, dL/dtheta = -dE/dtheta and
      dE/dA_cd = |K|/12 (sum_i Lam_ic U_id + (sum_i Lam_ic)(sum_i U_id)),
      dE/dF_c  = -|K|/3 sum_i Lam_ic;
    these go back to the frames through _element_data_chain."""
    f1, f2 = _c(f1), _c(f2)
    H, W = f1.shape
    U, Lam = np.asarray(U, np.float64), np.asarray(Lam, np.float64)
    vy, vx = _tri_vertex_index(W, H)
    Ue = np.moveaxis(U[:, vy, vx], 0, -1)      # [H-1][W-1][2][3 vertices][3 comps]
    Le = np.moveaxis(Lam[:, vy, vx], 0, -1)
    K = 0.5
    M = K / 12.0 * (np.einsum("...ic,...id->...cd", Le, Ue)
                    + np.einsum("...c,...d->...cd", Le.sum(-2), Ue.sum(-2)))
    GA = np.stack([M[..., c, c] if c == d else M[..., c, d] + M[..., d, c] for c, d in SYM6], -1)
    GF = -K / 3.0 * Le.sum(-2)
    d2, d1 = _element_data_chain(f1, f2, GA, GF, model, rho)
    return -d2, -d1


def _element_data_chain(f1, f2, GA, GF, model, rho):
    """Frame gradients of a function of the element data (Section 1: A_rho =
    K_rho * (g g^T), F = K_rho * (-ft g)) given its derivatives GA with
    respect to the 6 stored entries SYM6 of A_rho and GF with respect to F,
    per element [H-1][W-1][2][.].  K_rho is linear, so these go back to the
    unsmoothed products through its transpose (smooth_transpose, per
    triangle family); the products g_c g_d and -ft g_c then give d/dg and
    d/dft, and g, ft depend on the frames through the P1 gradient of f2 and
    the vertex means (_frames_chain)."""
    f1, f2 = _c(f1), _c(f2)
    H, W = f1.shape
    GA, GF = np.array(GA, dtype=np.float64), np.array(GF, dtype=np.float64)
    for t in range(2):  # K_rho^T per family
        for k in range(6):
            GA[:, :, t, k] = smooth_transpose(GA[:, :, t, k], rho)
        for k in range(3):
            GF[:, :, t, k] = smooth_transpose(GF[:, :, t, k], rho)
    g, ft = coefficients(f1, f2, model)
    dg = np.zeros_like(g)
    for k, (c, d) in enumerate(SYM6):
        dg[..., c] += GA[..., k] * g[..., d]
        dg[..., d] += GA[..., k] * g[..., c]
    dg -= ft[..., None] * GF
    dft = -np.sum(GF * g, axis=-1)
    return _frames_chain(W, H, dg, dft, model)


# gradients of the P1 basis functions of each triangle family (t = 0: vertices
# (x,y), (x+1,y), (x+1,y+1); t = 1: (x,y), (x,y+1), (x+1,y+1))
GPHI_X = np.array([[-1.0, 1.0, 0.0], [0.0, -1.0, 1.0]])
GPHI_Y = np.array([[0.0, -1.0, 1.0], [-1.0, 1.0, 0.0]])


def _frames_chain(W, H, dg, dft, model):
    """Per-element derivatives w.r.t. g = (d/dx f2_h, d/dy f2_h, -gms mean f1)
    and ft = mean (f2 - f1) carried to the frame pixels (the vertices)."""
    vy, vx = _tri_vertex_index(W, H)
    gms = 0.0 if model == 1 else 1.0
    d2 = np.zeros((H, W))
    d1 = np.zeros((H, W))
    for t in range(2):
        for i in range(3):
            c2 = dg[:, :, t, 0] * GPHI_X[t, i] + dg[:, :, t, 1] * GPHI_Y[t, i] + dft[:, :, t] / 3.0
            c1 = -gms * dg[:, :, t, 2] / 3.0 - dft[:, :, t] / 3.0
            np.add.at(d2, (vy[:, :, t, i], vx[:, :, t, i]), c2)
            np.add.at(d1, (vy[:, :, t, i], vx[:, :, t, i]), c1)
    return d2, d1


def alpha_update_vjp(eta, alpha, kappa, eta_thr, alpha_th, v):
    """Vector-Jacobian product of the alpha update of Section 2.3
      alpha' = max(alpha / (1 + kappa max(eta / max(eta) - eta_thr, 0)), alpha_th)
    for dL/dalpha' = v: returns (dL/dalpha through the update, dL/deta).
    One-sided pieces take the branch the forward took (alpha' = alpha_th and
    eta / max(eta) - eta_thr <= 0 are the flat branches); max(eta) passes
    its derivative to the first element that attains it.  No update (eta = 0)
    is the identity."""
    eta, alpha, v = (np.asarray(a, dtype=np.float64) for a in (eta, alpha, v))
    shape = eta.shape
    eta, alpha, v = eta.ravel(), alpha.ravel(), v.ravel()
    m = eta.max()
    if not m > 0:
        return v.reshape(shape).copy(), np.zeros(shape)
    rel = eta / m - eta_thr
    pos = rel > 0
    sr = np.where(pos, rel, 0.0)
    den = 1.0 + kappa * sr
    active = alpha / den > alpha_th
    da = np.where(active, v / den, 0.0)
    ds = np.where(active, -v * alpha * kappa / den ** 2, 0.0)
    w = np.where(pos, ds / m, 0.0)
    w[int(np.argmax(eta))] += -np.sum(np.where(pos, ds * eta / (m * m), 0.0))
    return da.reshape(shape), w.reshape(shape)


def _element_neighbours(W, H):
    """For edge k of element (y, x, t) (the edge order of orc_indicator):
    outward normal, length, neighbour element (y, x, t) and a mask of
    interior edges."""
    ys, xs = np.mgrid[0:H - 1, 0:W - 1]
    r2 = np.sqrt(0.5)
    nrm = np.array([[[0, -1], [1, 0], [-r2, r2]], [[-1, 0], [0, 1], [r2, -r2]]])  # [t][k][2]
    he = np.array([[1.0, 1.0, np.sqrt(2.0)], [1.0, 1.0, np.sqrt(2.0)]])
    nb = np.zeros((H - 1, W - 1, 2, 3, 3), dtype=np.int64)  # (y, x, t) of the neighbour
    ok = np.zeros((H - 1, W - 1, 2, 3), dtype=bool)
    nb[:, :, 0, 0] = np.stack([ys - 1, xs, np.ones_like(ys)], -1); ok[:, :, 0, 0] = ys > 0
    nb[:, :, 0, 1] = np.stack([ys, xs + 1, np.ones_like(ys)], -1); ok[:, :, 0, 1] = xs < W - 2
    nb[:, :, 0, 2] = np.stack([ys, xs, np.ones_like(ys)], -1); ok[:, :, 0, 2] = True
    nb[:, :, 1, 0] = np.stack([ys, xs - 1, np.zeros_like(ys)], -1); ok[:, :, 1, 0] = xs > 0
    nb[:, :, 1, 1] = np.stack([ys + 1, xs, np.zeros_like(ys)], -1); ok[:, :, 1, 1] = ys < H - 2
    nb[:, :, 1, 2] = np.stack([ys, xs, np.zeros_like(ys)], -1); ok[:, :, 1, 2] = True
    nb[..., 0] = np.clip(nb[..., 0], 0, H - 2)
    nb[..., 1] = np.clip(nb[..., 1], 0, W - 2)
    return nrm, he, nb, ok


def indicator_vjp(f1, f2, alpha, lam, U, w, model=0, rho=0.0):
    """Vector-Jacobian product of the error indicator eta_K (Section 2.3,
    Eq. errind, read as in orc_indicator: interior term h_K ||Lambda^-1/2 R||
    with R = -g (g.U_h + ft), edge terms 1/2 h_e sqrt(q_e) with the flux
    jump J and Lambda_e = max of the two sides) for dL/deta = w.  Returns
    (dL/dU [3][H][W], dL/dalpha [H-1][W-1][2], dL/df2, dL/df1).  An edge term
    appears in the indicators of both elements that share it; Lambda_e at
    equal sides passes half of its derivative to each (the mean of the
    one-sided derivatives, what central differences see).  With rho > 0 the
    interior residual is R = F - A_rho U_h (orc_indicator_el) and its frame
    derivatives go through the element data (_element_data_chain)."""
    f1, f2 = _c(f1), _c(f2)
    H, W = f1.shape
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (H - 1, W - 1, 2))
    U = np.asarray(U, np.float64)
    w = np.asarray(w, np.float64)
    g, ft = coefficients(f1, f2, model)
    vy, vx = _tri_vertex_index(W, H)
    Ue = np.moveaxis(U[:, vy, vx], 0, -1)                     # [y][x][t][vertex][c]
    Lam = np.stack([alpha, alpha, np.full_like(alpha, lam)], -1)  # [y][x][t][c]
    grad = np.stack([np.einsum("yxtic,ti->yxtc", Ue, GPHI_X),
                     np.einsum("yxtic,ti->yxtc", Ue, GPHI_Y)], -1)  # [y][x][t][c][2]
    dU_v = np.zeros_like(Ue)
    dal = np.zeros_like(alpha)
    dg = np.zeros_like(g)
    dft = np.zeros_like(ft)
    if rho > 0:
        return _indicator_vjp_general(f1, f2, alpha, lam, Ue, w, model, rho, vy, vx, grad, Lam)
    # interior: integ = 1/6 G sum_a s_a^2, val = sqrt(2 integ)
    G = np.sum(g * g / Lam, -1)
    s_a, Um = [], []
    for a in range(3):
        b = (a + 1) % 3
        um = 0.5 * (Ue[..., a, :] + Ue[..., b, :])
        Um.append(um)
        s_a.append(ft + np.sum(g * um, -1))
    S2 = sum(x * x for x in s_a)
    integ = G * S2 / 6.0
    wi = np.where(integ > 0, w / np.sqrt(2.0 * np.where(integ > 0, integ, 1.0)), 0.0)
    for a in range(3):
        b = (a + 1) % 3
        coef = (wi * G * s_a[a] / 3.0)[..., None] * g      # d/dUm
        dU_v[..., a, :] += 0.5 * coef
        dU_v[..., b, :] += 0.5 * coef
        dg += (wi * G * s_a[a] / 3.0)[..., None] * Um[a]
        dft += wi * G * s_a[a] / 3.0
    dg += (wi * S2 / 6.0)[..., None] * 2.0 * g / Lam
    dal += wi * S2 / 6.0 * (-(g[..., 0] ** 2 + g[..., 1] ** 2) / alpha ** 2)
    _indicator_vjp_edges(W, H, w, Lam, grad, alpha, dU_v, dal)
    dU = _scatter_vertices(W, H, dU_v, vy, vx)
    d2, d1 = _frames_chain(W, H, dg, dft, model)
    return dU, dal, d2, d1


def _indicator_vjp_edges(W, H, w, Lam, grad, alpha, dU_v, dal):
    """The edge terms of indicator_vjp (they do not involve the data term):
    adds their derivatives to the per-vertex dU_v and to dal in place."""
    dgradK = np.zeros_like(grad)
    nrm, he, nb, ok = _element_neighbours(W, H)
    for t in range(2):
        for k in range(3):
            n = nrm[t, k]
            oy, ox, ot = nb[:, :, t, k, 0], nb[:, :, t, k, 1], nb[:, :, t, k, 2]
            m = ok[:, :, t, k]
            LK = Lam[:, :, t, :]
            LO = Lam[oy, ox, ot, :]
            fin = LK * (grad[:, :, t, :, :] @ n)
            fout = np.where(m[..., None], LO * (grad[oy, ox, ot, :, :] @ n), 0.0)
            Le = np.where(m[..., None], np.maximum(LK, LO), LK)
            J = fout - fin
            q = np.sum(J * J / Le, -1)
            wt = w[:, :, t] + np.where(m, w[oy, ox, ot], 0.0)
            ce = np.where(q > 0, wt * 0.25 * he[t, k] / np.sqrt(np.where(q > 0, q, 1.0)), 0.0)
            dJ = ce[..., None] * 2.0 * J / Le                  # d/dJ_c
            dgradK[:, :, t, :, :] += (-(LK * dJ))[..., None] * n
            share = np.where(m[..., None], np.where(LK > LO, 1.0, np.where(LK == LO, 0.5, 0.0)), 1.0)
            dLK = dJ * (-(grad[:, :, t, :, :] @ n)) + ce[..., None] * (-(J * J) / (Le * Le)) * share
            dal[:, :, t] += dLK[..., 0] + dLK[..., 1]
    # vertex gradients of the element gradients
    dU_v += np.einsum("yxtc,ti->yxtic", dgradK[..., 0], GPHI_X) + np.einsum("yxtc,ti->yxtic", dgradK[..., 1], GPHI_Y)


def _scatter_vertices(W, H, dU_v, vy, vx):
    """Per-element vertex values [H-1][W-1][2][3][3] summed into [3][H][W]."""
    dU = np.zeros((3, H, W))
    for t in range(2):
        for i in range(3):
            for c in range(3):
                np.add.at(dU[c], (vy[:, :, t, i], vx[:, :, t, i]), dU_v[:, :, t, i, c])
    return dU


def _indicator_vjp_general(f1, f2, alpha, lam, Ue, w, model, rho, vy, vx, grad, Lam):
    """indicator_vjp with the K_rho element data (rho > 0).  Interior term
    val = h_K sqrt(integ), integ = |K|/3 sum_a sum_c R_ac^2 / Lambda_c over
    the edge midpoints m_a, R_a = F - A_rho U_h(m_a):
      d val / d integ = h_K / (2 sqrt(integ)),
      d integ / d R_ac = (2|K|/3) R_ac / Lambda_c,
    and R_a is linear in F (identity), in A_rho (-U_h(m_a)) and in the
    midpoint values (-A_rho)."""
    H, W = np.asarray(f1).shape
    Ael, Fel = element_data(f1, f2, rho, model)
    Am = np.zeros(Ael.shape[:-1] + (3, 3))
    for k, (c, d) in enumerate(SYM6):
        Am[..., c, d] = Ael[..., k]
        Am[..., d, c] = Ael[..., k]
    K, hK = 0.5, np.sqrt(2.0)
    dU_v = np.zeros_like(Ue)
    dal = np.zeros_like(np.asarray(alpha, dtype=np.float64))
    Um, Ra = [], []
    for a in range(3):
        b = (a + 1) % 3
        um = 0.5 * (Ue[..., a, :] + Ue[..., b, :])
        Um.append(um)
        Ra.append(Fel - np.einsum("...cd,...d->...c", Am, um))
    integ = K / 3.0 * sum(np.sum(R * R / Lam, -1) for R in Ra)
    dv = np.where(integ > 0, w * hK / (2.0 * np.sqrt(np.where(integ > 0, integ, 1.0))), 0.0)
    GAm = np.zeros_like(Am)
    GF = np.zeros_like(Fel)
    for a in range(3):
        b = (a + 1) % 3
        dR = dv[..., None] * (2.0 * K / 3.0) * Ra[a] / Lam
        GF += dR
        GAm -= np.einsum("...c,...d->...cd", dR, Um[a])
        dum = -np.einsum("...cd,...c->...d", Am, dR)
        dU_v[..., a, :] += 0.5 * dum
        dU_v[..., b, :] += 0.5 * dum
        dal += dv * (K / 3.0) * (-(Ra[a][..., 0] ** 2 + Ra[a][..., 1] ** 2) / np.asarray(alpha) ** 2)
    GA = np.stack([GAm[..., c, c] if c == d else GAm[..., c, d] + GAm[..., d, c] for c, d in SYM6], -1)
    _indicator_vjp_edges(W, H, w, Lam, grad, alpha, dU_v, dal)
    dU = _scatter_vertices(W, H, dU_v, vy, vx)
    d2, d1 = _element_data_chain(f1, f2, GA, GF, model, rho)
    return dU, dal, d2, d1


def adaptation_forward(f1, f2, alpha0, lam, npasses, kappa, eta_thr, alpha_th, model=0, rho=0.0):
    """npasses adaptation passes (Section 2.3 on the fixed mesh): solve,
    indicator, alpha update; then the final solve.  Returns the final U and
    the per-pass (alpha_k, U_k, eta_k) checkpoints."""
    a = np.array(np.broadcast_to(np.asarray(alpha0, dtype=np.float64), (f1.shape[0] - 1, f1.shape[1] - 1, 2)))
    passes = []
    for _ in range(npasses):
        S = System.from_frames(f1, f2, a, lam, model, rho=rho)
        U = S.solve_direct()
        eta = S.indicator(U)
        passes.append((a.copy(), U, eta))
        a = alpha_update(eta, a, kappa, eta_thr, alpha_th)
    S = System.from_frames(f1, f2, a, lam, model, rho=rho)
    return S.solve_direct(), a, passes


def adaptation_grad(f1, f2, alpha0, lam, npasses, kappa, eta_thr, alpha_th, dLdU, model=0, rho=0.0):
    """dL/dalpha_0, dL/df2, dL/df1 of L(U_final) through the adaptation
    passes, in reverse: the adjoint solve of each pass (adjoint_grad), then
    the alpha update (alpha_update_vjp) and the indicator (indicator_vjp)
    that produced its alpha, whose dL/dU starts the previous pass's adjoint
    solve."""
    U, a, passes = adaptation_forward(f1, f2, alpha0, lam, npasses, kappa, eta_thr, alpha_th, model, rho)
    S = System.from_frames(f1, f2, a, lam, model, rho=rho)
    v, g2, g1 = adjoint_grad(f1, f2, a, lam, U, S.solve_with(dLdU), model=model, rho=rho)
    for a_k, U_k, eta_k in reversed(passes):
        da_upd, w = alpha_update_vjp(eta_k, a_k, kappa, eta_thr, alpha_th, v)
        dU_k, da_eta, d2e, d1e = indicator_vjp(f1, f2, a_k, lam, U_k, w, model, rho)
        S = System.from_frames(f1, f2, a_k, lam, model, rho=rho)
        ga, g2k, g1k = adjoint_grad(f1, f2, a_k, lam, U_k, S.solve_with(dU_k), model=model, rho=rho)
        v = da_upd + da_eta + ga
        g2 = g2 + d2e + g2k
        g1 = g1 + d1e + g1k
    return v, g2, g1


def mean_epe(U, flow_gt):
    """Mean endpoint error (Section 4) of the flow part of U."""
    d = np.asarray(U[:2], dtype=np.float64) - np.asarray(flow_gt, dtype=np.float64)
    return float(np.mean(np.sqrt(d[0] ** 2 + d[1] ** 2)))


def mean_epe_grad(U, flow_gt):
    """dL/dU of the mean endpoint error; 0 where the endpoint error is 0."""
    U = np.asarray(U, dtype=np.float64)
    d = U[:2] - np.asarray(flow_gt, dtype=np.float64)
    e = np.sqrt(d[0] ** 2 + d[1] ** 2)
    n = e.size
    out = np.zeros_like(U)
    nz = e > 0
    out[0][nz] = d[0][nz] / (n * e[nz])
    out[1][nz] = d[1][nz] / (n * e[nz])
    return out


def aae_deg(U, flow_gt):
    """Average angular error in degrees (Section 4)."""
    u, v = np.asarray(U[0], dtype=np.float64), np.asarray(U[1], dtype=np.float64)
    ue, ve = np.asarray(flow_gt[0], dtype=np.float64), np.asarray(flow_gt[1], dtype=np.float64)
    c = (u * ue + v * ve + 1.0) / np.sqrt((u * u + v * v + 1.0) * (ue * ue + ve * ve + 1.0))
    return float(np.degrees(np.mean(np.arccos(np.clip(c, -1.0, 1.0)))))
