"""The bounds-check build (-DOF_BOUNDS_CHECK: every guarded device index is
checked against its buffer, a violation sets a bit of the device error word
and the entry point returns OF_ERR_CUDA) run over the odd shapes of the apply
tests, clipped and overlapped tiles, both precisions, the FP16 paired and the
FP32 sweeps and the stationary Schwarz iteration: every call returns OF_OK and
gives the results of the normal build.

The bounds-check library runs in a child process (OFSOLVE_LIB selects it at
import); the normal build's results come from this process."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1508_02977_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = [(64, 48), (7, 5), (130, 67), (2, 2), (2, 9), (9, 2), (300, 40), (97, 101)]
# (precision, tile, overlap, sweeps, omega, half_sweeps, schwarz)
GRIDS = [(1, (48, 48), 0, 4, 1.6, 0, 0), (1, (12, 12), 0, 2, 1.5, 1, 0), (1, (32, 32), 2, 2, 1.0, -1, 0),
         (0, (16, 12), 4, 2, 1.6, 0, 0), (0, (16, 12), 2, 8, 1.8, 0, 1)]

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_1508_02977_gb300 import ofsolve as S, synth
out = {}
for gi, (prec, tile, ov, sw, om, half, schw) in enumerate(GRIDS):
    for si, (W, H) in enumerate(SHAPES):
        f1, f2 = synth.random_frames(W, H, 300 + si)
        al = synth.random_alpha(W, H, 310 + si)
        dt = torch.float64 if prec == 0 else torch.float32
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
        h = S.of_create(0)
        try:
            S.of_setup_grid(h, [(W, H)], tile=tile, overlap=ov, sweeps=sw, omega=om, precision=prec,
                            half_sweeps=half if prec == 1 else 0, schwarz=schw)
            S.of_set_frames(h, 0, d(f1), d(f2))
            S.of_set_alpha(h, 0, d(al))
            p = d(np.random.default_rng(320 + si).standard_normal((3, H, W)))
            q = torch.zeros_like(p)
            S.of_apply(h, 0, p, q)
            z = torch.zeros_like(p)
            if not schw:
                S.of_precondition(h, 0, p, z)
            U = torch.zeros(3, H, W, dtype=torch.float64, device="cuda")
            st, info = S.of_solve(h, [U], rtol=1e-8, max_inner=400, raise_on=False)
            assert st in (S.OF_OK, S.OF_ERR_NOT_CONVERGED, S.OF_ERR_BREAKDOWN), (st, S.of_last_error(h))
            assert "index check" not in S.of_last_error(h)
            out[f"q{gi}_{si}"] = q.cpu().numpy()
            out[f"z{gi}_{si}"] = z.cpu().numpy()
            out[f"u{gi}_{si}"] = U.cpu().numpy()
            out[f"s{gi}_{si}"] = np.array([st])
        finally:
            S.of_destroy(h)
np.savez(OUT, **out)
'''


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1508_02977_gb300 import ofsolve
    return ofsolve


def run_child(lib, out):
    code = f"ROOT = {ROOT!r}\nOUT = {out!r}\nGRIDS = {GRIDS!r}\nSHAPES = {SHAPES!r}\n" + CHILD
    env = dict(os.environ, OFSOLVE_LIB=lib)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return dict(np.load(out))


def test_bounds_checked_build_matches_normal_build(S, tmp_path):
    from paper_1508_02977_gb300 import build
    lib_bc = build.build(bounds_check=True)
    checked = run_child(lib_bc, str(tmp_path / "bc.npz"))
    normal = run_child(build.LIB, str(tmp_path / "n.npz"))
    assert checked.keys() == normal.keys()
    for k in normal:
        a, b = checked[k], normal[k]
        if k.startswith("s"):
            assert np.array_equal(a, b), k
            continue
        scale = max(np.abs(b).max(), 1e-30)
        assert np.abs(a - b).max() <= 1e-6 * scale, (k, np.abs(a - b).max(), scale)
