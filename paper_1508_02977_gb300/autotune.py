"""Autotuner for the subdomain tile, overlap, sweep count and relaxation factor.

For a frame size class it times complete solves (to the same relative
residual) of a representative pair for each candidate configuration and
keeps the fastest.  Candidates are ordered by the partition prior of Section
3.1 (largest area/perimeter ratio of the owned tile first), so a budget that
stops early has tried the shapes the paper's rule prefers.  Results are
cached in a JSON file keyed by size class, precision and device name.
"""
from __future__ import annotations

import json
import os
import time

from . import partition

# (tile, overlap, sweeps[, omega]); omega defaults to 1 (block Gauss-Seidel).
# Tiles 32..128 and overlaps 0..16 as far as one CTA holds the extended tile
# (at most 2304 nodes: 48 x 48, or 64 x 36, 96 x 24, 128 x 18 without overlap);
# extended heights of 6k nodes also run the FP16 paired sweeps.
DEFAULT_CANDIDATES = (
    ((48, 48), 0, 4, 1.6), ((48, 48), 0, 3, 1.6), ((48, 48), 0, 3, 1.0), ((48, 48), 0, 2, 1.5),
    ((48, 48), 0, 4, 1.7), ((48, 48), 0, 5, 1.7), ((32, 32), 0, 3, 1.6), ((64, 32), 0, 3, 1.6),
    ((64, 36), 0, 4, 1.6), ((96, 24), 0, 4, 1.6), ((128, 18), 0, 4, 1.6), ((40, 40), 0, 3, 1.6),
    ((44, 44), 2, 4, 1.6), ((40, 40), 4, 4, 1.6), ((36, 36), 6, 4, 1.6), ((32, 32), 8, 4, 1.6),
    ((32, 32), 8, 6, 1.6), ((16, 16), 16, 4, 1.6), ((32, 32), 2, 2, 1.0), ((32, 32), 0, 1, 1.0),
)
FALLBACK = {"tile": (48, 48), "overlap": 0, "sweeps": 4, "omega": 1.6}


def _norm(c):
    (tx, ty), ov, sw = c[0], c[1], c[2]
    om = float(c[3]) if len(c) > 3 else 1.0
    return (int(tx), int(ty)), int(ov), int(sw), om


def size_class(W: int, H: int) -> str:
    """Frames whose pixel count is within a factor 2 share a class."""
    px = max(W * H, 1)
    return f"px2^{int(round(__import__('math').log2(px)))}"


def cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_1508_02977_gb300", "autotune.json")


def prior_order(candidates, W: int, H: int):
    """Candidates sorted by the Section 3.1 prior: larger area/perimeter of
    the owned tile first (then fewer overlap nodes, then fewer sweeps)."""
    def key(c):
        (tx, ty), ov, sw, _ = _norm(c)
        return (-partition.part_ratio(tx, ty, 1, 1), partition.overlap_inflation(tx, ty, ov), sw)
    return sorted(candidates, key=key)


def _key(W, H, precision, device_name):
    return f"{device_name}|prec{precision}|{size_class(W, H)}"


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(d: dict, path=None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(W: int, H: int, precision: int = 1, device_name: str = "", path=None) -> dict:
    """The cached best configuration for this size class, else the default."""
    d = load_cache(path).get(_key(W, H, precision, device_name))
    if d:
        return {"tile": tuple(d["tile"]), "overlap": int(d["overlap"]), "sweeps": int(d["sweeps"]),
                "omega": float(d.get("omega", 1.0))}
    return dict(FALLBACK)


def autotune(W: int, H: int, f1=None, f2=None, alpha0: float = 0.05, lam: float = 1.0, precision: int = 1,
             device: int = 0, candidates=None, reps: int = 2, rtol: float = 1e-6, cache: bool = True,
             path=None, verbose: bool = False) -> dict:
    """Times every candidate on (f1, f2) (a synthetic layered pair of the same
    size if not given) and returns (and caches) the fastest configuration."""
    import torch

    from . import ofsolve as S
    from . import synth

    dev = torch.device("cuda", device)
    if f1 is None or f2 is None:
        p = synth.layers(W, H)
        f1, f2 = p.f1, p.f2
    dt = torch.float64 if precision == S.OF_PREC_FP64 else torch.float32
    t1 = torch.as_tensor(f1).to(dev, dt).contiguous()
    t2 = torch.as_tensor(f2).to(dev, dt).contiguous()
    results = []
    stream = torch.cuda.current_stream(dev)
    for cand in prior_order(candidates or DEFAULT_CANDIDATES, W, H):
        tile, ov, sw, om = _norm(cand)
        h = S.of_create(device, stream)
        try:
            try:
                S.of_setup_grid(h, [(W, H)], tile=tile, overlap=ov, sweeps=sw, precision=precision, lam=lam,
                                omega=om)
            except S.OFError:
                continue  # shape not supported for this precision (shared memory / registers)
            S.of_set_frames(h, 0, t1, t2)
            S.of_set_alpha(h, 0, None, alpha0)
            U = torch.zeros(3, H, W, dtype=torch.float64, device=dev)
            S.of_solve(h, [U], rtol=rtol)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                _, info = S.of_solve(h, [U], rtol=rtol)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            results.append({"tile": list(tile), "overlap": ov, "sweeps": sw, "omega": om, "ms": ms,
                            "iters": info[0]["inner_iters"]})
            if verbose:
                print(json.dumps(results[-1]), flush=True)
        finally:
            S.of_destroy(h)
    if not results:
        return dict(FALLBACK)
    best = min(results, key=lambda r: r["ms"])
    out = {"tile": tuple(best["tile"]), "overlap": best["overlap"], "sweeps": best["sweeps"], "omega": best["omega"]}
    if cache:
        name = torch.cuda.get_device_name(dev)
        d = load_cache(path)
        d[_key(W, H, precision, name)] = dict(best, when=time.time(), all=results)
        save_cache(d, path)
    return out
