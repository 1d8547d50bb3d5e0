"""Launch-shape autotuner of the draw kernel.

Sweeps (block threads, split = warp groups per pixel tile, chunk = point groups per shared-memory
stage) through ``pcmd_set_launch``, times the draw kernel with the library's CUDA-event hooks
(``pcmd_profile`` / ``pcmd_kernel_times``) and keeps the fastest shape.  Results are cached in a
JSON file keyed by GPU name and workload signature (image sizes, isochrone points, bands,
flags), so a second process picks the shape without sweeping.  Star counts do not depend on the
shape; only the FP32 summation order of the fluxes does.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

CACHE = os.environ.get("PCMD_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning.json"))

DEFAULT_CANDIDATES: List[Tuple[int, int, int]] = [
    (256, 4, 64), (256, 4, 128), (256, 4, 256), (256, 2, 64), (256, 2, 128), (256, 8, 64),
    (256, 8, 256), (256, 1, 64), (128, 2, 64), (128, 4, 64), (128, 1, 128), (256, 4, 32),
    (256, 8, 128), (128, 2, 128), (256, 2, 32), (256, 1, 32),
]


def _digest(values) -> str:
    h = hashlib.sha1()
    for v in values:
        h.update(repr(v).encode())
    return h.hexdigest()[:16]


def _key(sim, n_ims: Sequence[int], fused: bool, params=()) -> str:
    """Workload signature: GPU, points, bands, flags, every image size (hashed) and every
    parameter set's values (hashed: Npix, distance and dust set the mix of sparse, dense and
    transformed-rejection draws, hence the best shape)."""
    import torch
    name = torch.cuda.get_device_name()
    sizes = [int(n) for n in n_ims]
    pvals = []
    for p in params:
        if hasattr(p, "log_sfh"):
            pvals.append(tuple(round(float(x), 6) for x in list(p.log_sfh) +
                               [p.feh_mean, p.feh_sigma, p.log_ebv, p.dust_sigma, p.dmod]))
        else:
            pvals.append(repr(p))
    sig = "%s|P=%d|B=%d|flags=%d|sets=%d|sizes=%s|params=%s|fused=%d" % (
        name, sim.n_points, sim.w.n_bands, sim.w.flags, len(n_ims), _digest(sizes),
        _digest(pvals), int(fused))
    return sig


def _load() -> Dict[str, dict]:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: Dict[str, dict]) -> None:
    tmp = CACHE + ".tmp"
    try:
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def tune(sim, params, n_ims: Sequence[int], candidates: Optional[Iterable[Tuple[int, int, int]]] = None,
         reps: int = 3, fused: bool = False, mock=None, use_cache: bool = True) -> dict:
    """Pick and apply the fastest launch shape for ``sim`` on this workload.  ``fused`` times the
    fused batched evaluation (needs ``mock`` = (hess tensor, moments, n_pix, mode)) instead of
    the image-mode draw kernel."""
    key = _key(sim, n_ims, fused, params)
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        best = cache[key]
        sim.set_launch(best["block"], best["split"], best["chunk"])
        return dict(best, cached=True)
    results = []
    for (block, split, chunk) in (candidates or DEFAULT_CANDIDATES):
        try:
            sim.set_launch(block, split, chunk)
        except Exception:
            continue
        run = (lambda i: sim.evaluate(params, n_ims, *mock, first_set_id=900_000 + i)) if fused else \
              (lambda i: sim.simulate(params, n_ims, 900_000 + i))
        run(0)
        sim.sync()
        sim.profile(True)
        for i in range(reps):
            run(1 + i)
        kt = sim.kernel_times()
        sim.profile(False)
        ms, cnt = kt["graph"] if fused else kt["draw"]
        if cnt:
            results.append((ms / cnt, block, split, chunk))
    if not results:
        raise RuntimeError("autotune: no candidate launch shape could be run on this workload")
    results.sort()
    t, block, split, chunk = results[0]
    sim.set_launch(block, split, chunk)
    best = {"block": block, "split": split, "chunk": chunk, "ms": t,
            "sweep": [[b, s, c, round(m, 4)] for (m, b, s, c) in results]}
    if use_cache:
        cache = _load()
        cache[key] = best
        _store(cache)
    return dict(best, cached=False)
