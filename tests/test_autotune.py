"""Host logic of the launch-shape autotuner (CPU, with a stand-in simulator): every candidate is
a shape the library accepts, the fastest timed shape is applied and reported with the sweep,
shapes the library rejects are skipped, and a cached choice is reused without sweeping."""
import dataclasses

import pytest

from paper_1904_00011_gb300 import autotune


def _valid(block, split, chunk):
    """pcmd_set_launch: block 32..256 in steps of 32, block / split a multiple of 32, chunk 1..256."""
    return 32 <= block <= 256 and block % 32 == 0 and split >= 1 and block % (split * 32) == 0 \
        and 1 <= chunk <= 256


def test_every_default_candidate_is_a_valid_launch_shape():
    assert len(set(autotune.DEFAULT_CANDIDATES)) == len(autotune.DEFAULT_CANDIDATES)
    for shape in autotune.DEFAULT_CANDIDATES:
        assert _valid(*shape), shape


@dataclasses.dataclass
class _W:
    n_bands: int = 2
    flags: int = 0


class _FakeSim:
    """Times each shape by a fixed table; rejects shapes the library would reject."""

    def __init__(self, times):
        self.times = times
        self.shape = None
        self.applied = []
        self.n_points = 14700
        self.w = _W()
        self._prof = False
        self._runs = 0

    def set_launch(self, block, split, chunk):
        if not _valid(block, split, chunk):
            raise ValueError("rejected")
        self.shape = (block, split, chunk)
        self.applied.append(self.shape)

    def simulate(self, params, n_ims, set_id):
        if self._prof:
            self._runs += 1

    def sync(self):
        pass

    def profile(self, on):
        self._prof = on
        if on:
            self._runs = 0

    def kernel_times(self):
        return {"draw": (self.times[self.shape] * self._runs, self._runs)}


def test_tune_applies_the_fastest_shape_and_skips_rejected_ones(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "stand-in")
    times = {(256, 4, 64): 0.9, (256, 1, 32): 0.6, (128, 2, 64): 0.7}
    cands = list(times) + [(256, 3, 64)]              # 256 / 3 is not a multiple of 32
    sim = _FakeSim(times)
    best = autotune.tune(sim, [None], [256], candidates=cands, reps=2, use_cache=True)
    assert (best["block"], best["split"], best["chunk"]) == (256, 1, 32)
    assert sim.shape == (256, 1, 32) and not best["cached"]
    assert [tuple(r[:3]) for r in best["sweep"]] == [(256, 1, 32), (128, 2, 64), (256, 4, 64)]
    # a second tuner call on the same workload takes the cached shape without timing anything
    sim2 = _FakeSim({k: 1.0 for k in times})
    again = autotune.tune(sim2, [None], [256], candidates=cands, use_cache=True)
    assert again["cached"] and sim2.applied == [(256, 1, 32)]


def test_tune_raises_when_no_candidate_runs(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "stand-in")
    sim = _FakeSim({})
    with pytest.raises(RuntimeError, match="no candidate"):
        autotune.tune(sim, [None], [256], candidates=[(256, 3, 64), (48, 1, 64)], use_cache=False)


def test_cache_key_covers_every_size_and_the_parameters(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "stand-in")
    from paper_1904_00011_gb300 import workloads as W
    sim = _FakeSim({})
    p = W.full().params[0]
    sizes = [128, 144, 160, 176, 192, 512]
    k0 = autotune._key(sim, sizes, False, [p])
    # a size in the middle of the list changes the key (not only the first four and last two)
    assert autotune._key(sim, sizes[:4] + [208] + sizes[5:], False, [p]) != k0
    # another Npix (the sampler mix) changes the key
    q = dataclasses.replace(p, log_sfh=p.log_sfh + 3.0)
    assert autotune._key(sim, sizes, False, [q]) != k0
    assert autotune._key(sim, sizes, False, [p]) == k0
