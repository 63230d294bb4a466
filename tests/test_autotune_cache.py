"""Host logic of the autotuner's cache (paper_1804_01390_gb300/autotune.py), with the
library calls replaced by a fake context: the chosen shape and the fastest one-step shape
(kept for single steps and the transposed step) are stored, and a cached entry restores
both without timing again."""
import json
import types

import pytest

from paper_1804_01390_gb300 import autotune


class FakeLib:
    """Variants 0..4: 0-2 advance one step per pass, 3-4 two; pml_autotune reports a table."""

    def __init__(self, times):
        self.times = list(times)
        self.selected = []
        self.cur = 0
        self.tuned = 0

    def pml_autotune(self, ctx, steps):
        self.tuned += 1
        best = min(range(len(self.times)), key=lambda v: self.times[v])
        self.cur = best
        return best, list(self.times)

    def pml_set_variant(self, ctx, v):
        self.cur = int(v)
        self.selected.append(int(v))

    def pml_get_time_block(self, ctx):
        return 2 if self.cur >= 3 else 1


@pytest.fixture
def fake(monkeypatch, tmp_path):
    lib = FakeLib([0.27, 0.38, 0.29, 0.17, 0.19])
    monkeypatch.setattr(autotune, "_lib", lib)
    monkeypatch.setattr(autotune, "_key", lambda solver: "dev|2d|fp32|160x160|w16")
    monkeypatch.setenv("PML_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    return lib


def _solver():
    return types.SimpleNamespace(ctx=object())


def test_tune_stores_choice_and_one_step_shape(fake, tmp_path):
    s = _solver()
    v, table = autotune.tune(s, steps=5)
    assert v == 3 and table[3] == pytest.approx(0.17)
    assert s.one_step_variant == 0                    # fastest among the one-step shapes 0..2
    assert fake.selected[-2:] == [0, 3]               # one-step shape first, then the choice
    rec = json.load(open(tmp_path / "cache.json"))["dev|2d|fp32|160x160|w16"]
    assert rec["variant"] == 3 and rec["one_step"] == 0


def test_cached_entry_skips_timing(fake):
    autotune.tune(_solver(), steps=5)
    assert fake.tuned == 1
    s = _solver()
    fake.selected.clear()
    v, table = autotune.tune(s, steps=5)
    assert fake.tuned == 1 and table is None and v == 3
    assert s.one_step_variant == 0 and fake.selected == [0, 3]


def test_retune_ignores_cache(fake):
    autotune.tune(_solver(), steps=5)
    autotune.tune(_solver(), steps=5, use_cache=False)
    assert fake.tuned == 2


def test_select_one_step_choice(fake):
    autotune.select(object(), 1, 1)
    assert fake.selected == [1]
    autotune.select(object(), 4, 2)
    assert fake.selected[-2:] == [2, 4]


def test_stale_cached_choice_is_timed_again(fake, tmp_path):
    """A cached index the library rejects (a build with fewer variants) falls back to
    timing instead of failing."""
    from paper_1804_01390_gb300 import _lib as real
    json.dump({"dev|2d|fp32|160x160|w16": {"variant": 9, "one_step": 9}}, open(tmp_path / "cache.json", "w"))

    def set_variant(ctx, v):
        if not 0 <= int(v) < len(fake.times):
            raise real.PMLError(real.PML_EINVAL, "variant out of range")
        fake.cur = int(v)
        fake.selected.append(int(v))

    fake.pml_set_variant = set_variant
    fake.PMLError = real.PMLError
    s = _solver()
    v, table = autotune.tune(s, steps=5)
    assert fake.tuned == 1 and v == 3 and table is not None
    assert json.load(open(tmp_path / "cache.json"))["dev|2d|fp32|160x160|w16"]["variant"] == 3
