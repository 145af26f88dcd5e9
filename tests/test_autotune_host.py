"""Host logic of the per-size kernel choice: picking the fastest finite time
and reusing a persisted table without re-timing (the C library is replaced by
a stand-in; no GPU)."""
import math

import numpy as np
import pytest

import paper_1605_04718_gb300 as rd
from paper_1605_04718_gb300 import autotune as at


def test_fastest_skips_missing_kernels():
    assert at.fastest([2e-3, 1e-3, math.nan]) == rd.RD_KERNEL_TC_STACKED
    assert at.fastest([2e-3, 3e-3, 1e-3]) == rd.RD_KERNEL_TC_RESIDENT
    assert at.fastest([5e-3, math.nan, math.nan]) == rd.RD_KERNEL_SIMT
    with pytest.raises(ValueError):
        at.fastest([math.nan] * 3)


class _FakeLib:
    """Stands in for the C entry points tune() uses."""

    def __init__(self, times):
        self.times = np.asarray(times, dtype=float)
        self.kernel = {}
        self.ctas = {}
        self.calls = 0

    def autotune(self, p, theta, n_trials, probe_steps, n_sizes):
        self.calls += 1
        for s in range(n_sizes):
            self.kernel[s] = at.fastest(self.times[s])
        return self.times[:n_sizes]

    def set_kernel(self, p, s, k):
        self.kernel[s] = k

    def get_kernel(self, p, s):
        return self.kernel[s]

    def set_schedule(self, p, s, c):
        self.ctas[s] = c

    def get_schedule(self, p, s):
        return 2 if self.kernel[s] == rd.RD_KERNEL_TC_STACKED else 1


def test_tune_times_once_then_reuses_the_table(tmp_path, monkeypatch):
    fake = _FakeLib([[3e-3, 1e-3, math.nan], [9e-3, 4e-3, 2e-3]])
    monkeypatch.setattr(at, "rd_autotune", fake.autotune)
    monkeypatch.setattr(at, "rd_set_size_kernel", fake.set_kernel)
    monkeypatch.setattr(at, "rd_get_size_kernel", fake.get_kernel)
    monkeypatch.setattr(at, "rd_set_size_schedule", fake.set_schedule)
    monkeypatch.setattr(at, "rd_get_size_schedule", fake.get_schedule)
    path = str(tmp_path / "kernels.json")
    theta = np.zeros((8, 4))
    out = at.tune(None, "GPU-X", 2, [64, 128], 8000, theta, cache_path=path)
    assert fake.calls == 1
    assert [out[s]["kernel"] for s in (0, 1)] == ["tc_stacked", "tc_resident"]
    assert out[0]["seconds_per_proposal"]["tc_resident"] is None
    fake.kernel = {}
    again = at.tune(None, "GPU-X", 2, [64, 128], 8000, theta, cache_path=path)
    assert fake.calls == 1 and all(again[s]["cached"] for s in (0, 1))
    assert fake.kernel == {0: rd.RD_KERNEL_TC_STACKED, 1: rd.RD_KERNEL_TC_RESIDENT}
    assert fake.ctas == {0: 2, 1: 1}  # the persisted schedules are applied too
    # another GPU, step count or size is a different key: timed again
    at.tune(None, "GPU-Y", 2, [64, 128], 8000, theta, cache_path=path)
    at.tune(None, "GPU-X", 2, [64, 96], 8000, theta, cache_path=path)
    assert fake.calls == 3
    assert len(at.load_table(path)) == 5
