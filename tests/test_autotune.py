"""Autotuner: host-side cache logic (CPU) and, on a GPU, that a tuned context
computes exactly what an untuned one does."""
import numpy as np
import pytest

from paper_2111_04577_gb300 import autotune, binding, build, workloads as wl


def test_signature_and_cache_roundtrip(tmp_path):
    g = wl.Grid(32, 1, 16, 4.0, 4.0 / 32, 2.0, 1)
    k1 = autotune.signature(g, binding.PF_MIXED)
    k2 = autotune.signature(g, binding.PF_FP64)
    assert k1 != k2 and "32x1x16" in k1
    path = str(tmp_path / "t.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({k1: {"xfft_pairs": 2}}, path)
    assert autotune.load_cache(path)[k1]["xfft_pairs"] == 2
    # every knob shapes at least one kernel the library profiles
    for name, cands, kernels in autotune.KNOBS.values():
        assert cands and kernels


@pytest.mark.gpu
def test_tuned_context_matches_default():
    build.build()
    w = wl.scaled(wl.config("c4"), 16, 8)
    g = w.grid
    choice = autotune.tune(g, w.params, binding.PF_MIXED, steps=1)
    for knob, (name, cands, _) in autotune.KNOBS.items():
        if name in choice:
            assert choice[name] in cands
    phi0 = wl.initial_phi(w)
    a = binding.Solver(g, w.params, binding.PF_MIXED)
    b = binding.Solver(g, w.params, binding.PF_MIXED)
    autotune.apply(b, choice)
    for s in (a, b):
        s.load_state(phi0)
        s.step(3)
    assert np.array_equal(a.get("phi"), b.get("phi"))
    assert np.array_equal(a.get("u"), b.get("u"))


@pytest.mark.gpu
@pytest.mark.parametrize("knob", sorted(autotune.KNOBS))
def test_every_candidate_matches_default(knob):
    """Each launch shape a knob offers computes the same bits as the built-in
    one: the knobs change how work is split, never the arithmetic of a cell."""
    build.build()
    w = wl.scaled(wl.config("c4"), 32, 16)
    g = w.grid
    name, cands, _ = autotune.KNOBS[knob]
    phi0 = wl.initial_phi(w)
    ref = binding.Solver(g, w.params, binding.PF_MIXED)
    ref.load_state(phi0)
    ref.step(3)
    for v in cands:
        s = binding.Solver(g, w.params, binding.PF_MIXED)
        s.set_tuning(knob, int(v))
        s.load_state(phi0)
        s.step(3)
        for f in ("phi", "u", "w", "p"):
            assert np.array_equal(ref.get(f), s.get(f)), (name, v, f)
