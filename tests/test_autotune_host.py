"""The launch-shape autotuner's search and cache, on the host with synthetic
timing functions (no GPU)."""
import json

import pytest

from paper_2603_24027_gb300 import _capi as A
from paper_2603_24027_gb300 import autotune as T
from paper_2603_24027_gb300 import inputs as I

START = {"zgroups": 0, "zchunk": 8, "zchunk_fwd": -1, "zchunk_fwd2": -1, "tile_y": 8,
         "stages": 2}


class FakeSim:
    """Option store with the library's defaults and a workload."""

    def __init__(self, w=None, opts=None):
        self.w = w or I.ragged_box()
        self.opts = {A.OPT_KERNEL: 5, A.OPT_ZGROUPS: 0, A.OPT_ZCHUNK: 8, A.OPT_ZCHUNK_FWD: -1,
                     A.OPT_ZCHUNK_FWD2: -1, A.OPT_TILE_Y: 8, A.OPT_STAGES: 2,
                     A.OPT_EXACT_REVERSAL: 0}
        self.opts.update(opts or {})

    def get_option(self, oid):
        return self.opts[oid]

    def set_option(self, oid, v):
        self.opts[oid] = v


def separable(best, scale=1.0):
    """Cost with its minimum at `best`, one term per option."""
    order = {name: list(vals) for name, _, vals in T.SPACE}

    def cost(o):
        assert T.valid(o), o
        return scale * (1.0 + sum(0.1 * abs(order[k].index(o[k]) - order[k].index(best[k]))
                                  for k in best))
    return cost


class Counter:
    def __init__(self, f):
        self.f, self.calls = f, []

    def __call__(self, o):
        self.calls.append(tuple(sorted(o.items())))
        return self.f(o)


def test_search_reaches_a_separable_minimum_and_times_each_setting_once():
    target = {"zgroups": 3, "zchunk": 6, "zchunk_fwd": 8, "zchunk_fwd2": 64, "tile_y": 4,
              "stages": 3}
    m = Counter(separable(target))
    best, t, tried = T.search(m, START)
    assert best == target
    assert len(m.calls) == len(set(m.calls)) == len(tried)


def test_search_needs_a_second_pass_for_coupled_options():
    """Height 16 runs only with 3 stages: the first pass moves to 3 stages,
    the second then finds height 16."""
    def cost(o):
        assert T.valid(o), o
        c = 1.0
        if o["stages"] == 3:
            c -= 0.1
        if o["tile_y"] == 16:
            c -= 0.3
        return c
    best, t, tried = T.search(cost, START)
    assert best["tile_y"] == 16 and best["stages"] == 3
    assert t == pytest.approx(0.6)


def test_search_ignores_gains_below_the_noise_floor():
    def cost(o):
        return 1.0 - (0.005 if o["zgroups"] == 6 else 0.0)
    best, _, _ = T.search(cost, START)
    assert best == START


def test_invalid_shapes_are_never_timed():
    assert not T.valid(dict(START, tile_y=16, stages=2))
    assert not T.valid(dict(START, tile_y=3))
    assert not T.valid(dict(START, stages=5))
    assert not T.valid(dict(START, zgroups=17))
    assert T.valid(dict(START, tile_y=16, stages=3))
    with pytest.raises(ValueError):
        T.search(lambda o: 1.0, dict(START, tile_y=16))


def test_cache_key_separates_what_changes_the_best_shape():
    w = I.ragged_box()
    rec = A.record_cfg("bf16", 4)
    k = T.cache_key("GB300", w, 5, rec)
    assert k != T.cache_key("B200", w, 5, rec)
    assert k != T.cache_key("GB300", w.replace(nx=w.nx + 1), 5, rec)
    assert k != T.cache_key("GB300", w.replace(pml_thickness=w.pml_thickness + 1), 5, rec)
    assert k != T.cache_key("GB300", w, 4, rec)
    assert k != T.cache_key("GB300", w, 5, A.record_cfg("bf16", 2))
    assert k != T.cache_key("GB300", w, 5, A.record_cfg("bdct10", 4))
    assert k == T.cache_key("GB300", w.replace(n_steps=w.n_steps + 7), 5, rec)


def test_tune_applies_caches_and_reuses(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    rec = A.record_cfg("bf16", 4)
    target = {"zgroups": 4, "zchunk": 10, "zchunk_fwd": 16, "zchunk_fwd2": -1, "tile_y": 8,
              "stages": 2}
    sim = FakeSim()
    r = T.tune(sim, None, rec, cache=path, measure=separable(target), gpu_name="GB300")
    assert not r["cached"] and r["options"] == target
    for name, value in target.items():
        assert sim.get_option(T.OPTION_IDS[name]) == value
    data = json.load(open(path))
    key = T.cache_key("GB300", sim.w, 5, rec)
    assert data[key]["options"] == target and data[key]["trials"] == r["trials"]

    def boom(o):
        raise AssertionError("a cache hit must not time anything")
    other = FakeSim()
    r2 = T.tune(other, None, rec, cache=path, measure=boom, gpu_name="GB300")
    assert r2["cached"] and r2["options"] == target
    assert other.get_option(A.OPT_ZCHUNK) == 10

    # another GPU type or tape misses the cache; refresh re-times
    r3 = T.tune(FakeSim(), None, rec, cache=path, measure=separable(START), gpu_name="B200")
    assert not r3["cached"] and r3["options"] == START
    r4 = T.tune(FakeSim(), None, rec, cache=path, measure=separable(START), gpu_name="GB300",
                refresh=True)
    assert not r4["cached"] and r4["options"] == START
    assert len(json.load(open(path))) == 2


def test_tune_leaves_other_kernels_and_exact_shapes_alone(tmp_path):
    path = str(tmp_path / "tune.json")
    rec = A.record_cfg("f32", 1)

    def boom(o):
        raise AssertionError("kernels other than 5 are not tuned")
    sim = FakeSim(opts={A.OPT_KERNEL: 0})
    r = T.tune(sim, None, rec, cache=path, measure=boom, gpu_name="GB300")
    assert r["options"] == {} and r["trials"] == 0

    seen = []

    def cost(o):
        seen.append(set(o))
        return 1.0 - 0.1 * (o.get("zgroups") == 3)
    sim = FakeSim(opts={A.OPT_EXACT_REVERSAL: 16})
    r = T.tune(sim, None, rec, cache=path, measure=cost, gpu_name="GB300")
    assert all(s == {"zgroups", "zchunk", "zchunk_fwd", "zchunk_fwd2"} for s in seen)
    assert r["options"]["zgroups"] == 3 and sim.get_option(A.OPT_TILE_Y) == 8


def test_unreadable_cache_is_empty(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert T.load_cache(str(p)) == {}
    assert T.load_cache(str(tmp_path / "missing.json")) == {}
    T.save_entry(str(p), "k", {"options": {}})
    assert T.load_cache(str(p)) == {"k": {"options": {}}}


def test_gpu_timing_wrapper_drives_a_trial_copy(tmp_path, monkeypatch):
    """gpu_measure's own logic with the simulation class and the device
    synchronisation replaced by fakes: the trial copy is shortened, inherits
    the handle's fixed options, receives each candidate, and its loop times
    (median of reps, after one untimed run) become the search's costs."""
    import torch
    from paper_2603_24027_gb300 import fdtd

    made = []

    class TrialSim(FakeSim):
        def __init__(self, w, device=None):
            super().__init__(w)
            self.device, self.runs = device, 0
            made.append(self)

        def forward(self, eps, rec):
            self.runs += 1

        def backward(self, seed):
            pass

        def last_timing(self):
            # forward cost falls with more z groups; the first (untimed) run is slow
            g = self.opts[A.OPT_ZGROUPS]
            slow = 100.0 if self.runs % 3 == 1 else 0.0
            return {"fwd_ms": 10.0 - 0.5 * g + slow, "bwd_ms": 20.0}

    monkeypatch.setattr(fdtd, "Simulation", TrialSim)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    w = I.ragged_box().replace(n_steps=500)
    sim = FakeSim(w, opts={A.OPT_USE_GRAPHS: 1, A.OPT_PDL: 0,
                           A.OPT_PREFETCH: 0, A.OPT_TILE_X: 40, A.OPT_COMPACT_AUX: 1})
    eps = torch.zeros(1)
    r = T.tune(sim, eps, A.record_cfg("bf16", 4), cache=str(tmp_path / "t.json"),
               trial_steps=50, reps=2, gpu_name="GB300", max_passes=1)
    (trial,) = made
    assert trial.w.n_steps == 50 and trial.device == eps.device
    assert trial.opts[A.OPT_TILE_X] == 40 and trial.opts[A.OPT_KERNEL] == 5
    assert r["options"]["zgroups"] == 8 and sim.get_option(A.OPT_ZGROUPS) == 8
    assert r["seconds"] == pytest.approx((10.0 - 4.0 + 20.0) / 1e3)
