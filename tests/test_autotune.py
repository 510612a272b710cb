"""The autotuner's choices, cache and wiring, from fake timings (no GPU)."""
import json

import pytest

import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import autotune, ensemble
from paper_1005_4713_gb300 import workloads as wl

DEV = "TestGPU"


@pytest.fixture()
def cache_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SPKMC_TUNE_CACHE", str(path))
    monkeypatch.setattr(autotune, "device_key", lambda: DEV)
    return path


def test_launch_choice_is_the_fastest_and_is_cached(cache_file):
    calls = []

    def fake(ipc, cps):
        calls.append((ipc, cps))
        # 96 items per CTA at the occupancy limit is fastest
        return {"s_per_cycle": 1e-5 + 1e-9 * abs(ipc - 96) + 1e-7 * cps, "events_per_s": 0.0}

    e = autotune.tune_launch(64, 4, measure=fake)
    assert (e["items_per_cta"], e["ctas_per_sm"]) == (96, 0)
    assert calls == list(autotune.LAUNCH_CANDIDATES)
    # persisted, keyed by device and (L, d); a second call does not measure
    stored = json.loads(cache_file.read_text())
    assert f"{DEV}|launch|L=64|d=4" in stored
    calls.clear()
    assert autotune.tune_launch(64, 4, measure=fake)["items_per_cta"] == 96
    assert calls == []
    assert autotune.cached_launch(64, 4) == (96, 0)
    assert autotune.cached_launch(64, 8) is None


def test_edge_is_chosen_on_flips_not_on_events(cache_file):
    # the smallest edge runs the most events but wastes more of them on nulls
    table = {16: (1.0e9, 0.95e9), 8: (1.5e9, 1.2e9), 4: (2.0e9, 1.1e9), 2: (3.0e9, 1.0e9)}

    def fake(d):
        ev, fl = table[d]
        return {"events_per_s": ev, "flips_per_s": fl, "s_per_cycle": 1e-5}

    assert autotune.choose_domain_edge(64, measure=fake) == 8
    entry = json.loads(cache_file.read_text())[f"{DEV}|edge|L=64"]
    assert entry["objective"] == "flips_per_s"
    assert set(entry["events_per_s"]) == {"16", "8", "4", "2"}


def test_resolved_edges_are_deterministic_and_reused(cache_file):
    seen = []

    def fake(L, d):
        seen.append((L, d))
        fl = 2.0 if (L == 24 and d == 2) else (1.0 if d == 4 else 0.5)
        return {"events_per_s": 1.0, "flips_per_s": fl, "s_per_cycle": 1.0}

    m1 = autotune.edge_map([16, 24, 16, 32], measure=fake)
    assert m1 == {16: 4, 24: 2, 32: 4}
    n = len(seen)
    m2 = autotune.edge_map([32, 24, 16], measure=fake)
    assert m2 == m1 and len(seen) == n  # from the cache, no new trial
    rep = autotune.edge_report([16, 24])
    assert rep["24"]["d"] == 2


def test_only_valid_edges_are_tried():
    assert autotune.valid_edges(24) == [4, 2]
    assert autotune.valid_edges(1024) == [16, 8, 4, 2]
    assert autotune.valid_edges(6) == []


def test_batch_key_follows_the_edge_mix_and_size(cache_file):
    a = [wl.LatticeSpec(L=32, d=2), wl.LatticeSpec(L=64, d=4)]
    b = [wl.LatticeSpec(L=64, d=4), wl.LatticeSpec(L=32, d=2)]
    c = [wl.LatticeSpec(L=32, d=4), wl.LatticeSpec(L=64, d=4)]
    assert autotune.batch_key(a) == autotune.batch_key(b)
    assert autotune.batch_key(a) != autotune.batch_key(c)
    e = autotune.tune_batch(a, measure=lambda ipc, cps: {"s_per_cycle": 1.0 / ipc, "events_per_s": 0.0})
    assert (e["items_per_cta"], e["ctas_per_sm"]) == (128, 0)
    assert autotune.cached_batch(b) == (128, 0)


def test_lattice_and_ensemble_configs_take_the_cached_geometry(cache_file):
    assert sp.tuned_config(64, 4, None) is None  # nothing tuned: library defaults
    autotune.tune_launch(64, 4, measure=lambda ipc, cps: {"s_per_cycle": 1.0 if ipc != 48 else 0.5})
    c = sp.tuned_config(64, 4, None)
    assert (c.items_per_cta, c.ctas_per_sm) == (48, 0)
    # a caller's own geometry wins, and other fields are kept
    mine = sp.make_config(items_per_cta=7, barrier_timeout_ns=123)
    assert sp.tuned_config(64, 4, mine) is mine
    base = sp.make_config(barrier_timeout_ns=456)
    c = sp.tuned_config(64, 4, base)
    assert (c.items_per_cta, c.barrier_timeout_ns) == (48, 456) and base.items_per_cta == 0
    specs = [wl.LatticeSpec(L=32, d=2), wl.LatticeSpec(L=64, d=4)]
    assert ensemble.batch_config(specs, None) is None
    autotune.tune_batch(specs, measure=lambda ipc, cps: {"s_per_cycle": 2.0 - cps})
    c = ensemble.batch_config(specs, None)
    assert (c.items_per_cta, c.ctas_per_sm) == (64, 1)


def test_a_spec_that_leaves_the_edge_to_the_library_is_keyed_by_the_resolved_edge():
    specs = [wl.LatticeSpec(L=64, d=0, seed=1), wl.LatticeSpec(L=48, d=0, seed=2)]
    resolved = [wl.LatticeSpec(L=64, d=sp.spkmc_resolve_domain_edge(64), seed=1),
                wl.LatticeSpec(L=48, d=sp.spkmc_resolve_domain_edge(48), seed=2)]
    assert [autotune.spec_edge(s) for s in specs] == [r.d for r in resolved]
    assert autotune.batch_key(specs, "dev") == autotune.batch_key(resolved, "dev")
