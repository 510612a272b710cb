"""The autotuner on the GPU: the launch geometry it picks (and every candidate
it tries) runs the same trajectory as the default launch, bit for bit, for a
lattice and for a batch."""
import numpy as np
import pytest

import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import autotune, ensemble
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def key(o):
    return (o.cycle, o.clock, o.M, o.B, o.n_flip, o.n_null, int(o.sum_null_rate_fx[0]), int(o.sum_null_rate_fx[1]))


@pytest.fixture()
def tmp_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("SPKMC_TUNE_CACHE", str(tmp_path / "tune.json"))


def test_tuned_lattice_reproduces_the_default_trajectory(tmp_cache):
    L, d, seed, n = 64, 4, 91, 150
    entry = autotune.tune_launch(L, d, cycles=16)
    assert autotune.cached_launch(L, d) == (entry["items_per_cta"], entry["ctas_per_sm"])
    with sp.Lattice(L, d, 1.0, 0.0, 4.5115, seed, tuned=False) as ref:
        ref.run(n)
        want, spins = key(ref.observables()), ref.spins()
        grid_default = ref.info().grid_ctas
    with sp.Lattice(L, d, 1.0, 0.0, 4.5115, seed) as lat:  # picks the cached geometry
        assert (lat.config.items_per_cta, lat.config.ctas_per_sm) == autotune.cached_launch(L, d)
        lat.run(n)
        assert key(lat.observables()) == want
        assert np.array_equal(lat.spins(), spins)
    grids = {grid_default}
    for ipc, cps in autotune.LAUNCH_CANDIDATES:
        with sp.Lattice(L, d, 1.0, 0.0, 4.5115, seed, config=sp.make_config(items_per_cta=ipc, ctas_per_sm=cps)) as lat:
            lat.run(n)
            grids.add(lat.info().grid_ctas)
            assert key(lat.observables()) == want, (ipc, cps)
            assert np.array_equal(lat.spins(), spins)
    assert len(grids) > 1  # the candidates really launch different grids


def test_tuned_batch_reproduces_the_default_results(tmp_cache):
    specs = wl.ensemble_specs(12)
    specs = [wl.LatticeSpec(L=s.L, d=2, T=s.T, H=s.H, seed=s.seed) for s in specs]
    autotune.tune_batch(specs, cycles=16)
    assert autotune.cached_batch(specs) is not None
    a = ensemble.run_batched(specs, 120, sample_every=40, tuned=False)
    b = ensemble.run_batched(specs, 120, sample_every=40)
    assert a.final == b.final
