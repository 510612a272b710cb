"""The entry point that allocates nothing (spkmc_run_cycles_noalloc), for
callers that cannot allocate device memory themselves (code running inside an
arena or pool owned by someone else, or that must not touch the CUDA
allocator), checked against the regular entry points on two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import paper_1005_4713_gb300 as sp

pytestmark = pytest.mark.gpu

CLOCK_RTOL = 1e-12


def test_no_alloc_matches_regular_entry_points_on_two_calls():
    torch = pytest.importorskip("torch")
    L, d, seed = 64, 8, 77
    p = sp.make_params(L, d, 1.0, 0.0, 4.5115, seed)
    with sp.Lattice(L, d, 1.0, 0.0, 4.5115, seed) as ref:
        dev = torch.from_numpy(ref.spins().copy()).to("cuda")
        torch.cuda.synchronize()
        state = sp.spkmc_state()
        for n in (25, 40):
            ref.run(n)
            sp.spkmc_run_cycles_noalloc(p, dev.data_ptr(), state, n)
            o = ref.observables()
            assert np.array_equal(dev.cpu().numpy(), ref.spins())
            assert (state.cycle, state.n_flip, state.n_null) == (o.cycle, o.n_flip, o.n_null)
            assert list(state.sum_null_rate_fx) == list(o.sum_null_rate_fx)
            assert state.clock == pytest.approx(o.clock, rel=CLOCK_RTOL)


def test_no_alloc_rejects_a_lattice_larger_than_its_array():
    torch = pytest.importorskip("torch")
    p = sp.make_params(512, 16)
    dev = torch.zeros(8, dtype=torch.int8, device="cuda")
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_run_cycles_noalloc(p, dev.data_ptr(), sp.spkmc_state(), 1)
    assert e.value.code == sp.SPKMC_EINVAL
    assert "no-allocation array" in sp.spkmc_last_error()
