"""Host logic of the continuous-batching server, on CPU: the batch is a fake
that advances budgets and reports completions like spkmc_batch_*, so the
admission, memory accounting, retry and rejection rules are checked without
a GPU."""
import ctypes

import pytest

import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import serve
from paper_1005_4713_gb300 import workloads as wl


class FakeBatch:
    """spkmc_batch_* as the server uses it: slots with cycle budgets; the
    cycles a slot runs each count K_act events (flips + nulls)."""
    fail_admit = {}  # seed -> number of admissions that fail with ENOMEM first
    instances = []

    def __init__(self, capacity, config=None):
        self.capacity = capacity
        self.slots = {}
        self.reported = set()
        self.log = []
        FakeBatch.instances.append(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def admit(self, L, d, J, H, T, seed, cold=False, cycles=-1):
        if FakeBatch.fail_admit.get(seed, 0) > 0:
            FakeBatch.fail_admit[seed] -= 1
            raise sp.SpkmcError(sp.SPKMC_ENOMEM, "device allocation failed")
        slot = next(i for i in range(self.capacity) if i not in self.slots)
        d = d or sp.spkmc_resolve_domain_edge(L)
        self.slots[slot] = {"L": L, "kact": (L // d // 2) ** 3, "budget": cycles, "t": 0, "seed": seed}
        self.log.append(("admit", seed, len(self.slots)))
        return slot

    def run(self, n):
        self.log.append(("run", n, len(self.slots)))
        for s in self.slots.values():
            s["t"] += n if s["budget"] < 0 else min(n, s["budget"] - s["t"])

    def poll(self):
        done = [i for i, s in self.slots.items() if s["budget"] >= 0 and s["t"] >= s["budget"]
                and i not in self.reported]
        self.reported.update(done)
        return done

    def observables_all(self):
        out = (sp.spkmc_obs * self.capacity)()
        for i, s in self.slots.items():
            out[i].cycle = s["t"]
            out[i].n_null = s["t"] * s["kact"] // 5
            out[i].n_flip = s["t"] * s["kact"] - out[i].n_null
        return out

    def retire(self, slot):
        del self.slots[slot]
        self.reported.discard(slot)
        self.log.append(("retire", slot, len(self.slots)))

    def spins(self, slot):
        return None


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    FakeBatch.fail_admit = {}
    FakeBatch.instances = []
    return FakeBatch


def requests(n, L=32, d=4, cycles=250):
    return [wl.Request(rid=i, arrival=0.0, spec=wl.LatticeSpec(L=L, d=d, seed=100 + i), cycles=cycles)
            for i in range(n)]


def need(L, d):
    return sp.spkmc_bytes_required(sp.make_params(L, d))


def test_budget_and_capacity_hold_at_every_step(fake):
    reqs = requests(9)
    budget = 3 * need(32, 4)  # three lattices at a time

    def check(stats, active):
        assert len(active) <= 2
        assert sum(b for _, _, b in active.values()) <= budget

    stats = serve.Server(budget, capacity=2, step_cycles=100).serve(reqs, realtime=False, on_step=check)
    assert sorted(c.rid for c in stats.completions) == list(range(9))
    assert stats.peak_live == 2 and not stats.rejected


def test_events_come_from_the_lattice_counters(fake):
    # d = 0: the edge is resolved by the library; the event count is the
    # lattice's flips + nulls, whatever the edge
    reqs = requests(3, L=64, d=0, cycles=130)
    stats = serve.Server(1 << 40, step_cycles=50).serve(reqs, realtime=False)
    kact = (64 // sp.spkmc_resolve_domain_edge(64) // 2) ** 3
    assert [c.events for c in stats.completions] == [130 * kact] * 3


def test_a_full_device_makes_a_request_wait(fake):
    # the second lattice's first two admissions fail while the first runs:
    # it is tried again at the following step boundaries, then admitted;
    # nothing is rejected and both complete
    reqs = requests(2)
    fake.fail_admit = {101: 2}
    stats = serve.Server(1 << 40, step_cycles=100).serve(reqs, realtime=False)
    assert sorted(c.rid for c in stats.completions) == [0, 1] and not stats.rejected
    log = fake.instances[0].log
    admitted = log.index(("admit", 101, 2))
    assert [e[0] for e in log[:admitted]] == ["admit", "run", "run"]


def test_a_failed_admission_with_nothing_live_is_rejected(fake):
    reqs = requests(3)
    fake.fail_admit = {100: 1}  # the first request fails with an empty device
    stats = serve.Server(1 << 40, step_cycles=100).serve(reqs, realtime=False)
    assert stats.rejected == [0]
    assert sorted(c.rid for c in stats.completions) == [1, 2]


def test_a_request_larger_than_the_budget_is_rejected(fake):
    reqs = requests(2) + [wl.Request(rid=9, arrival=0.0, spec=wl.LatticeSpec(L=128, d=8, seed=7), cycles=10)]
    stats = serve.Server(2 * need(32, 4), step_cycles=100).serve(reqs, realtime=False)
    assert stats.rejected == [9]
    assert sorted(c.rid for c in stats.completions) == [0, 1]


def test_cancellation_drops_a_request_at_the_next_step(fake):
    reqs = requests(2, cycles=10_000)
    srv = serve.Server(1 << 40, step_cycles=100)

    def cancel_second(stats, active):
        if stats.steps == 3:
            srv.cancel(1)

    stats = srv.serve(reqs, realtime=False, on_step=cancel_second)
    by = {c.rid: c for c in stats.completions}
    assert by[1].cancelled and by[1].cycles == 300
    assert not by[0].cancelled and by[0].cycles == 10_000
