"""Model check of the cycle kernel's synchronisation between CTAs (host
logic, no GPU).

The kernel runs many spkMC cycles (Sec. 3.1 steps 1-6, eight colours in
rotation, Sec. 3.2 step 4a) in one launch.  Each CTA holds a contiguous range
of the colour's active domains in (ax, ay, az) order, the same range in every
cycle.  Between cycles it does not always wait for the whole grid:
  - within a cycle, with the exact R_max, every CTA's step 1 precedes every
    CTA's prepass and flip step (barrier 1, Sec. 3.1 step 2);
  - after an even cycle, a CTA waits for the CTAs that share a row of domains
    (fixed dy, dz) with its own items (the row waits);
  - after an odd cycle t it waits for nobody with the exact R_max (barrier 1
    of the next cycle orders what must be ordered); with the bounds of
    Sec. 3.2 step 4b, which have no barrier 1, the whole grid meets.

This test builds, on small lattices and for several grid sizes, every access
of every cycle at the granularity of a domain's rows, each of its six ghost
faces, and its count line:
  - staging and step 1 read the rows, the ghost faces and the count line of
    the active domain;
  - the flip step reads the rows of its face and edge neighbours (sites two
    steps out, diagonal sites), XORs bits into its own rows and into the
    ghost faces of its face neighbours that mirror it, adds class moves to
    their count lines (atomics, which commute among themselves) and stores its
    own count line (a plain store).
  - the ring of exact R_max maxima: every CTA's maximum of cycle t into slot
    t mod 16 (an atomic), the clear of slot t + 4 by the CTA holding the
    first domain, and the read of slot t (exact, after barrier 1) or t - 8
    (the learned bound, at the start of the cycle).
Each pair of accesses of different CTAs in different cycles that conflict
(a write against a read, or a plain store against any write) must be ordered
by the kernel's happens-before relation: program order in each CTA, barrier 1,
the row waits and the grid barriers.  A plausible mistake in the schedule --
the row wait taken after odd cycles instead of even ones, the row wait
narrowed to the CTA itself, or, with the bounds, the grid barrier skipped
after t = 3, 7 mod 8 (where cycles t + 1 and t + 2 follow without one, so
the flip steps of cycles t - 1 and t + 1, and of t and t + 2, whose colours
differ in the y and z bits, could overlap) -- must fail it."""
import itertools

import pytest


def items(nd):
    h = nd // 2
    return h * h * h


def domain_of(a, c, nd):
    """Active domain of item a in colour c (parity bits x, y, z)."""
    h = nd // 2
    ax, ay, az = a % h, (a // h) % h, a // (h * h)
    return (2 * ax + (c & 1), 2 * ay + ((c >> 1) & 1), 2 * az + ((c >> 2) & 1))


def shift(d, delta, nd):
    return tuple((d[i] + delta[i]) % nd for i in range(3))


UNIT = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
EDGE = [tuple(sa * (i == a) + sb * (i == b) for i in range(3))
        for a, b in itertools.combinations(range(3), 2) for sa in (-1, 1) for sb in (-1, 1)]


def accesses(dom, nd):
    """(phase, object, kind) of one active domain's cycle; phase 0 = staging and
    step 1, phase 1 = prepass and flip step; kind r = read, a = atomic write,
    w = plain write.  A block is its rows and its six ghost faces; ghost face
    i of D mirrors the boundary plane of D's neighbour across direction i."""
    faces = [shift(dom, u, nd) for u in UNIT]
    edges = [shift(dom, e, nd) for e in EDGE]
    acc = [(0, ("rows", dom), "r")] + [(0, ("ghost", dom, i), "r") for i in range(6)]
    acc += [(0, ("cnt", dom), "r")]
    # the flip step reads the rows of the face and edge neighbours
    acc += [(1, ("rows", f), "r") for f in faces] + [(1, ("rows", e), "r") for e in edges]
    # and writes the flipped bit, the ghost face of each face neighbour that
    # mirrors this domain (direction i ^ 1 seen from the neighbour), the class
    # moves of the neighbours' sites and its own count line
    acc += [(1, ("rows", dom), "a")] + [(1, ("ghost", f, i ^ 1), "a") for i, f in enumerate(faces)]
    acc += [(1, ("cnt", f), "a") for f in faces] + [(1, ("cnt", dom), "w")]
    return acc


def conflict(k1, k2):
    if k1 == "r" and k2 == "r":
        return False
    if k1 == "a" and k2 == "a":
        return False  # atomic adds and XORs commute
    return True


def cta_ranges(nd, G):
    Q = items(nd)
    return [(Q * b // G, Q * (b + 1) // G) for b in range(G)]


def owner(a, ranges):
    for b, (lo, hi) in enumerate(ranges):
        if lo <= a < hi:
            return b
    raise AssertionError(a)


def row_wait_set(b, ranges, nd):
    """CTAs that hold items of a row (fixed ay, az) that CTA b holds items of."""
    lo, hi = ranges[b]
    if lo >= hi:
        return {b}
    h = nd // 2
    r0, r1 = (lo // h) * h, (hi - 1) // h * h + h - 1
    return {owner(r0, ranges), owner(r1, ranges)} | set(range(owner(r0, ranges), owner(r1, ranges) + 1))


def end_sync(t, mode):
    """What the kernel does after cycle t (t = the lattice's cycle index)."""
    if t % 2 == 0:
        return "row"
    return "none" if mode == "exact" else "grid"


def happens_before(nd, G, mode, t0, ncycles, end_rule=end_sync, row_rule=row_wait_set):
    """Reachability between the events of every CTA's cycles: node (b, g, k)
    with k = 0 start, 1 end of step 1 (arrival), 2 start of the prepass,
    3 end of the flip step.  Returns a function hb(u, v)."""
    ranges = cta_ranges(nd, G)
    succ = {}

    def edge(u, v):
        succ.setdefault(u, set()).add(v)

    for b in range(G):
        for g in range(ncycles):
            edge((b, g, 0), (b, g, 1))
            edge((b, g, 1), (b, g, 2))
            edge((b, g, 2), (b, g, 3))
            if g + 1 < ncycles:
                edge((b, g, 3), (b, g + 1, 0))
    for g in range(ncycles):
        t = t0 + g
        if mode == "exact":
            for x in range(G):
                for y in range(G):
                    edge((y, g, 1), (x, g, 2))
        if g + 1 < ncycles:
            kind = end_rule(t, mode)
            for x in range(G):
                if kind == "grid":
                    src = range(G)
                elif kind == "row":
                    src = row_rule(x, ranges, nd)
                elif isinstance(kind, tuple) and kind[0] == "set":
                    src = kind[1][x]
                else:
                    src = ()
                for y in src:
                    edge((y, g, 3), (x, g + 1, 0))
    reach = {}

    def closure(u):
        if u in reach:
            return reach[u]
        seen, stack = set(), [u]
        while stack:
            w = stack.pop()
            for v in succ.get(w, ()):
                if v not in seen:
                    seen.add(v)
                    stack.append(v)
        reach[u] = seen
        return seen

    return ranges, lambda u, v: v in closure(u)


def ring_accesses(t, b, first, mode, ring=32, clear=8):
    """The ring of exact R_max maxima (cycle t in slot t mod ring): in cycle t
    every CTA takes its maximum into slot t after step 1 (an atomic); the CTA
    holding the lattice's first domain clears slot t + clear in its prepass (a
    plain store); the exact mode reads slot t in the prepass, after barrier 1,
    and the learned bound reads slot t - 8 at the start of the cycle."""
    acc = [(0, ("ring", t % ring), "a")]
    if b == first:
        acc.append((1, ("ring", (t + clear) % ring), "w"))
    if mode == "exact":
        acc.append((1, ("ring", t % ring), "r"))
    else:
        acc.append((0, ("ring", (t - 8) % ring), "r"))
    return acc


def unordered_conflicts(nd, G, mode, t0, ncycles, ring=32, clear=8, **kw):
    ranges, hb = happens_before(nd, G, mode, t0, ncycles, **kw)
    Q = items(nd)
    by_obj = {}  # object -> list of (g, cta, phase, kind)
    for g in range(ncycles):
        c = (t0 + g) % 8
        for a in range(Q):
            b = owner(a, ranges)
            for ph, obj, kind in accesses(domain_of(a, c, nd), nd):
                by_obj.setdefault(obj, []).append((g, b, ph, kind))
        # the ring (every CTA with items takes part; the first domain's CTA clears)
        for b in range(G):
            if ranges[b][0] < ranges[b][1]:
                for ph, obj, kind in ring_accesses(t0 + g, b, owner(0, ranges), mode, ring, clear):
                    # a learned read of a slot written before the launch is not a conflict here
                    if kind == "r" and mode != "exact" and g < 8:
                        continue
                    by_obj.setdefault(obj, []).append((g, b, ph, kind))
    bad = []
    for obj, acc in by_obj.items():
        for (g1, b1, p1, k1), (g2, b2, p2, k2) in itertools.combinations(sorted(acc), 2):
            if g1 == g2 or b1 == b2 or not conflict(k1, k2):
                continue
            # the earlier cycle's access must end before the later one starts
            u = (b1, g1, 1 if p1 == 0 else 3)
            v = (b2, g2, 0 if p2 == 0 else 2)
            if not hb(u, v):
                bad.append((obj, (g1, b1, p1, k1), (g2, b2, p2, k2)))
    return bad


CASES = [(4, 3), (8, 3), (8, 5), (8, 7), (8, 16), (12, 20), (16, 30)]


@pytest.mark.parametrize("mode", ["exact", "bound"])
@pytest.mark.parametrize("nd,G", CASES)
@pytest.mark.parametrize("t0", [0, 1, 3, 6])
def test_kernel_schedule_orders_every_conflict(nd, G, mode, t0):
    assert unordered_conflicts(nd, G, mode, t0, 12) == []


def test_row_waits_after_odd_cycles_fail():
    def swapped(t, mode):
        r = end_sync(t, mode)
        return "row" if t % 2 == 1 and r == "none" else ("none" if r == "row" else r)
    assert unordered_conflicts(8, 5, "exact", 0, 12, end_rule=swapped)


def test_bound_modes_need_a_barrier_after_every_odd_cycle():
    def skip_3_7(t, mode):  # the barrier after t = 3, 7 mod 8 skipped
        r = end_sync(t, mode)
        return "none" if r == "grid" and t % 4 == 3 else r

    def skip_1_5(t, mode):
        r = end_sync(t, mode)
        return "none" if r == "grid" and t % 4 == 1 else r
    assert unordered_conflicts(8, 5, "bound", 0, 12, end_rule=skip_1_5)
    bad = unordered_conflicts(8, 5, "bound", 0, 12, end_rule=skip_3_7)
    assert bad
    # without the barrier after t = 3, 7 what goes unordered is the flip steps
    # of cycles t - 1 and t + 1, or t and t + 2: colours two cycles apart that
    # differ in the y and z bits
    assert all(p1 == p2 == 1 for _, (g1, b1, p1, k1), (g2, b2, p2, k2) in bad)
    assert {(g1 % 8, g2 % 8) for _, (g1, *_), (g2, *_) in bad} <= {(2, 4), (3, 5), (6, 0), (7, 1)}


def test_row_wait_on_the_cta_alone_fails():
    assert unordered_conflicts(8, 5, "exact", 0, 12, row_rule=lambda b, ranges, nd: {b})


# ---- several lattices in one launch (the batched ensembles and the served
# stream): the lattices' active domains are concatenated in one item range,
# each lattice keeps its own cycle index (all with the launch's parity), the
# row waits use the segment-aware row edges, and with the bounds the grid
# meets after every odd cycle (the near wait is for single-lattice launches).

def batch_unordered_conflicts(nds, t0s, modes, G, ncycles, own_rows_only=False):
    assert len({t % 2 for t in t0s}) == 1  # the row waits need one parity
    bases, Q = [], 0
    for nd in nds:
        bases.append(Q)
        Q += items(nd)
    ranges = [(Q * b // G, Q * (b + 1) // G) for b in range(G)]
    exact_any = "exact" in modes

    def seg_of(q):
        j = 0
        while j + 1 < len(bases) and bases[j + 1] <= q:
            j += 1
        return j

    def row_edge(q, end):
        j = seg_of(q)
        h = nds[j] // 2
        r0 = bases[j] + ((q - bases[j]) // h) * h
        return r0 + h - 1 if end else r0

    def rows(b, ranges_, nd_):
        lo, hi = ranges_[b]
        if lo >= hi or own_rows_only:
            return {b}
        c0, c1 = owner(row_edge(lo, False), ranges_), owner(row_edge(hi - 1, True), ranges_)
        return set(range(c0, c1 + 1))

    def rule(t, mode):  # t = the launch's cycle with the shared parity
        if t % 2 == 0:
            return "row"
        return "none" if exact_any else "grid"

    succ = {}

    def edge(u, v):
        succ.setdefault(u, set()).add(v)
    for b in range(G):
        for g in range(ncycles):
            edge((b, g, 0), (b, g, 1))
            edge((b, g, 1), (b, g, 2))
            edge((b, g, 2), (b, g, 3))
            if g + 1 < ncycles:
                edge((b, g, 3), (b, g + 1, 0))
    for g in range(ncycles):
        if exact_any:
            for x in range(G):
                for y in range(G):
                    edge((y, g, 1), (x, g, 2))
        if g + 1 < ncycles:
            kind = rule(t0s[0] + g, None)
            for x in range(G):
                src = range(G) if kind == "grid" else (rows(x, ranges, None) if kind == "row" else ())
                for y in src:
                    edge((y, g, 3), (x, g + 1, 0))
    reach = {}

    def hb2(u, v):
        if u not in reach:
            seen, stack = set(), [u]
            while stack:
                w = stack.pop()
                for n in succ.get(w, ()):
                    if n not in seen:
                        seen.add(n)
                        stack.append(n)
            reach[u] = seen
        return v in reach[u]

    by_obj = {}
    for g in range(ncycles):
        for j, nd in enumerate(nds):
            c = (t0s[j] + g) % 8
            for a in range(items(nd)):
                b = owner(bases[j] + a, ranges)
                for ph, obj, kind in accesses(domain_of(a, c, nd), nd):
                    by_obj.setdefault((j,) + obj, []).append((g, b, ph, kind))
    bad = []
    for obj, acc in by_obj.items():
        for (g1, b1, p1, k1), (g2, b2, p2, k2) in itertools.combinations(sorted(acc), 2):
            if g1 == g2 or b1 == b2 or not conflict(k1, k2):
                continue
            if not hb2((b1, g1, 1 if p1 == 0 else 3), (b2, g2, 0 if p2 == 0 else 2)):
                bad.append((obj, (g1, b1, p1, k1), (g2, b2, p2, k2)))
    return bad


@pytest.mark.parametrize("nds,t0s", [((4, 8), (0, 2)), ((8, 4, 4), (1, 5, 3)), ((4, 4, 8), (6, 0, 2))])
@pytest.mark.parametrize("modes", [("exact",), ("bound",), ("exact", "bound")])
@pytest.mark.parametrize("G", [3, 5, 9])
def test_batched_launch_schedule_orders_every_conflict(nds, t0s, modes, G):
    mode_of = [modes[i % len(modes)] for i in range(len(nds))]
    assert batch_unordered_conflicts(nds, t0s, mode_of, G, 10) == []


def test_batched_row_wait_on_the_cta_alone_fails():
    assert batch_unordered_conflicts((4, 8), (0, 2), ("exact", "exact"), 5, 10, own_rows_only=True)


def wide_wait_rows(b, ranges, nd, max_list=128):
    """The kernel's wait set after an odd cycle with the bounds: every CTA
    holding an item of the rows y - 1, y, y + 1 of the planes z - 1, z, z + 1
    of a row (y, z) of CTA b (each index wrapping), built from row runs: a run
    of b's rows within one plane maps to a run of whole rows of each image
    plane, with the row that the y shift wraps taken on its own."""
    lo, hi = ranges[b]
    h = nd // 2
    if lo >= hi:
        return {b}
    out = []
    r0, r1 = lo // h, (hi - 1) // h
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            r = r0
            while r <= r1:
                ay, az = r % h, r // h
                e = min((az + 1) * h - 1, r1)
                if (dy < 0 and ay == 0) or (dy > 0 and ay == h - 1):
                    e = r
                elif dy > 0:
                    e = min(e, az * h + h - 2)  # stop before the row that wraps
                first = (((ay + dy) % h) + h * ((az + dz) % h)) * h
                c0, c1 = owner(first, ranges), owner(first + (e - r + 1) * h - 1, ranges)
                for c in range(c0, c1 + 1):
                    if c not in out:
                        out.append(c)
                r = e + 1
    if len(out) > max_list:
        return set(range(len(ranges)))
    return set(out) | {b}


def wide_rule_for(t0, sets):
    """The bound modes' schedule: the grid after every 8th cycle of the launch,
    otherwise the row wait after even cycles and the wide wait after odd ones."""
    def rule(t, mode):
        g = t - t0
        if mode != "exact" and g % 8 == 7:
            return "grid"
        if t % 2 == 0:
            return "row"
        return "none" if mode == "exact" else ("set", sets)
    return rule


@pytest.mark.parametrize("nd,G", CASES)
@pytest.mark.parametrize("t0", [0, 1, 3, 6])
def test_bound_modes_with_wide_waits_and_a_grid_barrier_every_8_cycles(nd, G, t0):
    ranges = cta_ranges(nd, G)
    sets = {b: wide_wait_rows(b, ranges, nd) for b in range(G)}
    assert unordered_conflicts(nd, G, "bound", t0, 20, end_rule=wide_rule_for(t0, sets)) == []
    assert unordered_conflicts(nd, G, "exact", t0, 20, end_rule=wide_rule_for(t0, sets)) == []


def test_a_grid_barrier_every_8_cycles_needs_the_32_slot_ring():
    nd, G, t0 = 24, 60, 0
    ranges = cta_ranges(nd, G)
    sets = {b: wide_wait_rows(b, ranges, nd) for b in range(G)}
    assert max(len(v) for v in sets.values()) < G // 2
    rule = wide_rule_for(t0, sets)
    assert unordered_conflicts(nd, G, "bound", t0, 24, end_rule=rule, ring=32, clear=8) == []
    bad = unordered_conflicts(nd, G, "bound", t0, 24, end_rule=rule, ring=16, clear=4)
    assert bad and all(obj[0] == "ring" for obj, *_ in bad)


def test_a_near_wait_confined_to_the_own_plane_fails():
    nd, G, t0 = 8, 5, 0
    ranges = cta_ranges(nd, G)

    def same_plane(b):
        lo, hi = ranges[b]
        h = nd // 2
        out = {b}
        for a in range(lo, hi):
            ax, ay, az = a % h, (a // h) % h, a // (h * h)
            for dy in (-1, 0, 1):
                out.add(owner(ax + h * ((ay + dy) % h) + h * h * az, ranges))
        return out
    sets = {b: same_plane(b) for b in range(G)}
    assert unordered_conflicts(nd, G, "bound", t0, 20, end_rule=wide_rule_for(t0, sets))


def test_without_the_grid_barrier_every_8_cycles_only_the_ring_races():
    # on a lattice large enough that the near waits are local, they order
    # every block, ghost and count access, but without a grid barrier the
    # CTAs drift apart and the clear of a ring slot races with its maxima and
    # reads
    nd, G, t0 = 24, 60, 0
    ranges = cta_ranges(nd, G)
    sets = {b: wide_wait_rows(b, ranges, nd) for b in range(G)}
    assert max(len(v) for v in sets.values()) < G // 4

    def no_grid(t, mode):
        return "row" if t % 2 == 0 else ("set", sets)
    bad = unordered_conflicts(nd, G, "bound", t0, 24, end_rule=no_grid)
    assert bad and all(obj[0] == "ring" for obj, *_ in bad)
    assert unordered_conflicts(nd, G, "bound", t0, 24, end_rule=wide_rule_for(t0, sets)) == []



def kernel_code():
    """The cycle kernel's code (its translation unit and internal header)
    without comments, whitespace collapsed."""
    import os
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = []
    for f in ("spkmc_kernels.cu", "spkmc_internal.h"):
        with open(os.path.join(root, "paper_1005_4713_gb300", "csrc", f)) as fh:
            text.append(bench._code_text(fh.read()))
    return " ".join(" ".join(text).split())


# The lines of the kernel whose schedule this file models.  A change to any of
# them must come with a change to the model above (and a new proof).
KERNEL_SCHEDULE = [
    # the R_max ring: 32 slots, the learned bound reads t - 8, slot t + 8 is
    # cleared at t (ring_accesses, ring=32, clear=8)
    "constexpr int kRmaxRing = 32;",
    "rmax[(t - 8) & (kRmaxRing - 1)]",
    "P.state[slot].rmax[(t + 8) & (kRmaxRing - 1)] = 0ULL;",
    # barrier 1 only when some lattice pads to the exact R_max
    "if (P.exact_any && !grid_barrier(P, S, epoch)) {",
    # the end of a cycle (end_sync, wide_rule_for)
    "const bool skip = odd && P.exact_any;",
    "const bool grid8 = !P.exact_any && (g & 7LL) == 7LL;",
    "const bool near = odd && !P.exact_any && !grid8 && P.done && P.nseg == 1;",
    "if (skip) { __syncthreads(); } else if (even && P.done && !grid8) { if (!row_wait(P, S, g)) return; } "
    "else if (near) { if (!near_wait(P, S, g)) return; } else if (!grid_barrier(P, S, epoch)) { return; }",
    # the near set: rows y - 1 .. y + 1 of planes z - 1 .. z + 1, at most 128
    # CTAs before it becomes every CTA (wide_wait_rows, max_list=128)
    "for (int dz = -1; dz <= 1 && S.nnear >= 0; ++dz) { for (int dy = -1; dy <= 1 && S.nnear >= 0; ++dy) {",
    "constexpr int kMaxNear = 128;",
    "if (S.nnear == kMaxNear) S.nnear = -1;",
]


@pytest.mark.parametrize("line", KERNEL_SCHEDULE)
def test_the_model_is_the_kernels_schedule(line):
    assert " ".join(line.split()) in kernel_code(), line
