"""Host-side check of the geometry behind the grid barriers between cycles
of the eight rotating colours (Sec. 3.2 step 4a with colour t mod 8 =
parity bits of the domain coordinates).

A flip moves the class of each neighbour site j of the flipped site, and
the new class depends on the spins of all of j's neighbours.  Two colours
whose flips may run at the same time must therefore have no site j next to
both of them.  Two consecutive cycles t, t + 1 (t odd) whose flips are not
ordered by a barrier may overlap safely only when their colours differ in all
three parity bits (t = 3, 7 mod 8).  This test enumerates the sites of a
small lattice to confirm that statement for every pair of colours.  Whether
the cycle kernel's barriers and waits order everything that must be ordered,
across all cycles and CTAs, is checked by tests/test_sync_schedule.py."""
import itertools

import pytest


def colour_of_site(x, y, z, d):
    return ((x // d) & 1) | (((y // d) & 1) << 1) | (((z // d) & 1) << 2)


def neighbours(x, y, z, L):
    for ax in range(3):
        for step in (-1, 1):
            p = [x, y, z]
            p[ax] = (p[ax] + step) % L
            yield tuple(p)


def shared_neighbour_exists(c1, c2, L, d):
    """Some site has a neighbour of colour c1 and a neighbour of colour c2."""
    for x, y, z in itertools.product(range(L), repeat=3):
        cols = {colour_of_site(*n, d) for n in neighbours(x, y, z, L)}
        if c1 in cols and c2 in cols:
            return True
    return False


@pytest.mark.parametrize("L,d", [(4, 2), (8, 2), (8, 4)])
def test_flips_of_two_colours_interact_unless_they_differ_in_three_bits(L, d):
    for c1, c2 in itertools.combinations(range(8), 2):
        bits = bin(c1 ^ c2).count("1")
        assert shared_neighbour_exists(c1, c2, L, d) == (bits <= 2), (c1, c2)


def test_consecutive_colours_after_odd_cycles():
    # the pairs the kernel may overlap without the exact R_max's barrier:
    # (t, t + 1) with t = 3, 7 mod 8 differ in three bits; t = 1, 5 in two
    three = [t for t in range(1, 8, 2) if bin(t ^ ((t + 1) % 8)).count("1") == 3]
    assert three == [3, 7]
    assert all(t % 4 == 3 for t in three)
