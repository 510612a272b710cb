"""Mistakes planted in the oracle must fail its pins.

Each mutant below is one plausible slip in oracle/spkmc_oracle.c: a wrong
sign, a dropped term, a neighbour or an axis taken wrong, a swapped operand,
a wrong random word, an index off by one, a bound read the other way.  It is
planted in a copy of the oracle package in a temporary folder; the pin tests
of tests/test_oracle_pins.py then run against that copy (CPU only) and must
fail.  An unmodified copy must pass them.  So the pins are checked against
the mistakes they exist to catch, not only against the oracle they were
written beside.  The oracle in the repository is never modified."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spkmc_oracle.c")

# name -> (text of the oracle, its replacement); each text occurs once
MUTANTS = {
    # Eq. 3, the Glauber rate
    "rate sign": ("r[c] = 1.0 / (1.0 + exp(x));", "r[c] = 1.0 / (1.0 + exp(-x));"),
    "rate factor of two": ("double x = dE / T;", "double x = dE / (2.0 * T);"),
    "field dropped": ("field = field + H;", "field = field + 0.0 * H;"),
    "field sign": ("field = field + H;", "field = field - H;"),
    # the six neighbours and the class of Sec. 3.1 step 1
    "neighbour axis": ("    u += s[gidx(L, X, Y, wrap(Z + 1, L))] > 0;",
                       "    u += s[gidx(L, X, wrap(Y + 1, L), Z)] > 0;"),
    "neighbour dropped": ("    u += s[gidx(L, X, wrap(Y - 1, L), Z)] > 0;\n", ""),
    "class spin swapped": ("return 7 * up + up_neighbours(L, s, X, Y, Z);",
                           "return 7 * (1 - up) + up_neighbours(L, s, X, Y, Z);"),
    # the counter-based random numbers and the hot start
    "philox Weyl constant": ("#define PHILOX_W1 0xBB67AE8584CAA73BULL", "#define PHILOX_W1 0xBB67AE8584CAA73DULL"),
    "philox words swapped": ("c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;",
                             "c[0] = n0; c[1] = lo0; c[2] = n2; c[3] = lo1;"),
    "hot start bit order": ("s[g] = ((w[b / 64] >> (b % 64)) & 1) ? 1 : -1;",
                            "s[g] = ((w[b % 4] >> (b / 4)) & 1) ? 1 : -1;"),
    # Eq. 1 and Eq. 4
    "bond dropped": ("s[gidx(L, X, Y, wrap(Z + 1, L))]);", "0);"),
    "magnetisation": ("                M += si;", "                M += si > 0;"),
    # Sec. 3.2 step 4a, the sublattice
    "colour shifted": ("if (sublattice == ORACLE_SUB_8_ROTATING) return (int)(t % 8);",
                       "if (sublattice == ORACLE_SUB_8_ROTATING) return (int)((t + 1) % 8);"),
    "active domain axis": ("*dx = 2 * (int)(a % h) + (c & 1);", "*dx = 2 * (int)(a % h) + ((c >> 1) & 1);"),
    "two-colour parity": ("*dx = 2 * (int)(a % h) + ((*dy + *dz + c) & 1);",
                          "*dx = 2 * (int)(a % h) + ((*dy + c) & 1);"),
    # Sec. 3.1 steps 1-4: frequency line, R_max, the event and its site
    "rate of another class": ("sum = sum + (double)n[q] * rate[q];", "sum = sum + (double)n[q] * rate[13 - q];"),
    "R_max as a minimum": ("if (cum[14 * a + 13] > Rmax) Rmax = cum[14 * a + 13];",
                           "if (Rmax == 0.0 || cum[14 * a + 13] < Rmax) Rmax = cum[14 * a + 13];"),
    "line not padded": ("double target = u01 * R;", "double target = u01 * cum[14 * a + 13];"),
    "rank from another word": ("uint64_t j = (uint64_t)(((u128)w[1] * nc) >> 64);",
                               "uint64_t j = (uint64_t)(((u128)w[2] * nc) >> 64);"),
    "rank off by one": ("if (seen == j) ev_site[a] = (int32_t)l;",
                        "if (seen == (j > 0 ? j - 1 : 0)) ev_site[a] = (int32_t)l;"),
    "local x and y swapped": ("int x = (int)(l % d), y = (int)((l / d) % d), z = (int)(l / ((int64_t)d * d));",
                              "int y = (int)(l % d), x = (int)((l / d) % d), z = (int)(l / ((int64_t)d * d));"),
    # Sec. 3.1 step 5, the clock, and Eq. 10's null rates
    "clock xi": ("double xi = (double)(2 * (wc[0] >> 12) + 1) * 0x1p-53;", "double xi = (double)(wc[0] >> 11) * 0x1p-53;"),
    "clock stream": ("oracle_philox((uint64_t)t, 0, 2, 0, seed, 0, wc);", "oracle_philox((uint64_t)t, 0, 1, 0, seed, 0, wc);"),
    "null rate of another class": ("acc += to_fixed64(R - cum[14 * a + 13]);", "acc += to_fixed64(R - cum[14 * a + 12]);"),
    # Sec. 3.2 step 4b, the bounds
    "bound field sign": ("const double dE = (6.0 * fabs(J) + fabs(H)) * -2.0 / T;",
                         "const double dE = (6.0 * fabs(J) - fabs(H)) * -2.0 / T;"),
    "margin halved": ("*margin = a + 12.0 * b;", "*margin = a + 6.0 * b;"),
    "learned from the last cycle": ("const double learned = (hist[0] + R_margin) * ORACLE_BOUND_SLACK;",
                                    "const double learned = (hist[7] + R_margin) * ORACLE_BOUND_SLACK;"),
    # the serial references: BKL (Sec. 4) and exact enumeration
    "BKL time step": ("double dt = -log(xi) / Rtot;", "double dt = -log(xi) / (Rtot + 1.0);"),
    "bond energy dropped": ("bonds += s[i] * (s[nb[1]] + s[nb[3]] + s[nb[5]]);", "bonds += s[i] * (s[nb[1]] + s[nb[3]]);"),
    "Boltzmann weight": ("double wgt = exp(-(E - Emin) / T);", "double wgt = exp(-(E - Emin) / (2.0 * T));"),
    "class BKL neighbour not moved": ("for (int a = 0; a < 7; ++a) {", "for (int a = 0; a < 6; ++a) {"),
}


def run_pins(folder, source):
    """The pins of tests/test_oracle_pins.py against a copy of the oracle
    package whose C source is `source`, built in `folder`."""
    os.makedirs(os.path.join(folder, "oracle"))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(folder, "oracle"))
    with open(os.path.join(folder, "oracle", "spkmc_oracle.c"), "w") as f:
        f.write(source)
    os.makedirs(os.path.join(folder, "tests"))
    for name in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", name), os.path.join(folder, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(folder, "tests", "golden"))
    env = dict(os.environ, PYTHONPATH=folder)
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                           "-p", "no:cacheprovider"], cwd=folder, env=env, capture_output=True, text=True,
                          timeout=900)


def test_the_unmodified_copy_passes_the_pins(tmp_path):
    r = run_pins(str(tmp_path / "unmodified"), open(SRC).read())
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, name

    def plant(item):
        i, (name, (old, new)) = item
        return name, run_pins(str(tmp_path / f"m{i}"), src.replace(old, new))

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(ex.map(plant, enumerate(MUTANTS.items())))
    # a pin failed (exit 1 with a failure), not the harness (collection, import)
    survivors = {name: r.stdout[-1500:] + r.stderr[-800:] for name, r in results.items()
                 if not (r.returncode == 1 and " failed" in r.stdout)}
    assert not survivors, survivors
