"""Mistakes planted in the oracle must fail its pins.

Each mutant below is one plausible slip in oracle/spkmc_oracle.c or in its
Python wrapper oracle/__init__.py: a wrong
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
WRAPPER = os.path.join(ROOT, "oracle", "__init__.py")

# name -> (text of oracle/spkmc_oracle.c, its replacement); each text occurs
# once.  Every mutant changes some result the pins can reach: a slip that is
# equal to the original on every input the pins use (floor(x 2^63) * 2 for
# floor(x 2^64), equal for x >= 2^-10; (w0 >> 12) 2^-52 for u01, within
# 2^-53 of it; the enumeration's ground-state shift, which cancels in every
# average; the class-grouped BKL's skip of a partner listed twice, whose
# second update finds the class already moved) is not one.
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
    # the history of R_max, the bound check and the fixed-point null sum
    "history records the bound": ("hist[7] = Rmax;", "hist[7] = R;"),
    "bound check off": ("if (R < Rmax) {", "if (R < 0.0) {"),
    "null sum scale": ("return (u128)ldexp(x, 64);", "return (u128)ldexp(x, 60);"),
    # the counters of the random streams
    "hot start stream": ("oracle_philox((uint64_t)(g / 256), 0, 3, 0, seed, 0, w);",
                         "oracle_philox((uint64_t)(g / 256), 0, 2, 0, seed, 0, w);"),
    "event counter by active index": ("oracle_philox((uint64_t)t, (uint64_t)k, 1, 0, seed, 0, w);",
                                      "oracle_philox((uint64_t)t, (uint64_t)a, 1, 0, seed, 0, w);"),
    "u01 from another word": ("double u01 = (double)(w[0] >> 11) * 0x1p-53;", "double u01 = (double)(w[1] >> 11) * 0x1p-53;"),
    "class BKL clock word": ("const double xi = (double)(2 * (w[2] >> 12) + 1) * 0x1p-53;",
                             "const double xi = (double)(2 * (w[3] >> 12) + 1) * 0x1p-53;"),
    "class BKL rank word": ("const uint64_t j = (uint64_t)(((u128)w[1] * (uint64_t)n[c]) >> 64);",
                            "const uint64_t j = (uint64_t)(((u128)w[2] * (uint64_t)n[c]) >> 64);"),
    "energy field sign": ("*E = -J * (double)bonds - H * (double)mag;", "*E = -J * (double)bonds + H * (double)mag;"),
    # the two-colour draw, the bounds' slack, the sampling of m(t)
    "two-colour draw bit": ("return (int)(w[0] >> 63);", "return (int)(w[0] & 1);"),
    "bound slack dropped": ("#define ORACLE_BOUND_SLACK (1.0 + 0x1p-32)", "#define ORACLE_BOUND_SLACK (1.0)"),
    "m sampled after the step": ("while (g < ntimes && times[g] < t + dt) m_out[g++] = (double)M / (double)N;",
                                 "while (g < ntimes && times[g] < t) m_out[g++] = (double)M / (double)N;"),
}

# name -> (text of oracle/__init__.py, its replacement): slips in the wrapper
WRAPPER_MUTANTS = {
    "wrapper M and B swapped": ("return int(M[0]), int(B[0])", "return int(B[0]), int(M[0])"),
    "wrapper null sum word": ("self.null_fx = int(fx[0]) | (int(fx[1]) << 64)",
                              "self.null_fx = int(fx[0]) | (int(fx[1]) << 63)"),
    "wrapper bounds swapped": ("return float(a[0]), float(b[0])", "return float(b[0]), float(a[0])"),
    "wrapper cold flag": ("lib().oracle_init_spins(L, seed, 1 if cold else 0, _p(s))",
                          "lib().oracle_init_spins(L, seed, 0 if cold else 1, _p(s))"),
}


def run_pins(folder, source, wrapper):
    """The pins of tests/test_oracle_pins.py against a copy of the oracle
    package with C source `source` and wrapper `wrapper`, built in `folder`."""
    os.makedirs(os.path.join(folder, "oracle"))
    for name, text in (("spkmc_oracle.c", source), ("__init__.py", wrapper)):
        with open(os.path.join(folder, "oracle", name), "w") as f:
            f.write(text)
    os.makedirs(os.path.join(folder, "tests"))
    for name in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", name), os.path.join(folder, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(folder, "tests", "golden"))
    env = dict(os.environ, PYTHONPATH=folder)
    # the copy's library is built first: a build that fails is the harness's
    # failure, not a pin's
    subprocess.run([sys.executable, "-c", "import oracle; oracle.build()"], cwd=folder, env=env, check=True,
                   capture_output=True, timeout=300)
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                           "-p", "no:cacheprovider"], cwd=folder, env=env, capture_output=True, text=True,
                          timeout=900)


def test_the_unmodified_copy_passes_the_pins(tmp_path):
    r = run_pins(str(tmp_path / "unmodified"), open(SRC).read(), open(WRAPPER).read())
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src, wrapper = open(SRC).read(), open(WRAPPER).read()
    plants = []
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, name
        plants.append((name, src.replace(old, new), wrapper))
    for name, (old, new) in WRAPPER_MUTANTS.items():
        assert wrapper.count(old) == 1, name
        plants.append((name, src, wrapper.replace(old, new)))

    def plant(item):
        i, (name, source, wrap) = item
        return name, run_pins(str(tmp_path / f"m{i}"), source, wrap)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(ex.map(plant, enumerate(plants)))
    # a pin failed (exit 1 with a failure), not the harness (collection, import)
    survivors = {name: r.stdout[-1500:] + r.stderr[-800:] for name, r in results.items()
                 if not (r.returncode == 1 and " failed" in r.stdout)}
    assert not survivors, survivors
