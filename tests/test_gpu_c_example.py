"""The C ABI from a plain C program (tests/abi_example.c, linked against the
in-tree library): its spkMC runs (Sec. 3.1 steps 1-6, eight rotating
colours of Sec. 3.2 step 4a) end where the oracle's do -- the flip and null
counts, the exact null-rate sum, M, B and the spins' up count bit for bit,
the clock within 1e-12 relative."""
import os

import pytest

import oracle
from test_abi import build_abi_example

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.mark.parametrize("L,d,J,H,T,seed,cycles", [
    (128, 8, 1.0, 0.0, 4.5115, 2, 800),   # 128^3 with d = 8, hot start seed 2
    (64, 4, -0.5, 0.02, 3.0, 7, 400),     # antiferromagnetic coupling, field, other edge
    (32, 16, 1.0, 0.01, 5.5, 11, 64),     # the 16-site edge on a 2-domain lattice
])
def test_c_program_matches_the_oracle(tmp_path, L, d, J, H, T, seed, cycles):
    import subprocess
    exe = build_abi_example(tmp_path)
    r = subprocess.run([exe, str(L), str(d), repr(J), repr(H), repr(T), str(seed), str(cycles)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = dict(kv.split("=") for kv in r.stdout.split())
    st = oracle.State(L, d, J, H, T, seed)
    st.run(cycles, threads=THREADS)
    M, B = st.observables()
    assert int(got["cycle"]) == cycles == st.cycle
    assert (int(got["n_flip"]), int(got["n_null"])) == (st.n_flip, st.n_null)
    assert int(got["null_fx_lo"]) | (int(got["null_fx_hi"]) << 64) == st.null_fx
    assert (int(got["M"]), int(got["B"])) == (M, B)
    assert int(got["up"]) == int((st.spins > 0).sum())
    assert float.fromhex(got["clock"]) == pytest.approx(st.clock, rel=1e-12, abs=0.0)
