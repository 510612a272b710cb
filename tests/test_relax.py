"""Relaxation harness: the bias of Eq. 8/9 against the serial reference of
Sec. 4, UR of Eq. 10, and the dynamic exponent of Eq. 13."""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1005_4713_gb300 import relax as rx


def test_effective_z_recovers_a_power_law():
    t = np.geomspace(0.1, 100, 40)
    for z in (2.04, 2.5):
        m = 0.9 * t ** (-rx.BETA_OVER_NU / z)
        zz = rx.effective_z(t, m, window=5)
        ok = np.isfinite(zz)
        assert ok.sum() == 36
        assert np.allclose(zz[ok], z, rtol=1e-10)


def test_bias_of_identical_ensembles_is_zero_and_shifts_are_seen():
    rng = np.random.default_rng(1)
    t = np.linspace(0.1, 5, 30)
    base = np.exp(-t / 3)
    ser = base + 0.01 * rng.standard_normal((20, 30))
    b_t, s_t, bi, sb = rx.bias(t, ser, ser, (0.5, 4.0))
    assert np.allclose(b_t, 0) and bi == 0.0 and sb > 0
    par = base + 0.05 + 0.01 * rng.standard_normal((20, 30))
    _, _, bi, sb = rx.bias(t, par, ser, (0.5, 4.0))
    assert abs(bi - 0.05) < 4 * sb and bi > 10 * sb


def serial_curves(L, times, n, seed0, T=rx.T_CRITICAL):
    def one(i):
        s = np.ones(L ** 3, dtype=np.int8)
        m, _, _ = oracle.bkl_relax((L, L, L), 1.0, 0.0, T, seed0 + i, s, times)
        return m
    with ThreadPoolExecutor(max_workers=8) as ex:  # the C calls release the GIL
        return np.array(list(ex.map(one, range(n))))


@pytest.mark.gpu
@pytest.mark.parametrize("d,sub", [(8, rx.SPKMC_SUBLATTICE_2_RANDOM), (8, rx.SPKMC_SUBLATTICE_8_ROTATING),
                                   (16, rx.SPKMC_SUBLATTICE_2_RANDOM)])
def test_bias_against_serial_bkl_64(d, sub):
    """64^3 (2^18 spins) from all +1 at T_c, 20 spkMC runs against 20 serial
    BKL runs: the time-integrated bias over 0.1 <= t <= 4 lies within 4
    sigma_b of zero; UR stays within (0.8, 1)."""
    L, n = 64, 20
    t = np.geomspace(0.05, 4.0, 30)
    par = rx.relax(L, d, t, n_runs=n, seed0=100, sublattice=sub)
    ser = serial_curves(L, t, n, 5000)
    b_t, s_t, bi, sb = rx.bias(t, par.m, ser, (0.1, 4.0))
    assert abs(bi) < 4 * sb, (bi, sb)
    se = np.sqrt(par.m.var(axis=0, ddof=1) / n + ser.var(axis=0, ddof=1) / n)
    assert np.all(np.abs(b_t) < 5 * se + 1e-12)
    ur = np.nanmean(par.ur[:, 5:])
    assert 0.8 < ur < 1.0
