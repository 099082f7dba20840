"""Host-side parts of the sweep server: the request generator and the EOS
set-up tables (checked against the oracle's independent Maxwell tools)."""
import numpy as np
import pytest

from oracle import physics as ph
from oracle.lbm import EOS
from paper_2112_01975_gb300 import eos_tables


def test_sweep_requests_deterministic_and_in_range():
    from paper_2112_01975_gb300 import serve
    a = serve.sweep_requests(count=200, rate=50.0, seed=5)
    b = serve.sweep_requests(count=200, rate=50.0, seed=5)
    assert a == b
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert np.all(gaps > 0)
    assert 0.7 / 50 < gaps.mean() < 1.3 / 50          # Poisson, mean 1/rate
    for r in a:
        assert 0.5 <= r.t_over_tc <= 0.95 and 0.15 <= r.radius_frac <= 0.35
        assert r.n % 32 == 0
        assert (64 <= r.n <= 192) if r.lattice == 1 else (64 <= r.n <= 512)
    frac3d = np.mean([r.lattice == 1 for r in a])
    assert 0.35 < frac3d < 0.65
    assert {r.storage for r in a} == {1, 2}                # FP32 and FP16-shifted
    assert 0.35 < np.mean([r.storage == 2 for r in a]) < 0.65


@pytest.mark.parametrize("eos,tr", [(0, 0.5), (0, 0.8), (0, 0.95), (1, 0.7)])
def test_set_up_tables_match_the_oracle(eos, tr):
    a = eos_tables.stable_a(eos, tr)
    rv, rl, ps = eos_tables.coexistence(eos, tr, a)
    e = EOS(eos, tr, a=a)
    ov, ol, ops = ph.maxwell(e)
    assert rv == pytest.approx(ov, rel=1e-8) and rl == pytest.approx(ol, rel=1e-8)
    assert eos_tables.kappa_for_width(eos, tr, a) == pytest.approx(
        ph.kappa_for_width(e, 5.0, (ov, ol, ops)), rel=1e-5)
    # the scaled attraction puts the liquid's dP/drho at (or below) 0.1
    h = 1e-6 * rl
    assert (e(rl + h) - e(rl - h)) / (2 * h) <= 0.1 + 1e-6


def test_setup_table_matches_direct_values():
    """The server's Chebyshev table of (a, rho_v, rho_l, kappa) over the
    sweep's T/Tc range reproduces the direct Maxwell/width computation at
    random T/Tc to 1e-7 relative (rho_v spans a factor of 40 there)."""
    t = eos_tables.SetupTable(0, 0.5, 0.95)
    rng = np.random.default_rng(3)
    for tr in rng.uniform(0.5, 0.95, 6):
        a = eos_tables.stable_a(0, tr)
        rv, rl, _ = eos_tables.coexistence(0, tr, a)
        k = eos_tables.kappa_for_width(0, tr, a)
        got = t(tr)
        for g, w in zip(got, (a, rv, rl, k)):
            assert g == pytest.approx(w, rel=1e-7)
    assert t(0.97)[2] == pytest.approx(eos_tables.coexistence(0, 0.97, eos_tables.stable_a(0, 0.97))[1])
