"""Pins of the oracle's Langevin electron-ion coupling (Sec. II.B, Eqs. 13-14):
the Gaussians are standard normal and independent; with k_B T_e = 0 the
velocities decay as c^n = e^{-gamma n dt} exactly; free particles reach
equipartition <m v^2> = k_B T_e per component; the velocity autocorrelation
is e^{-gamma t} (Ornstein-Uhlenbeck); the charge dynamics does not see it."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def test_gaussians_standard_normal_and_independent():
    from scipy import stats
    g = O.gaussians(99, np.arange(100_000), 3)
    assert np.abs(g.mean(0)).max() < 0.015
    assert np.abs(g.var(0) - 1).max() < 0.015
    for k in range(3):
        assert stats.kstest(g[:, k], "norm").pvalue > 1e-3
    g2 = O.gaussians(99, np.arange(100_000), 4)      # next step
    g3 = O.gaussians(100, np.arange(100_000), 3)     # another seed
    for other in (g2, g3):
        assert abs(np.corrcoef(g[:, 0], other[:, 0])[0, 1]) < 0.015
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 0.015


def test_friction_only_decays_exactly():
    v0 = np.random.default_rng(1).normal(size=(50, 3))
    gam, dt = 3.0, 0.01
    v = v0.copy()
    for n in range(100):
        v = O.langevin_update(v, 12.0, gam, 0.0, dt, O.gaussians(5, np.arange(50), n))
    assert np.allclose(v, v0 * np.exp(-gam * dt) ** 100, rtol=1e-12, atol=0)


def test_equipartition_at_the_electron_temperature():
    n, m, gam, dt, kT = 4000, 12.0, 5.0, 0.01, 2.5   # kT in kJ/mol
    v = np.zeros((n, 3))
    ids = np.arange(n)
    for k in range(600):                              # 30 relaxation times
        v = O.langevin_update(v, m, gam, kT, dt, O.gaussians(11, ids, k))
    t = m * (v ** 2).mean()
    assert t == pytest.approx(kT, rel=0.03)


def test_velocity_autocorrelation_is_exponential():
    n, m, gam, dt, kT = 20000, 1.0, 2.0, 0.05, 1.0
    v0 = np.random.default_rng(2).normal(size=(n, 3)) * np.sqrt(kT / m)
    v = v0.copy()
    ids = np.arange(n)
    for k in range(10):
        v = O.langevin_update(v, m, gam, kT, dt, O.gaussians(21, ids, k))
        ac = (v0 * v).mean() / (v0 * v0).mean()
        assert ac == pytest.approx(np.exp(-gam * dt * (k + 1)), abs=0.02)


def test_charges_unaffected_and_zero_coupling_is_plain_verlet():
    from paper_2401_03180_gb300 import workloads as W
    wl = W.workload("c1_methane_1500", scale=0.1)
    s = wl.sample
    atom = W.atomic_data(8.0, pi_scale=3000.0, ci_scale=20.0)
    pulses = [W.Pulse(8.0, 5.0, 1e12, 0.0)]
    kw = dict(r_cut=1.2, t_start_fs=-2.0, pulses=[pulses], n_steps_max=40)
    plain = O.OracleMD(s, atom, **kw)
    zero = O.OracleMD(s, atom, langevin_g=np.zeros(5), **kw)
    hot = O.OracleMD(s, atom, langevin_g=np.full(5, 0.05), **kw)
    for _ in range(30):
        plain.step(); zero.step(); hot.step()
    assert np.array_equal(plain.x, zero.x) and np.array_equal(plain.v, zero.v)
    assert np.array_equal(plain.q, hot.q) and np.array_equal(plain.n_e, hot.n_e)
    assert plain.n_e[0] > 0 and not np.allclose(plain.v, hot.v, rtol=1e-9)
