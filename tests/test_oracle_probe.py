"""Pins of the oracle's probe-weighted displacement (Sec. II.C, Eq. 17):

* the weights sum to 1, follow the probe's pulse table when f is constant,
  and vanish where no bound electrons are left (f = 0);
* over a window symmetric about the pulse centre the weighted mean time is
  the centre (symmetry), and a falling f moves it earlier;
* a constant displacement comes back unchanged, and the weights of a species
  follow its own bound fraction;
* the squared displacement of a rigid translation is its length squared, the
  same across a periodic face (minimum image); charge sums per species;
* the records of OracleMD: record 0 is the initial state (zero displacement).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_03180_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


PROBE = [W.Pulse(8.0, 15.0, 1e12, 40.0)]


def test_weights_normalised_and_follow_the_pulse():
    n, t0, dt = 400, 0.0, 0.2
    w = O.probe_weights(PROBE, t0, dt, np.ones(n))
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
    g = O.pulse_table(PROBE, t0, dt, n)
    assert np.allclose(w, g / g.sum(), rtol=1e-13, atol=0)
    f = np.ones(n)
    f[150:250] = 0.0
    w0 = O.probe_weights(PROBE, t0, dt, f)
    assert not w0[150:250].any() and w0.sum() == pytest.approx(1.0, rel=1e-14)
    assert not O.probe_weights(PROBE, t0, dt, np.zeros(n)).any()


def test_weighted_mean_time_is_the_centre_and_moves_with_f():
    tc, half, dt = 40.0, 60.0, 0.25
    n = int(round(2 * half / dt))
    t_mid = tc - half + dt * (np.arange(n) + 0.5)
    w = O.probe_weights(PROBE, tc - half, dt, np.ones(n))
    assert float((w * t_mid).sum()) == pytest.approx(tc, abs=1e-9)
    # atoms lose electrons during the probe, f linear in t: for a Gaussian g the
    # weighted mean time moves to t_c + sigma^2 f'(t_c) / f(t_c)
    b = 0.8 / (2 * half)
    f = 0.6 - b * (t_mid - tc)
    wf = O.probe_weights(PROBE, tc - half, dt, f)
    sig = PROBE[0].fwhm_fs / (2 * np.sqrt(2 * np.log(2)))
    assert float((wf * t_mid).sum()) == pytest.approx(tc - sig ** 2 * b / 0.6, abs=2e-3)


def test_weighted_displacement_of_simple_series():
    n, S = 300, 2
    q = np.zeros((n, S), np.int64)
    q[:, 1] = np.linspace(0, 6 * 10, n).astype(np.int64)  # 10 atoms of Z = 6 ionising to C6+
    d2 = np.zeros((n, S))
    d2[:, 0] = 4 * 0.3 ** 2                              # 4 atoms, 0.3 nm each, constant
    d2[:, 1] = 10 * (np.arange(n) * 1e-3) ** 2           # RMS displacement 1e-3 k
    D = O.probe_weighted_displacement(PROBE, 0.0, 0.3, q, d2, [4, 10], [1, 6])
    assert D[0] == pytest.approx(0.3, rel=1e-13)
    f = 1.0 - (q[:, 1] / 10.0) / 6.0
    w = O.probe_weights(PROBE, 0.0, 0.3, f)
    assert D[1] == pytest.approx(float((w * np.arange(n) * 1e-3).sum()), rel=1e-13)
    # the fully stripped late steps weigh nothing: less than with f = 1
    assert D[1] < float((O.probe_weights(PROBE, 0.0, 0.3, np.ones(n)) * np.arange(n) * 1e-3).sum())
    assert O.probe_weighted_displacement(PROBE, 0.0, 0.3, q, d2, [0, 10], [1, 6])[0] == 0.0


def test_probe_sums_translation_periodic_and_charges():
    rng = np.random.default_rng(4)
    x0 = rng.uniform(0, 2.0, (50, 3))
    sp = rng.integers(0, 3, 50)
    q = rng.integers(0, 4, 50)
    shift = np.array([0.3, -0.2, 0.1])
    vac = np.zeros((50, 3))
    qs, ds = O.probe_sums(x0 + shift, x0, q, sp, vac, 3)
    for k in range(3):
        assert qs[k] == q[sp == k].sum()
        assert ds[k] == pytest.approx((sp == k).sum() * float(shift @ shift), rel=1e-12)
    L = 2.0
    box = np.full((50, 3), L)
    qs2, ds2 = O.probe_sums(np.mod(x0 + shift, L), x0, q, sp, box, 3)
    assert np.array_equal(qs2, qs) and np.allclose(ds2, ds, rtol=1e-12)


def test_oracle_records_start_at_zero_displacement():
    wl = W.workload("c1_methane_1500", scale=0.05)
    atom = W.atomic_data(8.0, pi_scale=3000.0)
    md = O.OracleMD(wl.sample, atom, r_cut=1.2, t_start_fs=-5.0, pulses=wl.pulses, n_steps_max=20)
    for _ in range(5):
        md.step()
    qs, ds = md.probe_series(0)
    assert qs.shape == (6, 5) and ds.shape == (6, 5)
    assert not ds[0].any() and (ds[1:, [0, 1]] > 0).all()
    assert np.array_equal(qs[-1], [int(md.q[md.sp == k].sum()) for k in range(5)])
    assert (np.diff(ds[:, 1]) > 0).all()                  # carbons drift away from the start
