"""Pins of the oracle's pulse integral, plasma scalars and stochastic CR
update (no GPU).

Sec. II.A: charges are integers drawn stochastically so that ensemble
averages follow rate equations.  The oracle's Monte-Carlo histograms are
compared with (i) closed forms for single-channel cases and (ii) the exact
distribution of the discrete chain P_{n+1} = M_n P_n propagated in FP64
(chi-squared).  Charge is conserved exactly (ions + free electrons).
The Debye length (Eq. 3) is pinned to the NRL Plasma Formulary.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from paper_2401_03180_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# pulse fluence per step
# --------------------------------------------------------------------------
def test_gaussian_pulse_integral_and_shape(oracle_mod):
    p = W.Pulse(8.0, 10.0, 1e12, 0.0)
    dt_fs = 0.05
    n = 2000                         # [-50, 50] fs = +-5 FWHM
    dF = oracle_mod.pulse_table([p], -50.0, dt_fs, n)
    total = 1e12 * 1e-6              # photons/nm^2
    assert math.isclose(dF.sum(), total, rel_tol=1e-12)
    assert np.all(dF >= 0)
    np.testing.assert_allclose(dF, dF[::-1], rtol=1e-9, atol=1e-12 * dF.max())
    # the window +-1 FWHM holds erf(2 sqrt(ln 2)) = 98.1% of the fluence
    win = oracle_mod.pulse_table([p], -10.0, dt_fs, 400).sum()
    assert math.isclose(win / total, math.erf(2 * math.sqrt(math.log(2))), rel_tol=1e-12)
    # half maximum at +-FWHM/2 (flux sampled at step midpoints)
    t_mid = -50.0 + (np.arange(n) + 0.5) * dt_fs
    flux = np.interp([-5.0, 0.0, 5.0], t_mid, dF)
    assert math.isclose(flux[0] / flux[1], 0.5, rel_tol=2e-4)
    assert math.isclose(flux[2] / flux[1], 0.5, rel_tol=2e-4)


def test_flat_top_and_two_pulses(oracle_mod):
    p = W.Pulse(8.0, 15.0, 2e12, 0.0, shape=W.FLAT_TOP)
    dF = oracle_mod.pulse_table([p], -10.0, 0.05, 400)
    inside = (np.arange(400) * 0.05 - 10.0 >= -7.5) & (np.arange(1, 401) * 0.05 - 10.0 <= 7.5)
    np.testing.assert_allclose(dF[inside], 2e6 * 0.05 / 15.0, rtol=1e-12)
    assert math.isclose(dF.sum(), 2e6, rel_tol=1e-12)
    a = W.Pulse(9.0, 10.0, 1e13, 0.0)
    b = W.Pulse(9.0, 10.0, 1e13, 50.0)
    both = oracle_mod.pulse_table([a, b], -40.0, 0.05, 3000)
    sep = oracle_mod.pulse_table([a], -40.0, 0.05, 3000) + oracle_mod.pulse_table([b], -40.0, 0.05, 3000)
    np.testing.assert_allclose(both, sep, rtol=1e-15, atol=0)


# --------------------------------------------------------------------------
# Debye length (Eq. 3)
# --------------------------------------------------------------------------
def test_debye_length_nrl(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "nrl_debye_length.txt"))
            if l.strip() and not l.startswith("#")]
    for ne_cm3, te_ev in ((float(a), float(b)) for a, b in rows):
        lam_nrl_nm = 7.43e2 * math.sqrt(te_ev / ne_cm3) * 1e7
        ne_nm3 = ne_cm3 * 1e-21
        s = oracle_mod.plasma_scalars(0, 0, 1.0, dt_ps=5e-5, te_floor_ev=0.0, dte_ev=4.0,
                                      n_te=1024, prescribed=(ne_nm3, te_ev))
        assert math.isclose(1.0 / s["kappa"], lam_nrl_nm, rel_tol=5e-3)
    # bookkeeping: T_e = (2/3) E/N_e, n_e = N_e/V
    s = oracle_mod.plasma_scalars(300, 300 * 150_000, 30.0, dt_ps=5e-5, te_floor_ev=1.0,
                                  dte_ev=4.0, n_te=1024)
    assert math.isclose(s["te_ev"], 100.0, rel_tol=1e-15)
    assert math.isclose(s["n_e"], 10.0, rel_tol=1e-15)
    assert s["it0"] == 25 and s["wt"] == 0.0
    s0 = oracle_mod.plasma_scalars(0, 0, 30.0, dt_ps=5e-5, te_floor_ev=1.0, dte_ev=4.0, n_te=1024)
    assert s0["kappa"] == 0.0 and s0["ne_dt"] == 0.0


# --------------------------------------------------------------------------
# single-species harnesses
# --------------------------------------------------------------------------
def _atoms(n, species, seed=11):
    return W.Sample(x=np.zeros((n, 3)), v=np.zeros((n, 3)),
                    species=np.full(n, species, np.uint8), fragment=np.arange(n, dtype=np.int32),
                    q0=np.zeros(n, np.uint8), replica_offset=np.array([0, n], np.int32),
                    seed=np.array([seed], np.uint64), box=np.zeros((1, 3)), volume=np.array([1.0]))


class _CRHarness:
    """Runs only the CR update of the oracle (no forces) with prescribed
    n_e, T_e and fluence per step."""

    def __init__(self, oracle_mod, sample, atomic, dF, ne, te, dt_ps=5e-5):
        self.o = oracle_mod
        steps = len(dF)
        self.md = oracle_mod.OracleMD.__new__(oracle_mod.OracleMD)
        md = self.md
        md.s, md.a, md.dt, md.te_floor, md.f = sample, atomic, dt_ps, 1.0, oracle_mod.COULOMB_F
        md.n, md.R = sample.n_atoms, 1
        md.z = np.ascontiguousarray(atomic.z, np.int32)
        md.sp = sample.species.copy(); md.q = sample.q0.copy(); md.h = np.zeros(md.n, np.uint8)
        md.rep_off = sample.replica_offset; md.rep_of = np.zeros(md.n, np.int32)
        md.local = np.arange(md.n, dtype=np.int32); md.seed = sample.seed
        md.vol = sample.volume
        md.etab, md.inv = oracle_mod.exp_tables()
        tau = atomic.tau_auger_ps
        md.auger_dt = np.where(tau > 0, dt_ps / np.where(tau > 0, tau, 1.0), 0.0)
        md.dF = np.asarray(dF, np.float64).reshape(1, -1)
        md.prescribed = (np.asarray(ne).reshape(1, -1), np.asarray(te).reshape(1, -1))
        md.n_e = np.array([0], np.int64); md.e_gas = np.array([0], np.int64)

    def step(self, n):
        md = self.md
        md.scal = [md._scalars(0, n)]
        return md.cr_step(n)


def _zero_rates(atom, keep=()):
    if "pi" not in keep:
        atom.sigma_pi[:] = 0
    if "auger" not in keep:
        atom.tau_auger_ps[:] = 0
    if "ci" not in keep:
        atom.k_ci[:] = 0
    if "rec" not in keep:
        atom.k_rec[:] = 0
    return atom


def _binom_ok(k, n, p, alpha=1e-5):
    lo = stats.binom.cdf(k, n, p)
    hi = stats.binom.sf(k - 1, n, p)
    return min(lo, hi) > alpha / 2


def test_photoionisation_only_survival(oracle_mod):
    n = 200_000
    s = _atoms(n, W.H)
    atom = _zero_rates(W.atomic_data(8.0), keep=("pi",))
    sig = atom.sigma_pi[atom.ts_offset[W.H], 0]
    dF = oracle_mod.pulse_table([W.Pulse(8.0, 10.0, 3e13 * 9.2e-9 / sig / 1e6 * 1e6, 0.0)],
                                -10.0, 0.05, 400)
    dF = dF / dF.sum() * (0.7 / sig)        # sigma * F = 0.7 in total
    h = _CRHarness(oracle_mod, s, atom, dF, np.zeros(401), np.zeros(401))
    for k in range(len(dF)):
        h.step(k)
        if k in (50, 199, 399):
            surv = np.exp(-sig * dF[:k + 1].sum())
            assert _binom_ok(int((h.md.q == 0).sum()), n, surv)
    assert set(np.unique(h.md.q)) <= {0, 1} and np.all(h.md.h == 0)


def test_auger_only_decay(oracle_mod):
    n = 200_000
    s = _atoms(n, W.C)
    s.q0[:] = 1
    atom = _zero_rates(W.atomic_data(8.0), keep=("auger",))
    tau = atom.tau_auger_ps[W.C]
    steps = 300
    h = _CRHarness(oracle_mod, s, atom, np.zeros(steps), np.zeros(steps + 1), np.zeros(steps + 1))
    h.md.h[:] = 1
    p_keep = math.exp(-5e-5 / tau)
    for k in range(steps):
        h.step(k)
        if k in (10, 100, 299):
            assert _binom_ok(int((h.md.h == 1).sum()), n, p_keep ** (k + 1))
    # an Auger event raises the charge by one and clears the hole
    assert np.all((h.md.q == 1) == (h.md.h == 1))
    assert np.all((h.md.q == 2) == (h.md.h == 0))


def _exact_chain(atom, z_s, off, dF, ne, te, steps, dt, sp_auger_dt, start):
    """Exact distribution over (q, h) of the discrete chain, FP64."""
    nstate = 2 * (z_s + 1)
    P = np.zeros(nstate); P[start] = 1.0
    out = []
    for n in range(steps):
        x = min(max(te[n] / atom.dte_ev, 0.0), atom.n_te - 1)
        i0 = min(int(x), atom.n_te - 2); w = x - i0
        M = np.zeros((nstate, nstate))
        for q in range(z_s + 1):
            for hh in (0, 1):
                st = 2 * q + hh
                ts = off + q
                if q == z_s and hh == 1:     # unreachable: a bare nucleus has no K hole
                    M[st, st] = 1.0
                    continue
                a = [atom.sigma_pi[ts, hh] * dF[n], sp_auger_dt if hh else 0.0,
                     ne[n] * dt * (atom.k_ci[ts, i0] + w * (atom.k_ci[ts, i0 + 1] - atom.k_ci[ts, i0])) if q < z_s else 0.0,
                     ne[n] * dt * (atom.k_rec[ts, i0] + w * (atom.k_rec[ts, i0 + 1] - atom.k_rec[ts, i0])) if (q > 0 and hh == 0) else 0.0]
                lam = sum(a)
                p = -math.expm1(-lam)
                M[st, st] += 1 - p
                if lam == 0:
                    continue
                # PI
                if a[0] > 0:
                    qn = q + 1
                    hn = 0 if qn == z_s else (1 if (z_s >= 3 and hh == 0 and z_s - qn >= 2) else hh)
                    M[st, 2 * qn + hn] += p * a[0] / lam
                if a[1] > 0:
                    M[st, 2 * (q + 1)] += p * a[1] / lam
                if a[2] > 0:
                    qn = q + 1
                    hn = 0 if qn == z_s else hh
                    M[st, 2 * qn + hn] += p * a[2] / lam
                if a[3] > 0:
                    M[st, 2 * (q - 1) + hh] += p * a[3] / lam
        P = P @ M
        out.append(P.copy())
    return out


@pytest.mark.parametrize("species", [W.C, W.O])
def test_master_equation_chi2(oracle_mod, species):
    n = 100_000
    s = _atoms(n, species, seed=31 + species)
    atom = W.atomic_data(8.0, pi_scale=4000.0, ci_scale=30.0, rec_scale=3000.0)
    z_s = int(W.Z[species]); off = int(atom.ts_offset[species])
    steps = 300
    dF = oracle_mod.pulse_table([W.Pulse(8.0, 10.0, 1e12, 0.0)], -7.5, 0.05, steps)
    ne = np.linspace(0.0, 40.0, steps + 1)
    te = np.concatenate([np.linspace(300.0, 6.0, steps // 2), np.full(steps + 1 - steps // 2, 6.0)])
    h = _CRHarness(oracle_mod, s, atom, dF, ne, te)
    tau = atom.tau_auger_ps[species]
    exact = _exact_chain(atom, z_s, off, dF, ne, te, steps, 5e-5, 5e-5 / tau, 0)
    checkpoints = set(np.linspace(29, steps - 1, 10).astype(int).tolist())
    counts_total = np.zeros(4, np.int64)
    for k in range(steps):
        _, _, cnt = h.step(k)
        counts_total += cnt[0]
        if k in checkpoints:
            obs = np.bincount(2 * h.md.q.astype(int) + h.md.h, minlength=2 * (z_s + 1))
            exp_ = exact[k] * n
            keep = exp_ > 5
            chi2 = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
            chi2 += (obs[~keep].sum() - exp_[~keep].sum()) ** 2 / max(exp_[~keep].sum(), 5)
            dof = int(keep.sum())
            assert stats.chi2.sf(chi2, dof) > 1e-3, (k, chi2, dof)
    assert np.all(counts_total > 100), counts_total    # every channel fired


def test_charge_conservation_full_step(oracle_mod):
    wl = W.workload("c1_methane_1500", scale=0.1)
    atom = W.atomic_data(8.0, pi_scale=3000.0)
    md = oracle_mod.OracleMD(wl.sample, atom, dF_table=np.full((1, 60), 1e3))
    seen = np.zeros(4, np.int64)
    for _ in range(60):
        before = md.n_e.copy()
        c_before = md.counts.copy()
        md.step()
        assert md.n_e[0] == int(md.q.astype(np.int64).sum())
        d = md.counts - c_before
        assert md.n_e[0] - before[0] == d[0, :3].sum() - d[0, 3]
        assert md.e_gas[0] >= 0
        assert np.all(md.q <= W.Z[md.sp]) and np.all(md.h <= 1)
        assert np.all(md.h[md.q == W.Z[md.sp]] == 0)
        seen += d[0]
    assert seen[0] > 0 and seen[1] > 0


def test_cr_is_counter_based(oracle_mod):
    """Same (seed, atom, step) -> same decisions, whatever else runs."""
    n = 5000
    atom = W.atomic_data(8.0, pi_scale=2000.0)
    dF = np.full(20, 1e6)
    a = _CRHarness(oracle_mod, _atoms(n, W.O, seed=5), atom, dF, np.full(21, 3.0), np.full(21, 50.0))
    b = _CRHarness(oracle_mod, _atoms(n, W.O, seed=5), atom, dF, np.full(21, 3.0), np.full(21, 50.0))
    for k in range(20):
        a.step(k)
    for k in range(20):
        b.step(k)
    np.testing.assert_array_equal(a.md.q, b.md.q)
    c = _CRHarness(oracle_mod, _atoms(n, W.O, seed=6), atom, dF, np.full(21, 3.0), np.full(21, 50.0))
    for k in range(20):
        c.step(k)
    assert not np.array_equal(a.md.q, c.md.q)


@pytest.mark.parametrize("mode", ["rates", "table"])
def test_charges_only_equals_the_full_step(oracle_mod, mode):
    """OracleMD(with_forces=False) skips the all-pairs forces: charges, K holes
    and the electron gas never read positions (Sec. II.A, homogeneous gas of
    fixed volume), so its charge sequence must be the full step's, bit for bit,
    on a batch of replicas with their own pulses and seeds, while the full run
    moves (and Coulomb-explodes) the atoms."""
    reps = [W.methane_cluster(n, seed=70 + k) for k, n in enumerate((30, 55, 12, 41, 23, 66))]
    for k, r in enumerate(reps):
        r.seed[:] = 3000 + 17 * k
    s = W.concat(reps)
    atom = W.atomic_data(8.0, pi_scale=2000.0, ci_scale=20.0, rec_scale=500.0)
    pulses = [[W.Pulse(8.0, 10.0, f, 0.0)] for f in (1e12, 3e11, 2e12, 5e11, 1.5e12, 8e11)]
    kw = dict(r_cut=1.2, t_start_fs=-4.0, pulses=pulses, n_steps_max=120)
    if mode == "table":
        kw["charge_table"] = np.stack([W.charge_fraction_table(p, -4.0, 0.05, 121, mean_final=1.0 + 0.4 * k)
                                       for k, p in enumerate(pulses)])
    full = oracle_mod.OracleMD(s, atom, **kw)
    fast = oracle_mod.OracleMD(s, atom, with_forces=False, **kw)
    x0 = full.x.copy()
    for n in range(100):
        full.step()
        fast.step()
        assert np.array_equal(fast.q, full.q) and np.array_equal(fast.h, full.h), n
        assert np.array_equal(fast.n_e, full.n_e) and np.array_equal(fast.e_gas, full.e_gas), n
        assert np.array_equal(fast.counts, full.counts), n
        assert [sc["kappa"] for sc in fast.scal] == [sc["kappa"] for sc in full.scal], n
    assert fast.q.any() and np.abs(full.x - x0).max() > 1e-3
    assert np.array_equal(fast.x, x0)
