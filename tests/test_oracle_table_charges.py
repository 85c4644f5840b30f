"""Pins of the oracle's table-driven charges (Sec. II.A: integer charges
assigned stochastically so that, averaged, they match the CR charge-state
fractions; read as quantile coupling): the populations match the table
(chi-squared), a one-state table puts every atom in that state, monotone
fractions give monotone charges, and N_e = sum q is conserved."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

Z = np.array([1, 6, 7, 8, 16])
OFF = np.concatenate([[0], np.cumsum(Z + 1)]).astype(np.int32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _row(mean_c):
    """A table row: truncated Poisson fractions of mean ~ mean_c * Z_s / 6 per species."""
    row = np.zeros(OFF[-1])
    for s, z in enumerate(Z):
        lam = mean_c * z / 6.0
        f = stats.poisson.pmf(np.arange(z + 1), lam) if lam > 0 else np.eye(z + 1)[0]
        f[-1] += 1.0 - f.sum()
        row[OFF[s]:OFF[s + 1]] = f
    return row


def test_quantiles_uniform():
    u = O.charge_quantiles(77, np.arange(200_000))
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert np.array_equal(u, O.charge_quantiles(77, np.arange(200_000)))      # fixed per atom


def test_populations_match_the_fractions():
    n = 100_000
    sp = np.full(n, 1, np.uint8)                                              # carbon
    u = O.charge_quantiles(5, np.arange(n))
    for mean_c in (0.3, 1.5, 4.0):
        row = _row(mean_c)
        q = O.table_charges(u, sp, Z, OFF, O.cumulative_fractions(row, OFF))
        f = row[OFF[1]:OFF[2]]
        obs = np.bincount(q, minlength=7).astype(float)
        exp = f * n
        keep = exp > 5
        chi2 = (((obs - exp) ** 2)[keep] / exp[keep]).sum()
        assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3, (mean_c, obs, exp)


def test_one_state_table():
    row = np.zeros(OFF[-1])
    for s, z in enumerate(Z):
        row[OFF[s] + min(3, z)] = 1.0
    sp = np.repeat(np.arange(5), 100).astype(np.uint8)
    q = O.table_charges(O.charge_quantiles(1, np.arange(500)), sp, Z, OFF, O.cumulative_fractions(row, OFF))
    assert np.array_equal(q, np.minimum(3, Z[sp]))


def test_monotone_fractions_give_monotone_charges():
    sp = np.repeat(np.arange(5), 2000).astype(np.uint8)
    u = O.charge_quantiles(9, np.arange(len(sp)))
    prev = None
    for mean_c in np.linspace(0.0, 5.0, 30):
        q = O.table_charges(u, sp, Z, OFF, O.cumulative_fractions(_row(mean_c), OFF))
        if prev is not None:
            assert np.all(q >= prev)
        prev = q


def test_oracle_md_follows_the_table_and_conserves_charge():
    from paper_2401_03180_gb300 import workloads as W
    wl = W.workload("c1_methane_1500", scale=0.2)
    s = wl.sample
    atom = W.atomic_data(8.0)
    rows = np.stack([_row(c) for c in np.linspace(0.0, 2.0, 31)])
    md = O.OracleMD(s, atom, r_cut=1.2, n_steps_max=40, charge_table=rows[None])
    for n in range(30):
        md.step()
        assert md.n_e[0] == int(md.q.astype(np.int64).sum())
        assert not md.h.any()
    u = O.charge_quantiles(int(s.seed[0]), md.local)
    assert np.array_equal(md.q, O.table_charges(u, md.sp, md.z, md.off, O.cumulative_fractions(rows[30], md.off)))
