"""Adaptive Verlet buffer (md_config.list_skin_adaptive), -m gpu.

With the adaptive buffer the device drops the skin while buffered lists live
fewer than 3 steps and takes it back once a buffered list would last 6 steps
or more.  Whatever the list carries, every pair within r_cut has to be in it:
at every step the forces must match the FP64 oracle's all-pair forces at the
GPU's own positions, and the number of pairs the force kernel finds within
r_cut the oracle's count (up to pairs within 1e-5 nm of the cutoff).

The system makes both switches happen in 100 steps: two C6+ ions fly at each
other at 22 nm/ps (1.1 nm apart, 0.5 fs steps, skin 0.04 nm: a buffered list
lasts 2 steps), slow down to a turning point under their Coulomb repulsion
(the skin comes back) and fly apart again (it goes again).  Next to them sit a
cold neutral methane cluster, whose many pairs near r_cut a list of the wrong
radius or on the wrong cells would miss, and atoms on a sparse lattice that
feel no force.
"""
import re

import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors, near_cutoff_pairs

pytestmark = pytest.mark.gpu
DT = 5e-4
RC = 1.2
SKIN = 0.04
TOL_F = {"mixed": 1e-5, "fp64": 1e-12}
TOL_X = {"mixed": 1e-5, "fp64": 1e-9}
# Forces are summed in 64-bit fixed point of grain 2^-32 kJ/mol/nm, one
# rounding per partial sum: the FP64 path's absolute floor, which bounds the
# error of the neutral cluster's small LJ forces before 1e-12 of their size does.
FIX_FLOOR = 64 * 2.0 ** -32
XQF = M.MD_FIELD_X | M.MD_FIELD_Q | M.MD_FIELD_F


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def collision_sample():
    g = np.arange(4) * 1.5                       # 64 atoms 1.5 nm apart: no pair within r_cut
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ions = np.array([[10.0, 10.0, 10.0], [11.1, 10.0, 10.0]])
    m = W.methane_cluster(60, seed=5)             # 300 atoms, at rest
    xm = m.x - m.x.min(0) + np.array([0.0, 8.0, 0.0])
    x = np.concatenate([lat, ions, xm])
    v = np.zeros_like(x)
    v[64, 0], v[65, 0] = 22.0, -22.0
    sp = np.concatenate([np.full(66, 1, np.uint8), m.species])
    q0 = np.zeros(len(x), np.uint8)
    q0[64:66] = 6
    frag = np.concatenate([np.arange(66, dtype=np.int32), m.fragment + 66])
    n = len(x)
    return W.Sample(x=x, v=v, species=sp, fragment=frag, q0=q0, replica_offset=np.array([0, n], np.int32),
                    seed=np.array([1], np.uint64), box=np.zeros((1, 3)), volume=np.array([1000.0]))


def _gpu_run(s, prec, adaptive, max_steps=120):
    return M.IonisingMD(s, W.atomic_data(8.0), precision=prec, dt_ps=DT, r_cut=RC, cr_enabled=False,
                        kappa_fixed=0.0, max_steps=max_steps, list_skin_nm=SKIN, list_skin_adaptive=adaptive)


def _check_pairs_and_forces(gpu, ora, prec, where):
    st = gpu.get_state(XQF)
    F, _, n_ref = ora.forces(x=st["x"], q=st["q"], kappa=np.zeros(1))
    _, _, n = gpu.energies()
    slack = near_cutoff_pairs(st["x"], None, RC, 1e-5)
    assert abs(n - n_ref) <= slack, (where, n, n_ref, slack)
    for sel in (slice(64, 66), slice(66, None)):    # the ions; the methane cluster
        if not np.any(F[sel]):                       # the ions once they are r_cut apart
            assert np.all(st["f"][sel] == 0.0), (where, sel)
            continue
        rms, mx = force_errors(st["f"][sel], F[sel])
        dmax = float(np.abs(st["f"][sel] - F[sel]).max())
        assert rms <= TOL_F[prec] or (prec == "fp64" and dmax <= FIX_FLOOR), (where, sel, rms, mx, dmax)
    assert np.all(st["f"][:64] == 0.0), where
    return st


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_adaptive_skin_switches_both_ways_and_keeps_every_pair(oracle_mod, prec):
    s = collision_sample()
    gpu = _gpu_run(s, prec, True)
    ora = oracle_mod.OracleMD(s, W.atomic_data(8.0), dt_ps=DT, r_cut=RC, cr_enabled=False, kappa_fixed=0.0)
    pattern = []
    b0 = u0 = 0
    for k in range(100):
        gpu.step(1)
        ora.step()
        t = gpu.timing()
        built, unbuf = t.list_builds - b0, t.list_unbuffered_builds - u0
        b0, u0 = t.list_builds, t.list_unbuffered_builds
        assert unbuf <= built <= 1
        pattern.append("U" if unbuf else ("B" if built else "."))
        st = _check_pairs_and_forces(gpu, ora, prec, k)
    pattern = "".join(pattern)
    # unbuffered while the ions close in, buffered through the turning point,
    # unbuffered again as they fly apart
    assert re.search(r"U+[B.]*\.[B.]*U", pattern), pattern
    d = st["x"] - ora.x
    assert float(np.sqrt((d ** 2).sum(1).mean())) <= TOL_X[prec]
    gpu.reset_timing()
    assert gpu.timing().list_unbuffered_builds == 0
    gpu.close()


def test_fixed_skin_reports_no_unbuffered_builds():
    s = collision_sample()
    g = _gpu_run(s, "mixed", False)
    g.step(40)
    t = g.timing()
    assert t.list_unbuffered_builds == 0 and 1 <= t.list_builds <= 40
    g.close()


def test_adaptive_skin_checkpoint_resumes_with_every_pair(oracle_mod):
    """A checkpoint taken while the lists are unbuffered: the restored handle
    starts again from a buffered list (md_set_state), switches as it needs to,
    finds every pair, and follows the straight run to rounding."""
    s = collision_sample()
    g = _gpu_run(s, "mixed", True)
    g.step(20)
    assert g.timing().list_unbuffered_builds > 0
    ck = g.get_state(M.MD_FIELD_ALL)
    g.step(40)
    straight = g.get_state(XQF)
    g.close()
    h = _gpu_run(s, "mixed", True)
    h.set_state(M.MD_FIELD_ALL, **{k: ck[k] for k in ("x", "v", "q", "h", "n_e", "e_gas_mev", "event_counts",
                                                      "x_list")}, step=ck["step"])
    ora = oracle_mod.OracleMD(s, W.atomic_data(8.0), dt_ps=DT, r_cut=RC, cr_enabled=False, kappa_fixed=0.0)
    for k in range(40):
        h.step(1)
        _check_pairs_and_forces(h, ora, "mixed", k)
    resumed = h.get_state(XQF)
    h.close()
    d = resumed["x"] - straight["x"]
    assert float(np.sqrt((d ** 2).sum(1).mean())) <= TOL_X["mixed"]


def test_adaptive_flag_is_validated():
    s = collision_sample()
    with pytest.raises(M.MDError) as e:
        _gpu_run(s, "mixed", 2)
    assert e.value.status == M.MD_ERR_INVALID_ARG


def _check_replicas(gpu, ora, rc, parts, where):
    """Pair count and forces of a batch against the oracle: parts lists each
    replica's (slice, periodic box or None)."""
    st = gpu.get_state(XQF)
    F, _, n_ref = ora.forces(x=st["x"], q=st["q"], kappa=np.zeros(len(parts)))
    _, _, n = gpu.energies()
    slack = sum(near_cutoff_pairs(st["x"][sl], box, rc, 1e-5) for sl, box in parts)
    assert abs(n - n_ref) <= slack, (where, n, n_ref, slack)
    for sl, _ in parts:
        if not np.any(F[sl]):
            assert np.all(st["f"][sl] == 0.0), (where, sl)
            continue
        rms, mx = force_errors(st["f"][sl], F[sl])
        assert rms <= TOL_F["mixed"], (where, sl, rms, mx)
    return st


def test_adaptive_skin_in_a_batch_with_a_periodic_replica(oracle_mod):
    """One decision serves every replica of a handle: next to the colliding
    ions (vacuum) a neutral periodic water box gets unbuffered lists too, whose
    cells stay sized for r_cut + skin while the list radius is r_cut.  Both
    replicas keep every pair at every step."""
    from gpu_common import water
    w, _ = water(1000)                      # 3.11 nm box, 3,000 atoms
    w.q0[:] = 0
    b = W.concat([collision_sample(), w])
    rc = 0.9                                # box >= 3 (r_cut + skin)
    gpu = M.IonisingMD(b, W.atomic_data(8.0), dt_ps=DT, r_cut=rc, cr_enabled=False, kappa_fixed=0.0,
                       max_steps=120, list_skin_nm=SKIN, list_skin_adaptive=True)
    ora = oracle_mod.OracleMD(b, W.atomic_data(8.0), dt_ps=DT, r_cut=rc, cr_enabled=False, kappa_fixed=0.0)
    off = b.replica_offset
    parts = [(slice(0, off[1]), None), (slice(off[1], off[2]), b.box[1])]
    pattern = []
    b0 = u0 = 0
    for k in range(100):
        gpu.step(1)
        ora.step()
        t = gpu.timing()
        built, unbuf = t.list_builds - b0, t.list_unbuffered_builds - u0
        b0, u0 = t.list_builds, t.list_unbuffered_builds
        pattern.append("U" if unbuf else ("B" if built else "."))
        st = _check_replicas(gpu, ora, rc, parts, k)
    pattern = "".join(pattern)
    assert re.search(r"U+[B.]*\.[B.]*U", pattern), pattern
    d = st["x"] - ora.x
    L = b.box[1]
    d[off[1]:] -= L * np.round(d[off[1]:] / L)
    assert float(np.sqrt((d ** 2).sum(1).mean())) <= TOL_X["mixed"]
    gpu.close()


def test_adaptive_skin_on_a_hot_periodic_box(oracle_mod):
    """A periodic water box in which 5 % of the atoms fly at 40 nm/ps: with a
    0.01 nm skin the buffered lists live 3 steps, then one lives 2 and the
    lists turn unbuffered for good; every pair is found at every step."""
    from gpu_common import water
    s, _ = water(1000)
    rng = np.random.default_rng(3)
    d = rng.normal(size=s.v.shape)
    d /= np.linalg.norm(d, axis=1)[:, None]
    hot = rng.random(s.n_atoms) < 0.05
    s.v[hot] = 40.0 * d[hot]
    rc = 0.9
    gpu = M.IonisingMD(s, W.atomic_data(6.0), r_cut=rc, cr_enabled=False, kappa_fixed=2.0, max_steps=60,
                       list_skin_nm=0.01, list_skin_adaptive=True)
    ora = oracle_mod.OracleMD(s, W.atomic_data(6.0), r_cut=rc, cr_enabled=False, kappa_fixed=2.0)
    parts = [(slice(0, s.n_atoms), s.box[0])]
    for k in range(40):
        gpu.step(1)
        ora.step()
        st = gpu.get_state(XQF)
        F, _, n_ref = ora.forces(x=st["x"], q=st["q"], kappa=np.full(1, 2.0))
        _, _, n = gpu.energies()
        slack = near_cutoff_pairs(st["x"], s.box[0], rc, 1e-5)
        assert abs(n - n_ref) <= slack, (k, n, n_ref, slack)
        rms, mx = force_errors(st["f"], F)
        assert rms <= TOL_F["mixed"], (k, rms, mx)
    t = gpu.timing()
    gpu.close()
    assert t.list_unbuffered_builds >= 20, (t.list_builds, t.list_unbuffered_builds)
