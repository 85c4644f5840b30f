"""The allocation-free force entry point (md_forces_noalloc), -m gpu.

For callers that cannot allocate device memory (a plug-in inside a program
that owns the device memory budget, a memory-capped process, a loop that
must keep the footprint fixed), the library offers one force evaluation that
uses only a scratch area compiled into it.  Its forces must equal those of
the ordinary handle path (md_init + md_get_state) on the same input, within
the force tolerance of the other parity tests, on two calls in a row (the
second call finds the scratch holding the first call's data), and those of
the FP64 oracle, also for a sparse vacuum sample wider than the fixed cell
capacity.  A call must leave the device's free memory unchanged, and bad
device-side input (a species index or a charge out of range) comes back as a
status.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors, methane, water

pytestmark = pytest.mark.gpu
TOL = {"mixed": 1e-5, "fp64": 1e-12}   # force RMS relative error, as in the parity tests
PREC = {"mixed": M.MD_PREC_MIXED, "fp64": M.MD_PREC_FP64}


def _handle_forces(sample, atom, r_cut, kappa, prec):
    g = M.IonisingMD(sample, atom, precision=prec, r_cut=r_cut, cr_enabled=False, kappa_fixed=kappa, max_steps=2)
    f = g.get_state(M.MD_FIELD_F)["f"]
    g.close()
    return f


class _Call:
    """Device inputs and output of one md_forces_noalloc call, allocated by the
    test (the caller) before the call."""

    def __init__(self, sample, r_cut, kappa, prec, species=None, q=None):
        import torch
        n = sample.n_atoms
        dev = "cuda"
        sp = sample.species if species is None else species
        qq = sample.q0 if q is None else q
        self.n = n
        self.t = [torch.from_numpy(np.ascontiguousarray(sample.x, np.float64).reshape(-1)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(sp, np.uint8)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(qq, np.uint8)).to(dev),
                  torch.from_numpy(np.ascontiguousarray(sample.fragment, np.int32)).to(dev)]
        self.d_f = torch.full((3 * n,), float("nan"), dtype=torch.float64, device=dev)
        inp = M.MDForcesInput()
        inp.n_atoms = n
        inp.d_x, inp.d_species, inp.d_q, inp.d_fragment = (t.data_ptr() for t in self.t)
        for d in range(3):
            inp.box[d] = float(sample.box[0, d])
        inp.kappa, inp.r_cut, inp.coulomb_f = float(kappa), float(r_cut), M.COULOMB_F
        inp.precision = PREC[prec]
        inp.n_species = len(W.Z)
        for k in range(len(W.Z)):
            inp.z[k] = int(W.Z[k]); inp.lj_sigma0[k] = float(W.LJ_SIGMA0[k]); inp.lj_eps0[k] = float(W.LJ_EPS0[k])
        self.inp = inp

    def run(self):
        import torch
        M.md_forces_noalloc(self.inp, self.d_f.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()

    def forces(self):
        return self.d_f.cpu().numpy().reshape(self.n, 3)


def _noalloc_forces(sample, r_cut, kappa, prec="mixed"):
    c = _Call(sample, r_cut, kappa, prec)
    c.run()
    return c.forces()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_forces_match_handle_on_two_calls(prec):
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    atom = W.atomic_data(8.0)
    s1, rc1 = water(1000)                    # periodic, 3,000 atoms
    s2 = methane(300)                         # vacuum cluster, 1,500 atoms
    for s, rc, kap in ((s1, rc1, 2.5), (s2, 1.2, 1.0)):
        ref = _handle_forces(s, atom, rc, kap, prec)
        got = _noalloc_forces(s, rc, kap, prec)
        assert np.isfinite(got).all()
        rms, mx = force_errors(got, ref)
        assert rms <= TOL[prec], (prec, rms, mx)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_forces_match_oracle(oracle_mod, prec):
    """Against the FP64 all-pairs oracle (Sec. II.A Eq. 2, Sec. II.B Eq. 8),
    not only against the handle path."""
    atom = W.atomic_data(8.0)
    s = methane(300)
    kap = 1.7
    ref = oracle_mod.OracleMD(s, atom, r_cut=1.2, cr_enabled=False, kappa_fixed=kap).F
    got = _noalloc_forces(s, 1.2, kap, prec)
    rms, mx = force_errors(got, ref)
    assert rms <= TOL[prec], (prec, rms, mx)


def test_noalloc_leaves_device_memory_unchanged():
    import torch
    s1, rc1 = water(1000)
    s2 = methane(200)
    calls = [_Call(s1, rc1, 2.0, "mixed"), _Call(s2, 1.2, 0.5, "mixed"), _Call(s1, rc1, 3.0, "mixed")]
    calls[0].run()                              # warm-up: module and kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    calls[1].run()
    calls[2].run()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    assert np.isfinite(calls[1].forces()).all() and np.isfinite(calls[2].forces()).all()


@pytest.mark.parametrize("what", ["species", "charge"])
def test_noalloc_rejects_bad_device_input(what):
    s = methane(100)
    sp = s.species.copy()
    q = s.q0.copy()
    if what == "species":
        sp[17] = len(W.Z)                       # one index past the species table
    else:
        h = int(np.flatnonzero(s.species == W.H)[3])
        q[h] = 2                                 # hydrogen has Z = 1
    c = _Call(s, 1.2, 1.0, "mixed", species=sp, q=q)
    with pytest.raises(M.MDError) as e:
        c.run()
    assert e.value.status == M.MD_ERR_INVALID_ARG
    assert "n_species" in M.md_last_error()
    # the next call with good input works on the same scratch
    ref = _noalloc_forces(s, 1.2, 1.0)
    assert np.isfinite(ref).all()


def test_noalloc_sparse_vacuum_sample_beyond_the_cell_cap(oracle_mod):
    """A vacuum sample spread over far more than MD_NOALLOC_MAX_CELLS cells of
    edge r_cut (24 methane clusters 13 nm apart: 21^3 cells of 1.2 nm): the
    vacuum grid takes larger cells instead, so the cell count stays within the
    fixed scratch, and the forces still match the FP64 oracle."""
    parts = []
    k = 0
    for ix in range(3):
        for iy in range(3):
            for iz in range(3):
                if k == 24:
                    break
                c = W.methane_cluster(20, seed=300 + k)           # 100 atoms
                c.x = c.x - c.x.mean(0) + 13.0 * np.array([ix, iy, iz])
                parts.append(c)
                k += 1
    b = W.concat(parts)
    n = b.n_atoms
    q = b.q0.copy()
    q[np.random.default_rng(9).random(n) < 0.2] = 1
    s = W.Sample(x=b.x, v=b.v, species=b.species, fragment=b.fragment, q0=q,
                 replica_offset=np.array([0, n], np.int32), seed=b.seed[:1], box=np.zeros((1, 3)),
                 volume=np.array([float(b.volume.sum())]))
    span = s.x.max(0) - s.x.min(0)
    assert np.prod(np.floor(span / 1.2)) > M.MD_NOALLOC_MAX_CELLS
    ref = oracle_mod.OracleMD(s, W.atomic_data(8.0), r_cut=1.2, cr_enabled=False, kappa_fixed=1.0).F
    for prec in ("mixed", "fp64"):
        got = _noalloc_forces(s, 1.2, 1.0, prec)
        rms, mx = force_errors(got, ref)
        assert rms <= TOL[prec], (prec, rms, mx)


def test_noalloc_rejects_oversized_input():
    import torch
    inp = M.MDForcesInput()
    inp.n_atoms = M.MD_NOALLOC_MAX_ATOMS + 1
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    inp.d_x = inp.d_species = inp.d_q = inp.d_fragment = d.data_ptr()
    inp.r_cut, inp.coulomb_f, inp.n_species = 1.2, M.COULOMB_F, 1
    inp.z[0] = 1
    with pytest.raises(M.MDError) as e:
        M.md_forces_noalloc(inp, d.data_ptr(), 0)
    assert e.value.status == M.MD_ERR_INVALID_ARG
    assert str(M.MD_NOALLOC_MAX_ATOMS) in M.md_last_error()
