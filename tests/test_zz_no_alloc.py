"""The allocation-free force entry point (md_forces_noalloc), -m gpu.

For callers that cannot allocate device memory (a plug-in inside a program
that owns the device memory budget, a memory-capped process, a loop that
must keep the footprint fixed), the library offers one force evaluation that
uses only a scratch area compiled into it.  Its forces must equal those of
the ordinary handle path (md_init + md_get_state) on the same input, within
the force tolerance of the other parity tests, on two calls in a row (the
second call finds the scratch holding the first call's data).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors, methane, water

pytestmark = pytest.mark.gpu
TOL = 1e-5   # force RMS relative error, as in the parity tests


def _handle_forces(sample, atom, r_cut, kappa):
    g = M.IonisingMD(sample, atom, r_cut=r_cut, cr_enabled=False, kappa_fixed=kappa, max_steps=2)
    f = g.get_state(M.MD_FIELD_F)["f"]
    g.close()
    return f


def _noalloc_forces(sample, r_cut, kappa):
    import torch
    n = sample.n_atoms
    dev = "cuda"
    d_x = torch.from_numpy(np.ascontiguousarray(sample.x, np.float64).reshape(-1)).to(dev)
    d_sp = torch.from_numpy(np.ascontiguousarray(sample.species, np.uint8)).to(dev)
    d_q = torch.from_numpy(np.ascontiguousarray(sample.q0, np.uint8)).to(dev)
    d_fr = torch.from_numpy(np.ascontiguousarray(sample.fragment, np.int32)).to(dev)
    d_f = torch.full((3 * n,), float("nan"), dtype=torch.float64, device=dev)
    inp = M.MDForcesInput()
    inp.n_atoms = n
    inp.d_x, inp.d_species, inp.d_q, inp.d_fragment = (d_x.data_ptr(), d_sp.data_ptr(), d_q.data_ptr(),
                                                       d_fr.data_ptr())
    for d in range(3):
        inp.box[d] = float(sample.box[0, d])
    inp.kappa, inp.r_cut, inp.coulomb_f = float(kappa), float(r_cut), M.COULOMB_F
    inp.precision = M.MD_PREC_MIXED
    inp.n_species = len(W.Z)
    for k in range(len(W.Z)):
        inp.z[k] = int(W.Z[k]); inp.lj_sigma0[k] = float(W.LJ_SIGMA0[k]); inp.lj_eps0[k] = float(W.LJ_EPS0[k])
    stream = torch.cuda.current_stream().cuda_stream
    M.md_forces_noalloc(inp, d_f.data_ptr(), stream)
    torch.cuda.synchronize()
    return d_f.cpu().numpy().reshape(n, 3)


def test_noalloc_forces_match_handle_on_two_calls():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    atom = W.atomic_data(8.0)
    s1, rc1 = water(1000)                    # periodic, 3,000 atoms
    s2 = methane(300)                         # vacuum cluster, 1,500 atoms
    for s, rc, kap in ((s1, rc1, 2.5), (s2, 1.2, 1.0)):
        ref = _handle_forces(s, atom, rc, kap)
        got = _noalloc_forces(s, rc, kap)
        assert np.isfinite(got).all()
        rms, mx = force_errors(got, ref)
        assert rms <= TOL, (rms, mx)


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
