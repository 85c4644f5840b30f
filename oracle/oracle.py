"""FP64 CPU oracle for the ionising-MD hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this module.  The product
path (the CUDA library and its Python binding) never does, and this module
never imports the product.  The two share only the seeded input generators
(``paper_2401_03180_gb300.workloads``), which hold none of the method's
arithmetic.

What it computes, in the paper's order (arXiv 2401.03180):

* Sec. II.A, Eq. 2: Debye-screened Coulomb between integer ion charges.
* Sec. II.A, Eq. 3: Debye length from the free-electron density and
  temperature, kappa = 1/lambda_D.
* Sec. II.A, Eqs. 4-7 (optional, ``screening="hybrid"``): ion-sphere inside
  the transition radius r' of Eq. 7 and Debye form outside, matched in value
  and first two derivatives (reading; see ``md_oracle.c``), the pair energy
  being the mean of the two ions' views.
* Sec. II.B, Eq. 8: screened LJ, with LJ parameters scaled per charge state
  (Eq. 11) and LJ excluded inside a native fragment.
* Sec. II.B, Eq. 12: Newton's equation, integrated with velocity Verlet.
* Sec. II.A (optional, ``charge_table``): charges assigned from per-step
  charge-state fractions of a CR calculation, drawn at random so that they
  reproduce the fractions on average -- read as quantile coupling: each atom keeps one uniform
  quantile u (Philox stream 2, counter (atom, 0, 2, 0), res53) and takes the
  smallest charge whose cumulative fraction of its species exceeds u.
* Sec. II.B, Eqs. 9-10 (optional, a sample with a ``topology``): Morse bonds
  D_e (1 - e^{-beta (r - b_e)})^2 (reading of the garbled Eq. 10) and
  harmonic angles (k/2)(theta - theta_0)^2 (Sec. III), each scaled by
  c = 1 - zbar/N clamped to [0, 1], zbar the summed charge of its N atoms
  (reading of Eq. 9).
* Sec. II.C, Eq. 17 (analysis): the probe-weighted displacement -- per
  species, the RMS displacement from the initial positions at each step,
  weighted by the probe profile times the fraction of bound electrons
  f = 1 - zbar/Z (reading: zbar the species' mean charge at the step).
* Sec. III (analysis): fractional ion yields -- fragments are the connected
  components of atoms closer than r_frag (reading), counted by mass number
  and net charge.
* Sec. II.C, Eq. 18 (analysis): radial distribution functions g_ab(r) from
  all-pairs distance histograms, and the partial structure factors
  S_ab(q) = 1 + (4 pi rho0 / q) int r (g_ab(r) - 1) sin(q r) dr.
* Sec. II.B, Eqs. 13-14 (optional, ``langevin_g``): electron-ion coupling as
  Langevin friction gamma = n_e g_s and a Gaussian force with
  <f f> = 2 m gamma k_B T_e, integrated as an exact Ornstein-Uhlenbeck
  velocity update after the first half kick (reading), with Gaussians from
  Philox stream 1 keyed by (seed, atom, step) through Box-Muller.
* Sec. II.A (stochastic integer charges, processes named there): the
  reading "RCM-1" -- at most one photo-ionisation, Auger, collisional
  ionisation or recombination event per atom per step, drawn with
  Philox4x32-10 keyed by (seed, atom, step); the free-electron gas is
  homogeneous, thermalised and never escapes, its energy is tracked in
  integer meV.

Parity pins (``tests/test_oracle_*.py``, all ``-m "not gpu"``):

* ``philox``: the cuRAND host generator CURAND_RNG_PSEUDO_PHILOX4_32_10 run
  as a library, block by block.
* ``u53``: extreme values and a uniformity test.
* ``one_minus_exp_neg``: numpy ``expm1`` to a few ulp over 0..40.
* ``lj_table``: textbook LJ facts (zero at sigma, minimum -eps at
  2^(1/6) sigma) and the Eq. 11 scaling limits (q = Z gives no LJ).
* ``pair``: force = -dU/dr by finite differences; the Coulomb energy of two
  elementary charges 1 nm apart (a CODATA-derived golden value); the
  Yukawa ratio e^{-kappa r}; the shift U(r_c) = 0.
* ``forces``: Newton III (net force 0), invariance under translation and
  periodic images, pair counts against a KD-tree.
* ``pulse_table``: total fluence, symmetry, flat-top closed form, FWHM.
* ``plasma_scalars``: the NRL-formulary Debye length.
* ``hybrid_coeffs`` / ``pair_hybrid``: continuity of phi, phi' and phi'' at
  r' (finite differences on both sides); the identity (r' + lambda)^3 =
  R^3 + lambda^3 of Eq. 7; the uniform-electron-gas ion sphere of Eq. 5 as
  lambda -> 0; Coulomb as kappa -> 0; Debye as R -> 0; force = -dU/dr.
* ``cr_step``: closed forms (PI-only survival e^{-sigma F}; Auger-only
  decay), master-equation chi-squared on histograms, exact charge
  conservation.
* ``OracleMD`` (velocity Verlet): NVE energy conservation and second-order
  convergence in dt.
* ``table_charges``: populations match the fractions (chi-squared); a
  one-state table puts every atom in that state; monotone fractions give
  monotone charges (no atom recombines while the distribution ionises);
  charge conservation N_e = sum q.
* ``rdf_counts`` / ``rdf`` / ``structure_factor``: histogram total = pairs
  within r_max (KD-tree); g -> 1 for an ideal gas (one and two species);
  S(q) of a step-function g(r) against its closed form
  1 - 4 pi rho0 (sin q s - q s cos q s) / q^3; S(q) -> 1 for an ideal gas.
* ``morse`` / ``harmonic_angle`` / ``bond_scale`` / ``bonded_forces``: the
  Morse zero at b_e, its dissociation limit D_e and curvature 2 D_e beta^2;
  dV/dr and F = -grad U by finite differences on every coordinate; zero net
  force and torque per molecule; the angle of the tetrahedral and right-angle
  geometries; the scaling limits; minimum image across a periodic boundary;
  the small-amplitude vibration period 2 pi / (beta sqrt(2 D_e / mu)) of a
  diatomic integrated with velocity Verlet.
* ``probe_weights`` / ``probe_sums`` / ``probe_weighted_displacement``:
  weights sum to 1; constant f gives the pulse-table shape; f = 0 steps get
  no weight; a symmetric window about the pulse centre gives a weighted mean
  time equal to the centre; a falling f moves it earlier; a constant
  displacement is returned unchanged; a rigid translation gives its length;
  minimum image across a periodic face.
* ``fragments`` / ``ion_yield_counts``: intact molecules are one fragment
  each (CH4: 16, H2O: 18); an atom pulled beyond r_frag splits off (CH3 +
  H); a molecule across a periodic face stays whole; labels equal those of a
  brute-force all-pairs union-find on small random gases; mass and charge
  are conserved over the fragments.
* ``gaussians`` / ``langevin_update``: normal moments and a KS test; the
  friction-only decay c^n exactly; equipartition <m v^2> -> k_B T_e; the
  Ornstein-Uhlenbeck autocorrelation e^{-gamma t}; charges unaffected.
Trajectory agreement with the GPU beyond short horizons is *parity
unpinned*: MD is chaotic, so only the first steps are compared.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "md_oracle.c")
_lock = threading.Lock()
_lib = None

# Physical constants in the units of the method (nm, ps, amu, kJ/mol, e).
COULOMB_F = 138.935458          # 1/(4 pi eps0), kJ mol^-1 nm e^-2
EV_KJMOL = 96.48533212          # kJ/mol per eV
N_ETAB = 16 * 40                # exp table covers lambda < 40


def build(force: bool = False) -> str:
    """Compile the oracle C file (FP contraction off, OpenMP on)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _declare(L):
    i32, i64, u64, u32, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
    L.orc_philox_many.argtypes = [u64, _P, _P, u32, u32, i64, _P]
    L.orc_philox_blocks.argtypes = [u64, _P, i64, _P]
    L.orc_u53.argtypes = [u32, u32]; L.orc_u53.restype = f64
    L.orc_exp_tables.argtypes = [_P, i32, _P]
    L.orc_one_minus_exp_neg_many.argtypes = [i64, _P, _P, _P, i32, _P]
    L.orc_lj_table.argtypes = [i32, _P, _P, _P, _P, _P]
    L.orc_pair.argtypes = [f64] * 8 + [i32, _P, _P]
    L.orc_forces.argtypes = [i32, _P, _P, _P, _P, i32, _P, _P, _P, _P, f64, f64, i32, _P, _P, _P, _P, _P]
    L.orc_forces_subset.argtypes = [i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, f64, f64, i32, _P, _P, i32, _P, _P]
    L.orc_hybrid_coeffs.argtypes = [f64, f64, f64, _P]
    L.orc_hybrid_phi.argtypes = [f64, _P, f64, f64, _P, _P]
    L.orc_pair_hybrid.argtypes = [f64] * 9 + [i32, _P, _P]
    L.orc_pulse_table.argtypes = [i32, _P, f64, f64, i32, _P]
    L.orc_cr_step.argtypes = ([i32, _P, _P, _P, _P, _P, i64, _P, _P, _P, _P, _P, i32, _P, _P, _P,
                               _P, _P, i32, _P, _P, _P, _P, i32, _P, _P, _P, _P])
    L.orc_cr_step.restype = i32


# ---------------------------------------------------------------------------
# Small building blocks
# ---------------------------------------------------------------------------
def philox(seed: int, c0, c1, c2: int = 0, c3: int = 0) -> np.ndarray:
    """Philox4x32-10 blocks for counters (c0[i], c1[i], c2, c3), key = seed."""
    c0 = np.ascontiguousarray(c0, dtype=np.uint32)
    c1 = np.ascontiguousarray(c1, dtype=np.uint32)
    out = np.empty((len(c0), 4), dtype=np.uint32)
    lib().orc_philox_many(int(seed), _ptr(c0), _ptr(c1), c2, c3, len(c0), _ptr(out))
    return out


def philox_blocks(seed: int, ctr4) -> np.ndarray:
    """Philox4x32-10 for arbitrary counters ctr4[n][4], key = seed."""
    ctr4 = np.ascontiguousarray(ctr4, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr4)
    lib().orc_philox_blocks(int(seed), _ptr(ctr4), len(ctr4), _ptr(out))
    return out


def u53(a: int, b: int) -> float:
    return lib().orc_u53(int(a), int(b))


def exp_tables():
    etab = np.empty(N_ETAB); inv = np.empty(13)
    lib().orc_exp_tables(_ptr(etab), N_ETAB, _ptr(inv))
    return etab, inv


def one_minus_exp_neg(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    etab, inv = exp_tables()
    p = np.empty_like(x)
    lib().orc_one_minus_exp_neg_many(x.size, _ptr(x), _ptr(p), _ptr(etab), N_ETAB, _ptr(inv))
    return p


def lj_table(z, sigma0, eps0):
    z = np.ascontiguousarray(z, dtype=np.int32)
    nts = int((z + 1).sum())
    c6 = np.zeros((nts, nts)); c12 = np.zeros((nts, nts))
    lib().orc_lj_table(len(z), _ptr(z), _ptr(np.ascontiguousarray(sigma0, np.float64)),
                       _ptr(np.ascontiguousarray(eps0, np.float64)), _ptr(c6), _ptr(c12))
    return c6, c12


def pair(r, qi, qj, c6, c12, kappa, rc, lj_on=True, coulomb_f=COULOMB_F):
    """(F(r)/r, U(r) - U(rc)) for one pair (Eqs. 2 and 8)."""
    fr = ctypes.c_double(); u = ctypes.c_double()
    lib().orc_pair(r, qi, qj, c6, c12, kappa, coulomb_f, rc, int(bool(lj_on)),
                   ctypes.byref(fr), ctypes.byref(u))
    return fr.value, u.value


def hybrid_coeffs(Q, ne, kappa):
    """(r', c1, c2, a) of the hybrid potential of an ion of charge Q (Eqs. 4-7);
    a = 3Q/(3 + 3x + x^2) is the Debye amplitude at r' (phi = a e^{-kappa (r - r')}/r)."""
    co = np.zeros(4)
    lib().orc_hybrid_coeffs(float(Q), float(ne), float(kappa), _ptr(co))
    return tuple(float(v) for v in co)


def hybrid_phi(Q, ne, kappa, r):
    """(phi(r), -dphi/dr) of one ion, in e/nm and e/nm^2 (multiply by f)."""
    co = np.ascontiguousarray(hybrid_coeffs(Q, ne, kappa))
    phi = ctypes.c_double(); m = ctypes.c_double()
    lib().orc_hybrid_phi(float(Q), _ptr(co), float(kappa), float(r), ctypes.byref(phi), ctypes.byref(m))
    return phi.value, m.value


def pair_hybrid(r, qi, qj, c6, c12, kappa, ne, rc, lj_on=True, coulomb_f=COULOMB_F):
    """(F(r)/r, U(r) - U(rc)) for one pair with the hybrid electrostatics."""
    fr = ctypes.c_double(); u = ctypes.c_double()
    lib().orc_pair_hybrid(r, qi, qj, c6, c12, kappa, ne, coulomb_f, rc, int(bool(lj_on)),
                          ctypes.byref(fr), ctypes.byref(u))
    return fr.value, u.value


def rdf_counts(x, species, n_species, box, rep_off, r_max, n_bins):
    """Unordered atom pairs per species pair (a <= b, mirrored) and distance
    bin k = floor(r / dr), dr = r_max / n_bins, for r < r_max (minimum image
    in periodic boxes), summed over replicas; all pairs, FP64."""
    x = np.asarray(x, np.float64)
    species = np.asarray(species, np.int64)
    box = np.asarray(box, np.float64).reshape(-1, 3)
    dr = r_max / n_bins
    out = np.zeros((n_species, n_species, n_bins), dtype=np.int64)
    for r in range(len(rep_off) - 1):
        a0, a1 = int(rep_off[r]), int(rep_off[r + 1])
        L = box[r]
        periodic = bool(np.all(L > 0))
        for i in range(a0, a1 - 1):
            d = x[i + 1:a1] - x[i]
            if periodic:
                d -= L * np.round(d / L)
            rr = np.sqrt((d * d).sum(1))
            sel = rr < r_max
            k = np.minimum((rr[sel] / dr).astype(np.int64), n_bins - 1)
            sa = species[i]
            sb = species[i + 1:a1][sel]
            lo, hi = np.minimum(sa, sb), np.maximum(sa, sb)
            np.add.at(out, (lo, hi, k), 1)
    for a in range(n_species):
        for b in range(a):
            out[a, b] = out[b, a]
    return out


def rdf(counts_ab, n_a, n_b, same, volume, r_max):
    """g_ab at the bin centres from a pair histogram: counts over the pairs
    an ideal gas of the same density puts in each spherical shell
    (N_a N_b / V, or N_a (N_a - 1) / (2V) for a = b, times the shell volume)."""
    n_bins = len(counts_ab)
    edges = np.linspace(0.0, r_max, n_bins + 1)
    shell = 4.0 * math.pi / 3.0 * (edges[1:] ** 3 - edges[:-1] ** 3)
    pairs = n_a * (n_a - 1) / 2.0 if same else float(n_a) * n_b
    return 0.5 * (edges[1:] + edges[:-1]), np.asarray(counts_ab, np.float64) / (pairs / volume * shell)


def structure_factor(r, g, rho0, q, dr):
    """S(q) = 1 + (4 pi rho0 / q) int_0^r_max r (g(r) - 1) sin(q r) dr (Eq. 18),
    midpoint rule over the histogram bins."""
    q = np.asarray(q, np.float64)
    integ = (np.asarray(r)[None, :] * (np.asarray(g)[None, :] - 1.0) * np.sin(q[:, None] * np.asarray(r)[None, :])).sum(1) * dr
    return 1.0 + 4.0 * math.pi * rho0 / q * integ


def charge_quantiles(seed: int, ids) -> np.ndarray:
    """Each atom's fixed quantile for the table-driven charges: res53 of the
    first two words of Philox4x32-10 with key = seed, counter = (atom id, 0, 2, 0)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    w = philox(seed, ids, np.zeros(len(ids), np.uint32), 2, 0)
    return ((w[:, 0] >> 5).astype(np.float64) * 67108864.0 + (w[:, 1] >> 6).astype(np.float64)) \
        * 1.1102230246251565e-16


def cumulative_fractions(frac_row, ts_off):
    """Per species, the running sums of the charge-state fractions of one table
    row (FP64, in charge order): cum[ts_off[s] + q] = sum_{q' <= q} f_{s,q'}."""
    frac = np.asarray(frac_row, dtype=np.float64)
    cum = np.empty_like(frac)
    for s in range(len(ts_off) - 1):
        acc = 0.0
        for k in range(ts_off[s], ts_off[s + 1]):
            acc = acc + float(frac[k])
            cum[k] = acc
    return cum


def table_charges(u, species, z, ts_off, cum_row):
    """Charges from one row of cumulative fractions: the smallest q with
    u < cum[ts_off[s] + q]; Z if rounding leaves none."""
    q = np.empty(len(u), dtype=np.uint8)
    for i in range(len(u)):
        s = int(species[i])
        c = cum_row[ts_off[s]:ts_off[s + 1]]
        k = int(np.searchsorted(c, u[i], side="right"))   # first c > u
        q[i] = min(k, int(z[s]))
    return q


def gaussians(seed: int, ids, step: int) -> np.ndarray:
    """Three standard normal numbers per atom for the Langevin force of one
    step (Sec. II.B, Eq. 14): Philox4x32-10 with key = seed and counter =
    (atom id, step, 1, 0) (stream 1; the charge update uses stream 0) gives
    four words w0..w3; Box-Muller on u = (w + 1/2) 2^-32 turns (w0, w1) and
    (w2, w3) into two pairs, of which the first three numbers are used:
    sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    w = philox(seed, ids, np.full(len(ids), step, np.uint32), 1, 0).astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    ra = np.sqrt(-2.0 * np.log(u[:, 0]))
    rb = np.sqrt(-2.0 * np.log(u[:, 2]))
    return np.stack([ra * np.cos(2.0 * np.pi * u[:, 1]), ra * np.sin(2.0 * np.pi * u[:, 1]),
                     rb * np.cos(2.0 * np.pi * u[:, 3])], axis=1)


def langevin_update(v, mass, gamma, kT, dt, xi):
    """Exact Ornstein-Uhlenbeck update of the velocities over dt for
    m dv/dt = -m gamma v + f(t), <f(t) f(t')> = 2 m gamma kT delta(t - t')
    (Eqs. 13-14 without the potential force): v <- c v + sqrt((1 - c^2) kT / m) xi,
    c = exp(-gamma dt).  kT in kJ/mol, mass in amu, v in nm/ps."""
    c = np.exp(-np.asarray(gamma, np.float64) * dt)
    sig = np.sqrt((1.0 - c * c) * kT / np.asarray(mass, np.float64))
    return np.asarray(c)[..., None] * v + np.asarray(sig)[..., None] * xi


def pulse_table(pulses, t_start_fs: float, dt_fs: float, n_steps: int) -> np.ndarray:
    """Photons/nm^2 per step for a list of pulses (photon keV, FWHM fs,
    fluence ph/um^2, centre fs, shape)."""
    P = np.ascontiguousarray([[p.photon_kev, p.fwhm_fs, p.fluence_ph_um2, p.t_center_fs, p.shape]
                              for p in pulses], dtype=np.float64).reshape(-1, 5)
    out = np.empty(n_steps)
    lib().orc_pulse_table(len(P), _ptr(P), float(t_start_fs), float(dt_fs), int(n_steps), _ptr(out))
    return out


def fragments(x, box, rep_off, r_frag):
    """Fragments of a state (the ion yields of Sec. III, reading): the
    connected components of the graph joining atoms of one replica closer
    than r_frag (minimum image), found by breadth-first search over the
    KD-tree's pair set.  Returns each atom's label, the smallest atom index
    of its fragment."""
    from scipy.spatial import cKDTree
    n = len(x)
    label = np.full(n, -1, dtype=np.int64)
    for r in range(len(rep_off) - 1):
        a0, a1 = int(rep_off[r]), int(rep_off[r + 1])
        L = np.asarray(box[r], np.float64)
        per = bool((L > 0).all())
        xr = np.mod(x[a0:a1], L) if per else x[a0:a1]
        tree = cKDTree(xr, boxsize=L if per else None)
        pairs = tree.query_pairs(r_frag, output_type="ndarray")
        adj = [[] for _ in range(a1 - a0)]
        for i, j in pairs:
            adj[i].append(j)
            adj[j].append(i)
        for s in range(a1 - a0):                    # ascending: s is its fragment's smallest index
            if label[a0 + s] >= 0:
                continue
            label[a0 + s] = a0 + s
            todo = [s]
            while todo:
                u = todo.pop()
                for v in adj[u]:
                    if label[a0 + v] < 0:
                        label[a0 + v] = a0 + s
                        todo.append(v)
    return label


def ion_yield_counts(label, q, mass_number, rep_off, mass_max, charge_max):
    """Fragments per replica by mass number (the sum of the atoms' mass
    numbers) and net charge (the sum of their charges), [R][mass_max + 1]
    [charge_max + 1]; larger values go to the last bin."""
    label = np.asarray(label)
    R = len(rep_off) - 1
    out = np.zeros((R, mass_max + 1, charge_max + 1), dtype=np.int64)
    m = np.zeros(len(label), dtype=np.int64)
    z = np.zeros(len(label), dtype=np.int64)
    np.add.at(m, label, np.asarray(mass_number, np.int64))
    np.add.at(z, label, np.asarray(q, np.int64))
    for r in range(R):
        for i in range(int(rep_off[r]), int(rep_off[r + 1])):
            if label[i] == i:
                out[r, min(m[i], mass_max), min(z[i], charge_max)] += 1
    return out


def probe_sums(x, x0, q, species, box_of_atom, n_species):
    """Per species: the summed charge (int64) and the summed squared
    displacement |x - x0|^2 from the reference positions (nm^2, minimum image
    of the replica's box) of the given atoms."""
    d = _min_image(np.asarray(x, np.float64) - np.asarray(x0, np.float64), box_of_atom)
    d2 = (d * d).sum(1)
    sp = np.asarray(species).astype(np.int64)
    qs = np.array([int(np.asarray(q, np.int64)[sp == k].sum()) for k in range(n_species)], dtype=np.int64)
    ms = np.array([float(d2[sp == k].sum()) for k in range(n_species)])
    return qs, ms


def probe_weights(pulses, t_start_fs, dt_fs, f):
    """Probe weights of Eq. 17 (Sec. II.C): w_k = int_{t_k}^{t_k + dt} g f dt /
    int g f dt over the recorded window, t_k = t_start + k dt.  The charges,
    hence f = 1 - zbar/Z, change only at step ends, so each step's integral is
    f_k times the integral of the probe profile g over the step (the pulse
    table); the pulse's fluence cancels in the ratio."""
    f = np.asarray(f, np.float64)
    gf = pulse_table(pulses, t_start_fs, dt_fs, len(f)) * f
    tot = gf.sum()
    return gf / tot if tot > 0 else np.zeros_like(gf)


def probe_weighted_displacement(pulses, t_start_fs, dt_fs, q_sum, d2_sum, n_of_species, z):
    """Probe-weighted displacement per species (Eq. 17 reading): records
    k = 0..n-1 of the summed charge and squared displacement of each species
    give f_k = 1 - (q_sum / N_s) / Z_s and the RMS displacement
    d_k = sqrt(d2_sum / N_s); the result is sum_k w_k d_k with the weights of
    probe_weights.  Species without atoms give 0."""
    q_sum = np.asarray(q_sum, np.float64)
    d2_sum = np.asarray(d2_sum, np.float64)
    out = np.zeros(q_sum.shape[1])
    for s in range(q_sum.shape[1]):
        n = float(n_of_species[s])
        if n <= 0:
            continue
        f = 1.0 - (q_sum[:, s] / n) / float(z[s])
        w = probe_weights(pulses, t_start_fs, dt_fs, f)
        out[s] = float((w * np.sqrt(d2_sum[:, s] / n)).sum())
    return out


def plasma_scalars(n_e_count: int, e_gas_mev: int, volume: float, *, dt_ps: float,
                   te_floor_ev: float, dte_ev: float, n_te: int,
                   coulomb_f: float = COULOMB_F, prescribed=None):
    """Free-electron-gas scalars (Sec. II.A, Eq. 3).

    T_e = (2/3) E_gas / N_e (E_gas in meV -> eV: divide by 1500 N_e),
    n_e = N_e / V, kappa^2 = 4 pi f n_e / (k_B T_e) with k_B T_e in kJ/mol
    and T_e floored at ``te_floor_ev``; kappa = 0 when n_e = 0.
    Also the CR helpers n_e*dt and the uniform-grid position (i0, w).
    ``prescribed`` = (n_e, T_e) replaces the bookkeeping values.
    """
    if prescribed is not None:
        n_e, te = float(prescribed[0]), float(prescribed[1])
    elif n_e_count > 0:
        te = float(e_gas_mev) / (1500.0 * float(n_e_count))
        n_e = float(n_e_count) / volume
    else:
        te, n_e = 0.0, 0.0
    if n_e > 0.0:
        tc = te if te > te_floor_ev else te_floor_ev
        four_pi_f = 4.0 * math.pi * coulomb_f
        k2 = (four_pi_f * n_e) / (tc * EV_KJMOL)
        kappa = math.sqrt(k2)
    else:
        kappa = 0.0
    ne_dt = n_e * dt_ps
    x = te * (1.0 / dte_ev)
    if x > float(n_te - 1):
        x = float(n_te - 1)
    if x < 0.0:
        x = 0.0
    i0 = int(x)
    if i0 > n_te - 2:
        i0 = n_te - 2
    w = x - float(i0)
    return dict(te_ev=te, n_e=n_e, kappa=kappa, ne_dt=ne_dt, it0=i0, wt=w)


# ---------------------------------------------------------------------------
# Whole-system oracle
# ---------------------------------------------------------------------------
def bond_scale(q_sum, n_atoms):
    """Scaling of a bonded term by the charges of its atoms (Sec. II.B, Eq. 9,
    reading): c = 1 - zbar/N with zbar the summed charge of the term's N atoms,
    clamped to [0, 1] -- 1 for neutral atoms, 0 once their mean charge is 1."""
    return np.clip(1.0 - np.asarray(q_sum, np.float64) / float(n_atoms), 0.0, 1.0)


def morse(r, De, be, beta):
    """Morse bond (Sec. II.B, Eq. 10, reading): V = D_e (1 - e^{-beta (r - b_e)})^2,
    zero at the equilibrium distance b_e and D_e at dissociation.  Returns
    (V, dV/dr)."""
    e = np.exp(-beta * (r - be))
    return De * (1.0 - e) ** 2, 2.0 * De * beta * e * (1.0 - e)


def harmonic_angle(theta, k, theta0):
    """Harmonic angle term (Sec. III: methane clusters): V = (k/2)(theta - theta0)^2.
    Returns (V, dV/dtheta)."""
    return 0.5 * k * (theta - theta0) ** 2, k * (theta - theta0)


def _min_image(d, L):
    """d minus the nearest multiple of the box L, per row (L = 0: vacuum)."""
    per = L > 0
    return np.where(per, d - L * np.round(d / np.where(per, L, 1.0)), d)


def bonded_forces(x, q, box_of_atom, topology):
    """Forces and per-atom energies of the bonded terms (Sec. II.B, Eqs. 9-10):
    Morse bonds and harmonic angles, each scaled by its bond_scale at the
    current charges (a constant factor of the term: charges are integers and
    are not differentiated).  A term's energy is shared equally among its
    atoms.  Distances take the minimum image of the replica's box."""
    n = len(x)
    F = np.zeros((n, 3))
    U = np.zeros(n)
    q = np.asarray(q, np.float64)
    b = np.asarray(topology.bonds)
    if len(b):
        i, j, t = b[:, 0], b[:, 1], b[:, 2]
        De, be, beta = np.asarray(topology.bond_params, np.float64)[t].T
        d = _min_image(x[i] - x[j], box_of_atom[i])
        r = np.sqrt((d * d).sum(1))
        V, dV = morse(r, De, be, beta)
        c = bond_scale(q[i] + q[j], 2)
        fi = (-c * dV / r)[:, None] * d
        np.add.at(F, i, fi)
        np.add.at(F, j, -fi)
        np.add.at(U, i, 0.5 * c * V)
        np.add.at(U, j, 0.5 * c * V)
    a = np.asarray(topology.angles)
    if len(a):
        i, j, k, t = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
        kt, th0 = np.asarray(topology.angle_params, np.float64)[t].T
        u = _min_image(x[i] - x[j], box_of_atom[j])
        w = _min_image(x[k] - x[j], box_of_atom[j])
        ru = np.sqrt((u * u).sum(1))
        rw = np.sqrt((w * w).sum(1))
        cos = (u * w).sum(1) / (ru * rw)
        theta = np.arccos(np.clip(cos, -1.0, 1.0))
        V, dV = harmonic_angle(theta, kt, th0)
        c = bond_scale(q[i] + q[j] + q[k], 3)
        # -dV/dx_i = (dV/dtheta / sin theta) d(cos theta)/dx_i, likewise for k
        g = c * dV / np.sin(theta)
        fi = g[:, None] * (w / (ru * rw)[:, None] - (cos / (ru * ru))[:, None] * u)
        fk = g[:, None] * (u / (ru * rw)[:, None] - (cos / (rw * rw))[:, None] * w)
        np.add.at(F, i, fi)
        np.add.at(F, k, fk)
        np.add.at(F, j, -(fi + fk))
        for m in (i, j, k):
            np.add.at(U, m, c * V / 3.0)
    return F, U


def forces_of_atoms(sample, atomic, idx, *, r_cut, kappa, coulomb_f=COULOMB_F, sigma0=None, eps0=None,
                    ne=None):
    """Forces on the atoms `idx` of `sample` (at its positions and charges q0),
    each summed over every other atom of its replica (all pairs, FP64), with a
    fixed screening kappa per replica (and, with ``ne``, the hybrid
    electrostatics at that electron density).  Costs len(idx) * n_atoms pair
    terms, so it checks or times a sample of a system too large for all pairs."""
    from paper_2401_03180_gb300 import workloads as W
    md = OracleMD.__new__(OracleMD)
    md.n, md.R = sample.n_atoms, sample.n_replicas
    md.rc, md.f = float(r_cut), float(coulomb_f)
    md.kappa_fixed = -1.0
    md.z = np.ascontiguousarray(atomic.z, np.int32)
    md.off = np.concatenate([[0], np.cumsum(md.z + 1)]).astype(np.int32)
    md.c6, md.c12 = lj_table(md.z, W.LJ_SIGMA0 if sigma0 is None else sigma0, W.LJ_EPS0 if eps0 is None else eps0)
    md.nts = md.c6.shape[0]
    md.x = np.ascontiguousarray(sample.x, np.float64)
    md.q = np.ascontiguousarray(sample.q0, np.uint8)
    md.sp = np.ascontiguousarray(sample.species, np.uint8)
    md.frag = np.ascontiguousarray(sample.fragment, np.int32)
    md.rep_off = np.ascontiguousarray(sample.replica_offset, np.int32)
    md.rep_of = np.repeat(np.arange(md.R, dtype=np.int32), np.diff(md.rep_off))
    md.box = np.ascontiguousarray(sample.box, np.float64).reshape(md.R, 3)
    kap = np.broadcast_to(np.asarray(kappa, np.float64), (md.R,))
    md.hybrid = ne is not None
    nev = None if ne is None else np.ascontiguousarray(np.broadcast_to(np.asarray(ne, np.float64), (md.R,)))
    out = md.forces_subset(np.asarray(idx), kappa=np.ascontiguousarray(kap), ne=nev)
    if getattr(sample, "topology", None) is not None:
        out += bonded_forces(md.x, md.q, md.box[md.rep_of], sample.topology)[0][np.asarray(idx)]
    return out


class OracleMD:
    """The full step of the method on the CPU, in FP64.

    Step n (reading of the step order; the paper is silent):
      1. v += (dt/2) F/m          2. x += dt v (periodic wrap)
      3. CR update with the plasma scalars of step n-1 and the step-n RNG
      4. reduce -> N_e, E_gas -> kappa for step n+1
      5. F(x, q, kappa)           6. v += (dt/2) F/m
    """

    def __init__(self, sample, atomic, *, dt_ps=5e-5, r_cut=1.2, cr_enabled=True,
                 kappa_fixed=-1.0, te_floor_ev=1.0, t_start_fs=0.0, pulses=None,
                 dF_table=None, prescribed=None, n_steps_max=0, coulomb_f=COULOMB_F,
                 sigma0=None, eps0=None, mass=None, threads=None, screening="debye", langevin_g=None,
                 charge_table=None, with_forces=True):
        from paper_2401_03180_gb300 import workloads as W
        self.s = sample
        self.a = atomic
        self.dt = float(dt_ps)
        self.rc = float(r_cut)
        self.cr_enabled = bool(cr_enabled)
        self.kappa_fixed = float(kappa_fixed)
        if screening not in ("debye", "hybrid"):
            raise ValueError("screening must be 'debye' or 'hybrid'")
        self.hybrid = screening == "hybrid"
        # charge-state fractions per replica and step, [R][rows][n_ts] (None: RCM-1 rates)
        self.charge_table = None if charge_table is None else np.asarray(charge_table, np.float64)
        # electron-ion coupling coefficient per species (nm^3/ps): gamma = n_e g_s
        self.langevin_g = None if langevin_g is None else np.asarray(langevin_g, dtype=np.float64)
        self.te_floor = float(te_floor_ev)
        self.f = float(coulomb_f)
        self.n = sample.n_atoms
        self.R = sample.n_replicas
        self.z = np.ascontiguousarray(atomic.z, dtype=np.int32)
        self.off = np.concatenate([[0], np.cumsum(self.z + 1)]).astype(np.int32)
        self.mass = np.asarray(W.MASS if mass is None else mass, dtype=np.float64)
        sig0 = W.LJ_SIGMA0 if sigma0 is None else sigma0
        e0 = W.LJ_EPS0 if eps0 is None else eps0
        self.c6, self.c12 = lj_table(self.z, sig0, e0)
        self.nts = self.c6.shape[0]
        self.x = np.array(sample.x, dtype=np.float64, copy=True)
        self.v = np.array(sample.v, dtype=np.float64, copy=True)
        self.sp = np.ascontiguousarray(sample.species, dtype=np.uint8)
        self.frag = np.ascontiguousarray(sample.fragment, dtype=np.int32)
        self.q = np.array(sample.q0, dtype=np.uint8, copy=True)
        self.h = np.zeros(self.n, dtype=np.uint8)
        self.rep_off = np.ascontiguousarray(sample.replica_offset, dtype=np.int32)
        self.rep_of = np.repeat(np.arange(self.R, dtype=np.int32), np.diff(self.rep_off))
        self.local = (np.arange(self.n) - self.rep_off[self.rep_of]).astype(np.int32)
        self.box = np.ascontiguousarray(sample.box, dtype=np.float64).reshape(self.R, 3)
        self.topology = getattr(sample, "topology", None)
        self.vol = np.asarray(sample.volume, dtype=np.float64)
        self.seed = np.ascontiguousarray(sample.seed, dtype=np.uint64)
        self.step_index = 0
        self.etab, self.inv = exp_tables()
        with np.errstate(divide="ignore"):
            tau = np.asarray(atomic.tau_auger_ps, dtype=np.float64)
            self.auger_dt = np.where(tau > 0, self.dt / np.where(tau > 0, tau, 1.0), 0.0)
        self.hdtm = (0.5 * self.dt) / self.mass
        self.prescribed = prescribed   # (ne[R][steps+1], te[R][steps+1]) or None
        # per-step fluence tables, per replica
        if dF_table is not None:
            self.dF = np.asarray(dF_table, dtype=np.float64).reshape(self.R, -1)
        elif pulses is not None:
            n_max = max(int(n_steps_max), 1)
            self.dF = np.stack([pulse_table(pulses[r], t_start_fs, self.dt * 1000.0, n_max)
                                for r in range(self.R)])
        else:
            self.dF = np.zeros((self.R, max(int(n_steps_max), 1)))
        self.n_e = np.array([int(self.q[self.rep_off[r]:self.rep_off[r + 1]].astype(np.int64).sum())
                             for r in range(self.R)], dtype=np.int64)
        self.e_gas = np.zeros(self.R, dtype=np.int64)
        self.counts = np.zeros((self.R, 4), dtype=np.int64)
        self.scal = [self._scalars(r, 0) for r in range(self.R)]
        # with_forces=False: the charge dynamics alone.  Charges, K holes and the
        # electron gas never read positions, velocities or forces (Sec. II.A: the
        # gas is homogeneous, its volume fixed), so step() then advances exactly
        # the charge sequence of the full step without the all-pairs forces; for
        # systems far too large for all pairs.  Positions stay at their input.
        self.with_forces = bool(with_forces)
        if self.with_forces:
            self.F, self.U, self.n_pairs = self.forces()
        else:
            self.F, self.U, self.n_pairs = np.zeros((self.n, 3)), np.zeros(self.n), 0
        # probe records (Eq. 17): per replica, the summed charge and squared
        # displacement from the initial positions of each species, after each step
        self.x0 = self.x.copy()
        self.probe = [[] for _ in range(self.R)]
        self.probe_record()

    # -- pieces ------------------------------------------------------------
    def _scalars(self, r, step):
        pres = None
        if self.prescribed is not None:
            pres = (self.prescribed[0][r][step], self.prescribed[1][r][step])
        return plasma_scalars(int(self.n_e[r]), int(self.e_gas[r]), float(self.vol[r]),
                              dt_ps=self.dt, te_floor_ev=self.te_floor, dte_ev=self.a.dte_ev,
                              n_te=self.a.n_te, coulomb_f=self.f, prescribed=pres)

    def kappa(self):
        if self.kappa_fixed >= 0.0:
            return np.full(self.R, self.kappa_fixed)
        return np.array([s["kappa"] for s in self.scal])

    def type_state(self):
        return (self.off[self.sp.astype(np.int64)] + self.q).astype(np.int32)

    def electron_density(self):
        """n_e (nm^-3) per replica at the current plasma state."""
        return np.ascontiguousarray([s["n_e"] for s in self.scal], dtype=np.float64)

    def forces(self, x=None, q=None, kappa=None, ne=None):
        x = self.x if x is None else x
        q = self.q if q is None else q
        kap = self.kappa() if kappa is None else np.asarray(kappa, np.float64)
        if self.hybrid and ne is None:
            ne = self.electron_density()
        ts = (self.off[self.sp.astype(np.int64)] + q).astype(np.int32)
        xf = np.ascontiguousarray(x, dtype=np.float64)
        qd = np.ascontiguousarray(q, dtype=np.float64)
        F = np.zeros((self.n, 3)); U = np.zeros(self.n); npairs = ctypes.c_int64(0)
        nep = None if ne is None else _ptr(np.ascontiguousarray(ne, dtype=np.float64))
        lib().orc_forces(self.n, _ptr(xf), _ptr(ts), _ptr(qd), _ptr(self.frag), self.R,
                         _ptr(self.rep_off), _ptr(self.box), _ptr(np.ascontiguousarray(kap)), nep,
                         self.rc, self.f, self.nts, _ptr(self.c6), _ptr(self.c12), _ptr(F),
                         _ptr(U), ctypes.byref(npairs))
        if getattr(self, "topology", None) is not None:
            Fb, Ub = bonded_forces(xf, q, self.box[self.rep_of], self.topology)
            F += Fb
            U += Ub
        return F, U, int(npairs.value)

    def forces_subset(self, sel, x=None, q=None, kappa=None, ne=None):
        x = self.x if x is None else x
        q = self.q if q is None else q
        kap = self.kappa() if kappa is None else np.asarray(kappa, np.float64)
        if getattr(self, "hybrid", False) and ne is None:
            ne = self.electron_density()
        ts = (self.off[self.sp.astype(np.int64)] + q).astype(np.int32)
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        out = np.zeros((len(sel), 3))
        lib().orc_forces_subset(self.n, _ptr(np.ascontiguousarray(x)), _ptr(ts),
                                _ptr(np.ascontiguousarray(q, np.float64)), _ptr(self.frag),
                                _ptr(self.rep_of), _ptr(self.rep_off), _ptr(self.box),
                                _ptr(np.ascontiguousarray(kap)),
                                None if ne is None else _ptr(np.ascontiguousarray(ne, dtype=np.float64)),
                                self.rc, self.f, self.nts,
                                _ptr(self.c6), _ptr(self.c12), len(sel), _ptr(sel), _ptr(out))
        if getattr(self, "topology", None) is not None:
            out += bonded_forces(np.ascontiguousarray(x, np.float64), q, self.box[self.rep_of], self.topology)[0][sel]
        return out

    def cr_step(self, step):
        """One CR update of all atoms with the current scalars."""
        R = self.R
        dF = np.ascontiguousarray([self.dF[r][step] for r in range(R)], dtype=np.float64)
        ne_dt = np.ascontiguousarray([s["ne_dt"] for s in self.scal], dtype=np.float64)
        it0 = np.ascontiguousarray([s["it0"] for s in self.scal], dtype=np.int32)
        wt = np.ascontiguousarray([s["wt"] for s in self.scal], dtype=np.float64)
        dNe = np.zeros(R, dtype=np.int64); dE = np.zeros(R, dtype=np.int64)
        cnt = np.zeros((R, 4), dtype=np.int64)
        a = self.a
        lib().orc_cr_step(self.n, _ptr(self.sp), _ptr(self.q), _ptr(self.h), _ptr(self.local),
                          _ptr(self.rep_of), int(step), _ptr(self.seed), _ptr(dF), _ptr(ne_dt),
                          _ptr(it0), _ptr(wt), len(self.z), _ptr(self.z),
                          _ptr(np.ascontiguousarray(a.sigma_pi, np.float64)), _ptr(self.auger_dt),
                          _ptr(np.ascontiguousarray(a.k_ci, np.float64)),
                          _ptr(np.ascontiguousarray(a.k_rec, np.float64)), int(a.n_te),
                          _ptr(np.ascontiguousarray(a.ip_mev, np.int64)),
                          _ptr(np.ascontiguousarray(a.e_pi_mev, np.int64)),
                          _ptr(np.ascontiguousarray(a.e_auger_mev, np.int64)), _ptr(self.etab),
                          N_ETAB, _ptr(self.inv), _ptr(dNe), _ptr(dE), _ptr(cnt))
        return dNe, dE, cnt

    def _wrap(self):
        for r in range(self.R):
            L = self.box[r]
            if L[0] > 0 and L[1] > 0 and L[2] > 0:
                sl = slice(self.rep_off[r], self.rep_off[r + 1])
                self.x[sl] -= L * np.floor(self.x[sl] / L)

    def probe_record(self):
        ns = len(self.z)
        for r in range(self.R):
            sl = slice(self.rep_off[r], self.rep_off[r + 1])
            self.probe[r].append(probe_sums(self.x[sl], self.x0[sl], self.q[sl], self.sp[sl],
                                            np.repeat(self.box[r:r + 1], sl.stop - sl.start, 0), ns))

    def probe_series(self, r):
        """Records 0..step of replica r: (q_sum [n][S] int64, d2_sum [n][S] nm^2)."""
        return (np.array([a for a, _ in self.probe[r]], dtype=np.int64),
                np.array([b for _, b in self.probe[r]], dtype=np.float64))

    # -- the step ----------------------------------------------------------
    def langevin(self, n):
        """The O step of step n (reading of Eqs. 13-14): each replica's atoms
        relax towards T_e with gamma = n_e g_s, n_e and T_e being the plasma
        scalars the charge update of step n reads."""
        for r in range(self.R):
            sl = slice(self.rep_off[r], self.rep_off[r + 1])
            sc = self.scal[r]
            gam = sc["n_e"] * self.langevin_g[self.sp[sl]]
            xi = gaussians(int(self.seed[r]), self.local[sl], n)
            self.v[sl] = langevin_update(self.v[sl], self.mass[self.sp[sl]], gam, sc["te_ev"] * EV_KJMOL, self.dt, xi)

    def table_step(self, step):
        """Charges of the state after step n from row n + 1 of the fractions
        table (reading of Sec. II.A); K holes are not tracked (h = 0)."""
        R = self.R
        dNe = np.zeros(R, dtype=np.int64); cnt = np.zeros((R, 4), dtype=np.int64)
        for r in range(R):
            sl = slice(self.rep_off[r], self.rep_off[r + 1])
            cum = cumulative_fractions(self.charge_table[r][step + 1], self.off)
            u = charge_quantiles(int(self.seed[r]), self.local[sl])
            qn = table_charges(u, self.sp[sl], self.z, self.off, cum)
            dq = qn.astype(np.int64) - self.q[sl].astype(np.int64)
            dNe[r] = int(dq.sum())
            cnt[r, 0] = int(dq[dq > 0].sum())
            cnt[r, 3] = int(-dq[dq < 0].sum())
            self.q[sl] = qn
            self.h[sl] = 0
        return dNe, np.zeros(R, dtype=np.int64), cnt

    def charge_update(self, n):
        """Steps 3-4 of step n: the charge update with the plasma scalars of
        step n - 1, then the reduction to the scalars of step n + 1."""
        if self.cr_enabled:
            dNe, dE, cnt = self.table_step(n) if self.charge_table is not None else self.cr_step(n)
            self.n_e += dNe
            self.e_gas = np.maximum(self.e_gas + dE, 0)
            self.counts += cnt
        self.scal = [self._scalars(r, n + 1) for r in range(self.R)]

    def step(self):
        n = self.step_index
        if not self.with_forces:
            self.charge_update(n)
            self.step_index = n + 1
            return
        hd = self.hdtm[self.sp][:, None]
        self.v += hd * self.F
        if self.langevin_g is not None:
            self.langevin(n)
        self.x += self.dt * self.v
        self._wrap()
        self.charge_update(n)
        self.F, self.U, self.n_pairs = self.forces()
        self.v += hd * self.F
        self.step_index = n + 1
        self.probe_record()

    def run(self, n_steps, record=None):
        for _ in range(n_steps):
            self.step()
            if record is not None:
                record(self)

    # -- observables ---------------------------------------------------------
    def kinetic(self):
        m = self.mass[self.sp]
        return np.array([0.5 * float((m[self.rep_off[r]:self.rep_off[r + 1], None]
                                      * self.v[self.rep_off[r]:self.rep_off[r + 1]] ** 2).sum())
                         for r in range(self.R)])

    def potential(self):
        return np.array([float(self.U[self.rep_off[r]:self.rep_off[r + 1]].sum())
                         for r in range(self.R)])
