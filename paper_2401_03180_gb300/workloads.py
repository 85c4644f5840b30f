"""Seeded synthetic inputs for the ionising-MD hot path.

This module only *creates inputs*: sample geometries, velocities, species and
fragment labels, pulse parameters, and the synthetic atomic-data tables that
the collisional-radiative (CR) update reads.  It holds none of the method's
arithmetic (no pair potential, no combining rule, no pulse integral, no rate
evaluation, no integrator), so both the CUDA library and the CPU oracle can
consume exactly the same inputs without sharing any computation.

Shapes follow the paper's samples (Sec. II.D): bulk water, a solvated
protein crystal, and methane clusters at liquid density, with the pulse
parameters of Sec. III/IV.  The real samples (PDB structures, Gromacs-inserted
clusters) and the Cretin atomic data are not available, so:

* geometries are built on jittered lattices at the stated densities, with
  random molecular orientations and inter-molecular clash removal (the paper
  inserts molecules by van der Waals radii and minimises; we reject clashes
  instead);
* LJ parameters are synthetic round numbers, not taken from any force field;
* cross sections, Auger lifetimes, ionisation potentials and rate
  coefficients are synthetic closed forms (Slater-screened hydrogenic binding
  energies, a Kramers-like Z^4/E^3 photo-absorption law, a Lotz-like
  collisional-ionisation law), with magnitudes chosen so the configured
  fluences give mean charges from ~0.01 to a few per heavy atom.

Units: nm, ps, amu, kJ/mol, elementary charge; pulse times in fs; fluence in
photons/um^2; energies stored for the CR update in integer meV.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Species (index, symbol, Z, mass in amu)
# ----------------------------------------------------------------------------
SPECIES = ("H", "C", "N", "O", "S")
Z = np.array([1, 6, 7, 8, 16], dtype=np.int32)
MASS = np.array([1.008, 12.011, 14.007, 15.999, 32.06], dtype=np.float64)
H, C, N, O, S = range(5)

# Synthetic neutral LJ parameters (sigma nm, epsilon kJ/mol); round numbers of
# the usual magnitude, not copied from any force field.
LJ_SIGMA0 = np.array([0.110, 0.340, 0.325, 0.300, 0.360], dtype=np.float64)
LJ_EPS0 = np.array([0.100, 0.360, 0.600, 0.650, 1.050], dtype=np.float64)

KB_KJ = 0.0083144626          # kJ/mol/K, used only to draw Maxwell velocities
RYDBERG_EV = 13.605693        # eV, scale of the synthetic binding energies


def ts_offsets(z: np.ndarray = Z) -> np.ndarray:
    """Row layout of the per-type-state tables: state (s, q) is row off[s]+q."""
    return np.concatenate([[0], np.cumsum(np.asarray(z) + 1)]).astype(np.int32)


def charge_fraction_table(pulses, t_start_fs: float, dt_fs: float, n_rows: int, z=Z,
                          mean_final: float = 2.0) -> np.ndarray:
    """A synthetic stand-in for a CR code's time-resolved charge-state
    fractions (the paper reads them from Cretin, which is not available):
    per species a Poisson distribution truncated at Z, whose mean rises with
    the pulses' cumulative fluence to ``mean_final`` * Z_s / 6 at the end.
    Row n holds the fractions at t_n = t_start + n dt; columns follow the
    type-state layout (species s, charge q) -> off[s] + q.  Input data only."""
    from math import erf, exp, factorial, log, sqrt
    z = np.asarray(z)
    off = ts_offsets(z)
    t = t_start_fs + dt_fs * np.arange(n_rows)
    cum = np.zeros(n_rows)
    tot = 0.0
    for p in pulses:
        sig = p.fwhm_fs / (2.0 * sqrt(2.0 * log(2.0)))
        cum += p.fluence_ph_um2 * np.array([0.5 * (1.0 + erf((tt - p.t_center_fs) / (sig * sqrt(2.0)))) for tt in t])
        tot += p.fluence_ph_um2
    frac_t = cum / tot if tot > 0 else np.zeros(n_rows)
    out = np.zeros((n_rows, int(off[-1])))
    for s, zs in enumerate(z):
        for n in range(n_rows):
            lam = mean_final * zs / 6.0 * frac_t[n]
            f = np.array([exp(-lam) * lam ** k / factorial(k) for k in range(zs + 1)])
            f[-1] = max(0.0, 1.0 - f[:-1].sum())
            out[n, off[s]:off[s + 1]] = f / f.sum()
    return out


# ----------------------------------------------------------------------------
# Synthetic atomic data
# ----------------------------------------------------------------------------
def _slater_binding_ev(z: int, n_el: int) -> float:
    """Binding energy of the outermost of n_el electrons around a nucleus of
    charge z, from Slater's screening rules and the hydrogenic formula."""
    if n_el <= 0:
        return 0.0
    if n_el <= 2:
        n, s = 1, 0.30 * (n_el - 1)
    elif n_el <= 10:
        n, s = 2, 0.85 * 2 + 0.35 * (n_el - 3)
    else:
        n, s = 3, 1.00 * 2 + 0.85 * 8 + 0.35 * (n_el - 11)
    zeff = max(z - s, 0.5)
    return RYDBERG_EV * zeff * zeff / (n * n)


def _e1(x: np.ndarray) -> np.ndarray:
    from scipy.special import exp1
    return exp1(x)


@dataclass
class AtomicData:
    photon_kev: float
    z: np.ndarray
    ts_offset: np.ndarray
    sigma_pi: np.ndarray      # [n_ts, 2] nm^2, column h (K-hole flag)
    tau_auger_ps: np.ndarray  # [n_species], <= 0 means no Auger channel
    ip_mev: np.ndarray        # [n_ts] int64, ionisation potential q -> q+1
    e_pi_mev: np.ndarray      # [n_ts, 2] int64, energy given to the gas per PI
    e_auger_mev: np.ndarray   # [n_species] int64
    k_ci: np.ndarray          # [n_ts, n_te] nm^3/ps on a uniform Te grid
    k_rec: np.ndarray         # [n_ts, n_te] nm^3/ps
    dte_ev: float
    n_te: int

    @property
    def n_ts(self) -> int:
        return int(self.ts_offset[-1])


def atomic_data(photon_kev: float, *, n_te: int = 1024, dte_ev: float = 4.0,
                ci_scale: float = 1.0, rec_scale: float = 1.0,
                pi_scale: float = 1.0, z: np.ndarray = Z) -> AtomicData:
    """Synthetic CR tables for the five species at one photon energy.

    sigma_pi[s,q,h]: per-electron K-shell cross section 0.5*9.2e-9 nm^2 *
      (Z/6)^4 * (8 keV/E)^3 (a Kramers-like law normalised to ~92 b for carbon
      at 8 keV) times the K occupancy, plus 5% of that per outer electron.
    tau_auger = 10 fs * (6/Z)^2 for Z >= 3 (no Auger for H).
    ip[s,q]: Slater-screened hydrogenic binding of the outermost electron.
    e_pi[s,q,h]: photon energy minus the binding of the removed electron
      (the K binding when the photo-ionisation opens a K hole).
    e_auger[s]: K binding minus twice the neutral outer binding.
    k_ci: Lotz-like  3e-6 cm^3/s * xi / (IP * sqrt(T)) * E1(IP/T)  (eV units),
      xi = number of outer electrons; converted to nm^3/ps.
    k_rec: 5 nm^3/ps * q^2 * (T/1 eV)^-1.5 (a cold-plasma recombination law).
    The Te grid is T_k = k*dte_ev (evaluated at max(T_k, 1 eV)).
    """
    z = np.asarray(z, dtype=np.int32)
    off = ts_offsets(z)
    n_ts = int(off[-1])
    e_kev = float(photon_kev)
    sig = np.zeros((n_ts, 2))
    ip = np.zeros(n_ts, dtype=np.int64)
    epi = np.zeros((n_ts, 2), dtype=np.int64)
    kci = np.zeros((n_ts, n_te))
    krec = np.zeros((n_ts, n_te))
    tau = np.zeros(len(z))
    eaug = np.zeros(len(z), dtype=np.int64)
    t_grid = np.maximum(np.arange(n_te) * dte_ev, 1.0)
    cm3s_to_nm3ps = 1e21 / 1e12
    for s, zs in enumerate(z):
        zs = int(zs)
        sig_k = 0.5 * 9.2e-9 * (zs / 6.0) ** 4 * (8.0 / e_kev) ** 3 * pi_scale
        sig_out = 0.05 * sig_k
        ip_k = _slater_binding_ev(zs, 2) if zs >= 2 else _slater_binding_ev(zs, 1)
        tau[s] = 0.010 * (6.0 / zs) ** 2 if zs >= 3 else 0.0
        if zs >= 3:
            eaug[s] = int(round(1000.0 * max(ip_k - 2.0 * _slater_binding_ev(zs, zs), 0.0)))
        for q in range(zs + 1):
            row = off[s] + q
            n_el = zs - q
            ip_q = _slater_binding_ev(zs, n_el)
            ip[row] = int(round(1000.0 * ip_q))
            for h in (0, 1):
                if n_el == 0:
                    continue
                n_k = max(min(2 - h, n_el), 0)
                n_out = n_el - n_k
                sig[row, h] = n_k * sig_k + n_out * sig_out
                opens_k_hole = (zs >= 3 and h == 0 and zs - (q + 1) >= 2)
                bind = ip_k if opens_k_hole else ip_q
                epi[row, h] = int(round(1000.0 * max(1000.0 * e_kev - bind, 0.0)))
            if n_el > 0:
                xi = max(n_el - 2, 1) if n_el > 2 else n_el
                x = ip_q / t_grid
                k = 3e-6 * xi / (ip_q * np.sqrt(t_grid)) * _e1(x)
                kci[row] = ci_scale * k * cm3s_to_nm3ps
            if q > 0:
                krec[row] = rec_scale * 5.0 * q * q * t_grid ** -1.5
    return AtomicData(photon_kev=e_kev, z=z, ts_offset=off, sigma_pi=sig,
                      tau_auger_ps=tau, ip_mev=ip, e_pi_mev=epi,
                      e_auger_mev=eaug, k_ci=kci, k_rec=krec,
                      dte_ev=float(dte_ev), n_te=int(n_te))


# ----------------------------------------------------------------------------
# Pulses
# ----------------------------------------------------------------------------
GAUSSIAN, FLAT_TOP = 0, 1


@dataclass
class Pulse:
    photon_kev: float
    fwhm_fs: float
    fluence_ph_um2: float
    t_center_fs: float
    shape: int = GAUSSIAN


# ----------------------------------------------------------------------------
# Sample geometry
# ----------------------------------------------------------------------------
@dataclass
class Sample:
    """Atoms of one or more independent replicas, concatenated."""
    x: np.ndarray            # [N,3] float64 nm
    v: np.ndarray            # [N,3] float64 nm/ps
    species: np.ndarray      # [N] uint8
    fragment: np.ndarray     # [N] int32 (LJ excluded within a fragment)
    q0: np.ndarray           # [N] uint8 initial charges
    replica_offset: np.ndarray   # [R+1] int32
    seed: np.ndarray         # [R] uint64 RNG key per replica
    box: np.ndarray          # [R,3] float64; zeros = vacuum
    volume: np.ndarray       # [R] electron-gas volume nm^3
    name: str = ""
    meta: dict = field(default_factory=dict)
    topology: "Topology | None" = None   # bonded terms (None: no bonds)

    @property
    def n_atoms(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_replicas(self) -> int:
        return int(self.replica_offset.shape[0] - 1)


@dataclass
class Topology:
    """Bonded terms of the native structure (Sec. II.B): Morse bonds i-j and
    angles i-j-k with vertex j, by type.  Atom indices are global (into the
    concatenated sample).  Input data only: the potentials are evaluated by
    the library and by the oracle."""
    bonds: np.ndarray          # [n_bonds, 3] int32: i, j, type
    bond_params: np.ndarray    # [n_bond_types, 3] float64: D_e (kJ/mol), b_e (nm), beta (1/nm)
    angles: np.ndarray         # [n_angles, 4] int32: i, j (vertex), k, type
    angle_params: np.ndarray   # [n_angle_types, 2] float64: k_theta (kJ/mol/rad^2), theta_0 (rad)


# Synthetic bonded parameters: round numbers of the usual magnitude, not copied
# from any force field.  The equilibrium geometry is that of the molecule
# templates below (O-H 0.1 nm, H-O-H 104.5 deg; C-H 0.109 nm, tetrahedral).
BOND_PARAMS = np.array([[450.0, 0.100, 22.0],     # 0: O-H
                        [420.0, 0.109, 18.0]])    # 1: C-H
ANGLE_PARAMS = np.array([[380.0, math.radians(104.5)],                  # 0: H-O-H
                         [320.0, math.acos(-1.0 / 3.0)]])               # 1: H-C-H


def molecular_topology(sample: "Sample") -> Topology:
    """Bonds and angles of every water (O, H, H) and methane (C, H, H, H, H)
    molecule of a sample, found as fragments of consecutive atoms with that
    species sequence.  Other fragments (the protein's pseudo-residues) get no
    bonded terms."""
    frag = np.asarray(sample.fragment)
    sp = np.asarray(sample.species)
    n = len(frag)
    if n == 0:
        return Topology(np.zeros((0, 3), np.int32), BOND_PARAMS.copy(), np.zeros((0, 4), np.int32),
                        ANGLE_PARAMS.copy())
    start = np.flatnonzero(np.concatenate([[True], frag[1:] != frag[:-1]]))
    length = np.diff(np.concatenate([start, [n]]))
    bonds, angles = [], []

    def match(ln, seq):
        ok = length == ln
        for k, s_k in enumerate(seq):
            ok &= sp[np.minimum(start + k, n - 1)] == s_k
        return start[ok]

    w = match(3, (O, H, H))
    if len(w):
        bonds += [np.stack([w, w + 1, np.zeros_like(w)], 1), np.stack([w, w + 2, np.zeros_like(w)], 1)]
        angles += [np.stack([w + 1, w, w + 2, np.zeros_like(w)], 1)]
    m = match(5, (C, H, H, H, H))
    if len(m):
        one = np.ones_like(m)
        bonds += [np.stack([m, m + k, one], 1) for k in range(1, 5)]
        angles += [np.stack([m + a, m, m + b, one], 1) for a in range(1, 5) for b in range(a + 1, 5)]
    b = np.concatenate(bonds).astype(np.int32) if bonds else np.zeros((0, 3), np.int32)
    a = np.concatenate(angles).astype(np.int32) if angles else np.zeros((0, 4), np.int32)
    return Topology(b[np.argsort(b[:, 0], kind="stable")], BOND_PARAMS.copy(),
                    a[np.argsort(a[:, 1], kind="stable")], ANGLE_PARAMS.copy())


def with_topology(sample: "Sample") -> "Sample":
    """The sample with the bonded terms of its water and methane molecules."""
    import dataclasses
    return dataclasses.replace(sample, topology=molecular_topology(sample))


def _rand_rotations(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                     2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                     2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
                    -1).reshape(n, 3, 3)


def _water_template():
    th = math.radians(104.5) / 2
    return (np.array([[0.0, 0.0, 0.0],
                      [0.1 * math.sin(th), 0.1 * math.cos(th), 0.0],
                      [-0.1 * math.sin(th), 0.1 * math.cos(th), 0.0]]),
            np.array([O, H, H], dtype=np.uint8))


def _methane_template():
    d = 0.109 / math.sqrt(3.0)
    return (np.array([[0, 0, 0], [d, d, d], [d, -d, -d], [-d, d, -d], [-d, -d, d]], dtype=np.float64),
            np.array([C, H, H, H, H], dtype=np.uint8))


def _place_rigid(rng, sites, tmpl, box=None, d_min=0.16, max_iter=60, fixed=None):
    """Put one copy of a rigid template at each site with a random orientation,
    re-drawing orientations (and jitter) of molecules whose atoms come closer
    than d_min to an atom of another molecule.  Returns [n_mol, n_at, 3]."""
    from scipy.spatial import cKDTree
    pos, _ = tmpl
    n_mol, n_at = len(sites), len(pos)
    centre = pos.mean(0)
    base = pos - centre
    jit = 0.02
    cur_sites = sites + rng.uniform(-jit, jit, sites.shape)
    rot = _rand_rotations(rng, n_mol)
    redo = np.arange(n_mol)
    coords = np.empty((n_mol, n_at, 3))
    for _ in range(max_iter):
        coords[redo] = cur_sites[redo, None, :] + np.einsum("mij,aj->mai", rot[redo], base)
        flat = coords.reshape(-1, 3)
        if box is not None:
            flat = np.mod(flat, box)
        mol_id = np.repeat(np.arange(n_mol), n_at)
        pts, ids = flat, mol_id
        if fixed is not None and len(fixed):
            pts = np.concatenate([flat, fixed])
            ids = np.concatenate([mol_id, np.full(len(fixed), -1)])
        tree = cKDTree(pts, boxsize=box) if box is not None else cKDTree(pts)
        pr = tree.query_pairs(d_min, output_type="ndarray")
        if len(pr) == 0:
            break
        a, b = ids[pr[:, 0]], ids[pr[:, 1]]
        bad = (a != b)
        clash = np.unique(np.concatenate([a[bad], b[bad]]))
        clash = clash[clash >= 0]
        if len(clash) == 0:
            break
        redo = clash
        rot[redo] = _rand_rotations(rng, len(redo))
        cur_sites[redo] = sites[redo] + rng.uniform(-jit, jit, (len(redo), 3))
    return coords


def _lattice(n_side, a, origin=0.0):
    g = np.arange(n_side)
    return (np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.5) * a + origin


def _maxwell(rng, species, temp_k=300.0):
    sd = np.sqrt(KB_KJ * temp_k / MASS[species])
    v = rng.normal(size=(len(species), 3)) * sd[:, None]
    # remove net momentum of the sample (input preparation)
    m = MASS[species][:, None]
    v -= (m * v).sum(0) / m.sum()
    return v


def _molecules_to_sample(coords, tmpl_species, rng, box, volume, seed, name, frag0=0):
    n_mol, n_at, _ = coords.shape
    x = coords.reshape(-1, 3)
    if box is not None:
        x = np.mod(x, box)
    sp = np.tile(tmpl_species, n_mol)
    frag = np.repeat(np.arange(n_mol, dtype=np.int32), n_at) + frag0
    return x, sp, frag


def _single(x, sp, frag, rng, box, volume, seed, name, meta=None):
    n = len(x)
    return Sample(x=np.ascontiguousarray(x, dtype=np.float64),
                  v=_maxwell(rng, sp),
                  species=sp.astype(np.uint8), fragment=frag.astype(np.int32),
                  q0=np.zeros(n, dtype=np.uint8),
                  replica_offset=np.array([0, n], dtype=np.int32),
                  seed=np.array([seed], dtype=np.uint64),
                  box=np.array([box if box is not None else [0.0, 0.0, 0.0]], dtype=np.float64),
                  volume=np.array([volume], dtype=np.float64), name=name, meta=meta or {})


def water_box(n_mol: int, box_nm: float, seed: int) -> Sample:
    """Bulk water in a periodic cube, O-H 0.1 nm, H-O-H 104.5 deg."""
    rng = np.random.default_rng(seed)
    n_side = int(math.ceil(n_mol ** (1 / 3)))
    a = box_nm / n_side
    sites = _lattice(n_side, a)
    sites = sites[np.sort(rng.permutation(len(sites))[:n_mol])]
    box = np.array([box_nm] * 3)
    tmpl = _water_template()
    coords = _place_rigid(rng, sites, tmpl, box=box)
    x, sp, frag = _molecules_to_sample(coords, tmpl[1], rng, box, None, seed, "water")
    return _single(x, sp, frag, rng, box, box_nm ** 3, seed, f"water_box_{len(x)}")


def _sphere_sites(n_mol, density_per_nm3, rng):
    a = density_per_nm3 ** (-1 / 3)
    radius = (3 * n_mol / (4 * math.pi * density_per_nm3)) ** (1 / 3)
    n_side = int(math.ceil(2 * radius / a)) + 2
    g = _lattice(n_side, a, origin=-n_side * a / 2)
    r = np.linalg.norm(g, axis=1) + rng.uniform(0, 1e-6, len(g))
    sites = g[np.argsort(r)[:n_mol]]
    return sites, radius


def water_droplet(n_mol: int, seed: int, density_g_cm3: float = 1.0) -> Sample:
    """Spherical water droplet in vacuum."""
    rng = np.random.default_rng(seed)
    nd = density_g_cm3 * 6.02214076e23 / 18.015 * 1e-21
    sites, radius = _sphere_sites(n_mol, nd, rng)
    tmpl = _water_template()
    coords = _place_rigid(rng, sites, tmpl)
    x, sp, frag = _molecules_to_sample(coords, tmpl[1], rng, None, None, seed, "droplet")
    vol = 4 / 3 * math.pi * radius ** 3
    return _single(x, sp, frag, rng, None, vol, seed, f"water_droplet_{len(x)}",
                   {"radius_nm": radius})


def methane_cluster(n_mol: int, seed: int, density_g_cm3: float = 0.42) -> Sample:
    """Methane cluster at liquid density in vacuum (C-H 0.109 nm, tetrahedral)."""
    rng = np.random.default_rng(seed)
    nd = density_g_cm3 * 6.02214076e23 / 16.043 * 1e-21
    sites, radius = _sphere_sites(n_mol, nd, rng)
    tmpl = _methane_template()
    coords = _place_rigid(rng, sites, tmpl)
    x, sp, frag = _molecules_to_sample(coords, tmpl[1], rng, None, None, seed, "methane")
    vol = 4 / 3 * math.pi * radius ** 3
    return _single(x, sp, frag, rng, None, vol, seed, f"methane_{len(x)}",
                   {"radius_nm": radius})


PROTEIN_COMPOSITION = {H: 50.0, C: 32.0, N: 9.0, O: 9.0, S: 0.3}


def protein_crystal(n_atoms: int = 200_000, seed: int = 1003, n_cells: int = 3,
                    globule_radius: float = 2.0, atom_density: float = 114.0) -> Sample:
    """Periodic lattice of compact globules (one per unit cell) in water.

    Heavy atoms sit on a jittered lattice inside each globule with one H per
    heavy atom on average; species are drawn from the stated composition
    (normalised).  Globule atoms are grouped into pseudo-residues of 8-20
    atoms along a space-filling order; water fills the remaining volume at
    1 g/cm^3 until the atom count is reached.
    """
    rng = np.random.default_rng(seed)
    comp = np.array([PROTEIN_COMPOSITION[s] for s in range(5)])
    comp = comp / comp.sum()
    glob_vol = 4 / 3 * math.pi * globule_radius ** 3
    n_glob_atoms = int(round(glob_vol * atom_density))
    frac_h = comp[H]
    heavy_p = comp.copy(); heavy_p[H] = 0; heavy_p /= heavy_p.sum()
    water_nd = 1.0 * 6.02214076e23 / 18.015 * 1e-21
    n_glob_total = n_cells ** 3 * n_glob_atoms
    n_water_mol = (n_atoms - n_glob_total) // 3
    # cell edge so that globules plus water fill the box at the given densities
    vol = n_cells ** 3 * glob_vol + n_water_mol / water_nd
    box_nm = vol ** (1 / 3)
    cell = box_nm / n_cells
    xs, sps, frags = [], [], []
    frag_id = 0
    n_heavy = int(round(n_glob_atoms * (1 - frac_h)))
    n_h = n_glob_atoms - n_heavy
    a_heavy = (glob_vol / n_heavy) ** (1 / 3)
    for ci in range(n_cells ** 3):
        cx = (np.array(np.unravel_index(ci, (n_cells,) * 3)) + 0.5) * cell
        n_side = int(math.ceil(2 * globule_radius / a_heavy)) + 2
        g = _lattice(n_side, a_heavy, origin=-n_side * a_heavy / 2)
        r = np.linalg.norm(g, axis=1) + rng.uniform(0, 1e-6, len(g))
        hv = g[np.argsort(r)[:n_heavy]] + rng.uniform(-0.02, 0.02, (n_heavy, 3))
        hsp = rng.choice(5, size=n_heavy, p=heavy_p).astype(np.uint8)
        owner = rng.permutation(n_heavy)[:n_h] if n_h <= n_heavy else rng.integers(0, n_heavy, n_h)
        hx = _attach_h(rng, hv, owner)
        pos = np.concatenate([hv, hx]) + cx
        sp = np.concatenate([hsp, np.full(n_h, H, np.uint8)])
        parent = np.concatenate([np.arange(n_heavy), owner])
        # pseudo-residues: order heavy atoms along a Morton curve, cut into
        # groups of 8-20 atoms (heavy atoms with their hydrogens)
        key = _morton3(np.floor((hv - hv.min(0)) / 0.25).astype(np.int64))
        order = np.argsort(key, kind="stable")
        res_of_heavy = np.empty(n_heavy, dtype=np.int64)
        i = 0
        while i < n_heavy:
            size = int(rng.integers(4, 11))  # 4-10 heavy atoms -> ~8-20 atoms
            res_of_heavy[order[i:i + size]] = frag_id
            frag_id += 1
            i += size
        fr = res_of_heavy[parent]
        pos = _relax_clashes(pos, fr)
        xs.append(pos); sps.append(sp); frags.append(fr)
    gx = np.concatenate(xs); gsp = np.concatenate(sps); gfr = np.concatenate(frags).astype(np.int32)
    # water on a lattice outside the globules
    cen = (np.stack(np.meshgrid(*[np.arange(n_cells)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) * cell
    from scipy.spatial import cKDTree
    ctree = cKDTree(cen, boxsize=box_nm)
    n_side = int(math.ceil(box_nm * water_nd ** (1 / 3)))
    while True:  # finest lattice that leaves room for all water molecules
        a_w = box_nm / n_side
        sites = _lattice(n_side, a_w)
        dmin, _ = ctree.query(np.mod(sites, box_nm))
        sites = sites[dmin > globule_radius + 0.15]
        if len(sites) >= n_water_mol:
            break
        n_side += 1
    sites = sites[np.sort(rng.permutation(len(sites))[:n_water_mol])]
    tmpl = _water_template()
    box = np.array([box_nm] * 3)
    coords = _place_rigid(rng, sites, tmpl, box=box, fixed=np.mod(gx, box_nm))
    wx, wsp, wfr = _molecules_to_sample(coords, tmpl[1], rng, box, None, seed, "water",
                                        frag0=frag_id)
    sp = np.concatenate([gsp, wsp]); fr = np.concatenate([gfr, wfr])
    x = np.mod(_relax_clashes(np.concatenate([gx, wx]), fr, box=box), box_nm)
    return _single(x, sp, fr, rng, box, box_nm ** 3, seed, f"protein_crystal_{len(x)}",
                   {"box_nm": box_nm, "n_globule_atoms": int(n_glob_total)})


def _attach_h(rng, heavy, owner, bond=0.1, n_try=24):
    """One H per owner heavy atom at ``bond`` nm, in the candidate direction
    farthest from the other heavy atoms and from H already placed."""
    from scipy.spatial import cKDTree
    tree = cKDTree(heavy)
    dirs = rng.normal(size=(len(owner), n_try, 3))
    dirs /= np.linalg.norm(dirs, axis=2, keepdims=True)
    cand = heavy[owner][:, None, :] + bond * dirs
    d, idx = tree.query(cand.reshape(-1, 3), k=2)
    d = d.reshape(len(owner), n_try, 2); idx = idx.reshape(len(owner), n_try, 2)
    # nearest heavy atom that is not the owner
    near = np.where(idx[..., 0] == owner[:, None], d[..., 1], d[..., 0])
    best = np.argmax(near, axis=1)
    hx = cand[np.arange(len(owner)), best]
    # re-draw H that sit too close to another H
    for _ in range(8):
        pr = cKDTree(hx).query_pairs(0.15, output_type="ndarray")
        if len(pr) == 0:
            break
        bad = np.unique(pr[:, 0])
        dd = rng.normal(size=(len(bad), n_try, 3))
        dd /= np.linalg.norm(dd, axis=2, keepdims=True)
        cc = heavy[owner[bad]][:, None, :] + bond * dd
        hx_others = cKDTree(np.delete(hx, bad, axis=0))
        dh, _ = hx_others.query(cc.reshape(-1, 3))
        dv, iv = tree.query(cc.reshape(-1, 3), k=2)
        dv = dv.reshape(len(bad), n_try, 2); iv = iv.reshape(len(bad), n_try, 2)
        nv = np.where(iv[..., 0] == owner[bad][:, None], dv[..., 1], dv[..., 0])
        score = np.minimum(nv, dh.reshape(len(bad), n_try))
        b2 = np.argmax(score, axis=1)
        hx[bad] = cc[np.arange(len(bad)), b2]
    return hx


def _relax_clashes(x, frag, d_min=0.16, iters=100, box=None):
    """Push apart atoms of different fragments that are closer than d_min
    (each moves half the deficit along the pair axis); a crude stand-in for
    the energy minimisation the paper applies to inserted samples."""
    from scipy.spatial import cKDTree
    x = x.copy()
    for _ in range(iters):
        if box is not None:
            x = np.mod(x, box)
        pr = cKDTree(x, boxsize=box).query_pairs(d_min, output_type="ndarray")
        if len(pr):
            pr = pr[frag[pr[:, 0]] != frag[pr[:, 1]]]
        if len(pr) == 0:
            break
        d = x[pr[:, 0]] - x[pr[:, 1]]
        if box is not None:
            d -= box * np.round(d / box)
        r = np.linalg.norm(d, axis=1, keepdims=True)
        u = np.where(r > 1e-9, d / np.maximum(r, 1e-12), np.array([[1.0, 0.0, 0.0]]))
        push = 0.5 * (d_min - r) * 1.05 * u
        np.add.at(x, pr[:, 0], push)
        np.add.at(x, pr[:, 1], -push)
    return x


def _morton3(ijk: np.ndarray) -> np.ndarray:
    out = np.zeros(len(ijk), dtype=np.int64)
    for b in range(16):
        for d in range(3):
            out |= ((ijk[:, d] >> b) & 1) << (3 * b + d)
    return out


def concat(samples: list[Sample], name: str = "batch") -> Sample:
    """Independent replicas in one system (each keeps its own seed/box/volume)."""
    offs = np.concatenate([[0], np.cumsum([s.n_atoms for s in samples])]).astype(np.int32)
    frag = []
    f0 = 0
    for s in samples:
        frag.append(s.fragment + f0)
        f0 += int(s.fragment.max()) + 1 if s.n_atoms else 0
    return Sample(x=np.concatenate([s.x for s in samples]),
                  v=np.concatenate([s.v for s in samples]),
                  species=np.concatenate([s.species for s in samples]),
                  fragment=np.concatenate(frag).astype(np.int32),
                  q0=np.concatenate([s.q0 for s in samples]),
                  replica_offset=offs,
                  seed=np.concatenate([s.seed for s in samples]),
                  box=np.concatenate([s.box for s in samples]),
                  volume=np.concatenate([s.volume for s in samples]),
                  name=name, topology=_concat_topology(samples, offs))


def _concat_topology(samples, offs):
    tops = [s.topology for s in samples]
    if all(t is None for t in tops):
        return None
    ref = next(t for t in tops if t is not None)
    bonds, angles = [], []
    for t, o in zip(tops, offs[:-1]):
        if t is None:
            continue
        if not (np.array_equal(t.bond_params, ref.bond_params) and np.array_equal(t.angle_params, ref.angle_params)):
            raise ValueError("replicas with bonded terms must share the parameter tables")
        b = t.bonds.copy(); b[:, :2] += o
        a = t.angles.copy(); a[:, :3] += o
        bonds.append(b); angles.append(a)
    return Topology(np.concatenate(bonds).astype(np.int32), ref.bond_params.copy(),
                    np.concatenate(angles).astype(np.int32), ref.angle_params.copy())


# ----------------------------------------------------------------------------
# The five workloads (shapes of the paper's samples and pulses)
# ----------------------------------------------------------------------------
DT_PS = 5e-5          # 50 as
R_CUT = 1.2           # nm


@dataclass
class Workload:
    name: str
    sample: Sample
    pulses: list          # list of lists (one per replica) of Pulse
    n_steps: int
    t_start_fs: float
    photon_kev: float


def _window(p: Pulse):
    return p.t_center_fs - p.fwhm_fs


def workload(name: str, *, scale: float = 1.0) -> Workload:
    """Build one of the named workloads.

    c1_methane_1500   300 CH4 (1,500 atoms), 0.42 g/cm^3 sphere, vacuum;
                      8 keV, 10 fs FWHM, 1e12 ph/um^2; 400 steps.
    c2_water_30k      10,000 H2O in a periodic 6.7 nm box; 6 keV, 25 fs,
                      5e12 ph/um^2; 1,000 steps.
    c3_protein_200k   200,000-atom globule lattice in water (periodic); two
                      9 keV 10 fs pulses 50 fs apart at 1e13 ph/um^2; 1,400 steps.
    c4_methane_batch  256 methane clusters of 500-20,000 atoms (log-uniform),
                      fluence log-uniform 1e11-1e13, 8 keV 10 fs; 400 steps.
    c5_droplet_2m     2,000,000-atom water droplet, vacuum; 8 keV, 20 fs,
                      1e13 ph/um^2; 800 steps.
    ``scale`` < 1 shrinks atom counts (for quick tests), keeping densities.
    """
    if name.startswith("c1"):
        n_mol = max(int(300 * scale), 2)
        s = methane_cluster(n_mol, seed=1001)
        p = Pulse(8.0, 10.0, 1e12, 0.0)
        return Workload(name, s, [[p]], 400, _window(p), 8.0)
    if name.startswith("c2"):
        n_mol = max(int(10_000 * scale), 8)
        box = 6.7 * (n_mol / 10_000) ** (1 / 3)
        s = water_box(n_mol, box, seed=1002)
        p = Pulse(6.0, 25.0, 5e12, 0.0)
        return Workload(name, s, [[p]], 1000, _window(p), 6.0)
    if name.startswith("c3"):
        s = (protein_crystal(int(200_000 * scale), seed=1003) if scale >= 1 else
             protein_crystal(max(int(200_000 * scale), 6000), seed=1003, n_cells=1))
        p1 = Pulse(9.0, 10.0, 1e13, 0.0)
        p2 = Pulse(9.0, 10.0, 1e13, 50.0)
        return Workload(name, s, [[p1, p2]], 1400, -10.0, 9.0)
    if name.startswith("c4"):
        rng = np.random.default_rng(1004)
        n_rep = max(int(256 * scale), 2)
        sizes = np.exp(rng.uniform(math.log(500), math.log(20_000), n_rep))
        flu = np.exp(rng.uniform(math.log(1e11), math.log(1e13), n_rep))
        reps, pulses = [], []
        for k in range(n_rep):
            n_mol = max(int(sizes[k] * (scale if scale < 1 else 1) / 5), 2)
            rep = methane_cluster(n_mol, seed=4000 + k)
            reps.append(rep)
            pulses.append([Pulse(8.0, 10.0, float(flu[k]), 0.0)])
        s = concat(reps, "methane_batch")
        return Workload(name, s, pulses, 400, -10.0, 8.0)
    if name.startswith("c5"):
        n_mol = max(int(2_000_000 * scale / 3), 8)
        s = water_droplet(n_mol, seed=1005)
        p = Pulse(8.0, 20.0, 1e13, 0.0)
        return Workload(name, s, [[p]], 800, _window(p), 8.0)
    raise KeyError(name)


WORKLOADS = ("c1_methane_1500", "c2_water_30k", "c3_protein_200k",
             "c4_methane_batch", "c5_droplet_2m")
