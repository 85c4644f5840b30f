/*
 * md.h -- C ABI of the GB300 ionising-MD hot path.
 *
 * One timestep of an X-ray-irradiated sample, following the hybrid
 * collisional-radiative / molecular-dynamics method of arXiv 2401.03180:
 *   (a) cell-list neighbour build (cutoff chosen from the screening, Sec. II.B);
 *   (b) screened Coulomb (Sec. II.A, Eq. 2) plus screened, charge-scaled LJ
 *       (Sec. II.B, Eqs. 8 and 11) pair forces, LJ excluded inside a native
 *       fragment (Sec. II.B);
 *   (c) stochastic integer charge update from photo-ionisation, Auger decay,
 *       collisional ionisation and recombination (Sec. II.A: processes named
 *       there, charges assigned stochastically per atom);
 *   (d) free-electron-gas reduction giving the Debye length (Sec. II.A, Eq. 3);
 *   (e) velocity-Verlet integration of Newton's equation (Sec. II.B, Eq. 12).
 *
 * Units: nm, ps, amu, kJ/mol, elementary charge; pulse times in fs, fluence
 * in photons/um^2, electron-gas energies in integer meV.
 *
 * Ownership: every pointer passed in is read during the call only (inputs are
 * copied); outputs are written to caller-owned buffers.  The library owns its
 * device memory, obtained from md_config.dev_alloc when set (e.g. a PyTorch
 * caching allocator) and from cudaMalloc otherwise.  Arrays are host pointers
 * unless a name starts with d_.
 *
 * Errors: every call returns an md_status; md_last_error() gives the text.
 * After a device-side error (MD_ERR_FIXED_OVERFLOW, MD_ERR_NONFINITE,
 * MD_ERR_CELL_OVERFLOW) the handle accepts only md_get_state, md_last_error
 * and md_finalize.  No kernel traps or spins without a bound.
 *
 * Threading: one handle is driven by one host thread at a time.  All device
 * work of a handle is issued on its stream (md_set_stream; default: the
 * legacy default stream).
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int md_status;
enum {
    MD_OK = 0,
    MD_ERR_INVALID_ARG = 1,    /* argument out of range / inconsistent      */
    MD_ERR_BAD_STATE = 2,      /* call order violated, or handle poisoned   */
    MD_ERR_OOM = 3,            /* device allocation failed                  */
    MD_ERR_CUDA = 4,           /* a CUDA runtime call failed                */
    MD_ERR_FIXED_OVERFLOW = 5, /* a force/energy exceeded the fixed-point range */
    MD_ERR_TIMEOUT = 6,        /* a bounded device wait gave up             */
    MD_ERR_NONFINITE = 7,      /* NaN/Inf in positions or velocities        */
    MD_ERR_CELL_OVERFLOW = 8,  /* cell-list or pair-list capacity exceeded  */
    MD_ERR_TABLE_END = 9       /* stepped past the per-step pulse table     */
};

#define MD_MAX_SPECIES 8
#define MD_MAX_Z 32
#define MD_MAX_TYPE_STATES 128 /* sum over species of (Z + 1)              */

enum { MD_PREC_MIXED = 0, MD_PREC_FP64 = 1 };
enum { MD_PLASMA_BOOKKEEPING = 0, MD_PLASMA_PRESCRIBED = 1 };
enum { MD_SCREEN_DEBYE = 0, MD_SCREEN_HYBRID = 1 };
enum { MD_CHARGE_RATES = 0, MD_CHARGE_TABLE = 1 };
enum { MD_PULSE_GAUSSIAN = 0, MD_PULSE_FLAT_TOP = 1 };

/*
 * Run configuration and atomic data.
 *
 * precision: MD_PREC_MIXED = FP32 pair arithmetic with per-atom 64-bit
 *   fixed-point force sums (scale 2^32 kJ/mol/nm), FP64 positions,
 *   velocities, integrator and plasma sums; MD_PREC_FP64 = the same path
 *   with FP64 pair arithmetic.
 * plasma_mode: MD_PLASMA_BOOKKEEPING derives n_e = N_e/V and
 *   k_B T_e = (2/3) E_gas/N_e from the integer electron count and gas energy
 *   of each replica; MD_PLASMA_PRESCRIBED reads n_e and T_e per step from
 *   md_set_plasma_table (the paper reads T_e from the CR calculation, Sec. II.B).
 * kappa_fixed: >= 0 forces 1/lambda_D to this value (nm^-1) in the pair
 *   forces (the CR rates still use the plasma scalars); < 0 derives it (Eq. 3).
 * The CR tables are indexed by type state ts = off[s] + q with
 *   off[0] = 0, off[s+1] = off[s] + Z[s] + 1, and:
 *   sigma_pi   [n_ts][2]    photo-ionisation cross section (nm^2), column = K-hole flag
 *   k_ci       [n_ts][n_te] collisional-ionisation rate coefficient (nm^3/ps)
 *   k_rec      [n_ts][n_te] recombination rate coefficient (nm^3/ps)
 *   ip_mev     [n_ts]       ionisation potential q -> q+1 (meV)
 *   e_pi_mev   [n_ts][2]    energy given to the electron gas per PI event (meV)
 *   e_auger_mev[n_species]  energy given per Auger event (meV)
 *   T_e grid: T_k = k * dte_ev, k = 0 .. n_te-1, linear interpolation, clamped.
 */
typedef struct md_config {
    double dt_ps;            /* timestep (ps), > 0                          */
    double r_cut;            /* pair cutoff (nm), > 0                       */
    int precision;           /* MD_PREC_*                                   */
    int cr_enabled;          /* 1: charge update on; 0: charges frozen      */
    int plasma_mode;         /* MD_PLASMA_*                                 */
    int max_steps;           /* length of the per-step tables (>= 1)        */
    double kappa_fixed;      /* see above                                   */
    double t_start_fs;       /* time of step 0 (fs)                         */
    double te_floor_ev;      /* lower bound of T_e used in kappa (eV), > 0  */
    double coulomb_f;        /* 1/(4 pi eps0) in kJ mol^-1 nm e^-2          */
    double photon_kev;       /* photon energy the sigma_pi column is for    */
    int n_species;           /* 1 .. MD_MAX_SPECIES                         */
    int z[MD_MAX_SPECIES];   /* nuclear charge, 1 .. MD_MAX_Z               */
    double mass[MD_MAX_SPECIES];        /* amu                              */
    double lj_sigma0[MD_MAX_SPECIES];   /* neutral LJ sigma (nm)            */
    double lj_eps0[MD_MAX_SPECIES];     /* LJ epsilon (kJ/mol)              */
    double tau_auger_ps[MD_MAX_SPECIES];/* K-hole Auger lifetime; <= 0: none */
    const double* sigma_pi;
    const double* k_ci;
    const double* k_rec;
    const int64_t* ip_mev;
    const int64_t* e_pi_mev;
    const int64_t* e_auger_mev;
    int n_te;                /* >= 2                                        */
    double dte_ev;           /* > 0                                         */
    /* optional device allocator (both or neither); ctx is passed back     */
    void* (*dev_alloc)(size_t bytes, void* ctx);
    void (*dev_free)(void* ptr, void* ctx);
    void* alloc_ctx;
    int autotune;            /* 1: time launch shapes at init and keep the fastest */
    int profile;             /* 1: time the pair kernel with CUDA events in md_step */
    int list_reserve;        /* cluster-pair list entries per cluster allocated
                                at init; 0: automatic (32, and at least twice
                                what the initial configuration needs).  The
                                list grows whenever a build needs more room
                                (see md_step)                                  */
    double list_skin_nm;     /* Verlet buffer of the cluster-pair list (nm).
                                0: cells and list are rebuilt every step.  > 0:
                                the list is built with r_cut + skin and kept
                                until some atom has moved more than skin/2 since
                                the build (then rebuilt within the same step);
                                the pair set within r_cut is the same, only the
                                grouping of the FP32 partial sums follows the
                                build (one schedule for all replicas).  Periodic
                                edges need >= 3 (r_cut + skin).                 */
    int screening;           /* MD_SCREEN_DEBYE: the Coulomb term is Debye-
                                screened (Sec. II.A, Eq. 2).  MD_SCREEN_HYBRID:
                                hybrid ion-sphere / Debye electrostatics (Sec.
                                II.A, Eqs. 4-7), read as follows.  An ion of
                                charge Q has R = (3Q/(4 pi n_e))^{1/3} and r'
                                from Eq. 7; its potential is Q/r + c1 - c2 r^2
                                for r < r' and G e^{-kappa r}/r outside, with
                                c1, c2 and G from the continuity of the
                                potential and its first two derivatives at r'.
                                A pair's Coulomb energy is f (q_j phi_i +
                                q_i phi_j) / 2, shifted to zero at r_cut.  The
                                mixed path keeps G in FP32 and saturates it at
                                1e30 (kappa r' > ~69).  0 (Debye) by default.  */
    double langevin_g[MD_MAX_SPECIES];
                             /* electron-ion coupling per species (nm^3/ps),
                                Sec. II.B, Eqs. 13-14, read as follows: each
                                atom of species s feels the friction
                                -m gamma v with gamma = n_e langevin_g[s] and a
                                Gaussian force with <f f> = 2 m gamma k_B T_e
                                (n_e and T_e: the plasma scalars the step's
                                charge update reads), integrated as the exact
                                Ornstein-Uhlenbeck update v <- c v +
                                sqrt((1 - c^2) k_B T_e / m) xi, c = e^{-gamma
                                dt}, after the first half kick.  xi: Philox4x32-
                                10 stream 1 (key = seed, counter = (atom index
                                in the replica, step, 1, 0)) through Box-Muller.
                                All zero (the default): no coupling.           */
    int charge_mode;         /* MD_CHARGE_RATES (default): the charge update
                                draws events from the rates (RCM-1).
                                MD_CHARGE_TABLE: charges follow per-step
                                charge-state fractions of a CR calculation
                                (md_set_charge_table), the paper's mode (Sec.
                                II.A: integer charges assigned stochastically
                                so that, averaged, they match the CR charge
                                states).  Read as quantile coupling: each atom
                                keeps one uniform quantile u (Philox4x32-10
                                stream 2, key = seed, counter = (atom index in
                                the replica, 0, 2, 0), 53-bit) and takes the
                                smallest q whose cumulative fraction of its
                                species exceeds u (Z if rounding leaves none).
                                K holes stay 0; N_e follows sum q; the gas
                                energy is not changed (use plasma_mode =
                                MD_PLASMA_PRESCRIBED for T_e).                 */
    int probe_record;        /* 1: keep, after every step k (record 0: the
                                initial state), per replica and species, the
                                summed charge and the summed squared
                                displacement from the initial positions, for
                                the probe-weighted displacement of Eq. 17
                                (md_get_probe_series, md_probe_displacement).
                                Costs one kernel per step. 0 (default): off.  */
    /* Launch shapes (the paper has no counterpart; they change no result: the
     * fixed-point sums and the list's layout do not depend on them).  0 keeps
     * the default, or the autotuner's choice when autotune = 1; a nonzero
     * value pins that axis (the autotuner then leaves it alone).            */
    int pair_warps;          /* warps per force-kernel block: 4, 8 or 12
                                (FP64: 4 or 8)                                 */
    int pair_blocks_per_sm;  /* force-kernel blocks per SM, >= 1, within the
                                occupancy the shape allows                     */
    int sort_threads;        /* threads per cell-sort block: 256 or 1024       */
    int list_blocks_per_sm;  /* list-build blocks (8 warps) per SM: 1 .. 16    */
    int list_skin_adaptive;  /* 1 (with list_skin_nm > 0): the device drops the
                                Verlet buffer while it does not pay and takes
                                it back when it would.  A buffered list that
                                lived fewer than 3 steps makes the next lists
                                unbuffered (cutoff r_cut, rebuilt every step,
                                no trimming pass); while unbuffered, once the
                                largest one-step displacement d of any atom is
                                at most list_skin_nm / 12 (a buffered list would
                                last 6 steps or more), the next list carries
                                the skin again.  md_set_state starts again from
                                a buffered list.  Same pair set within r_cut
                                either way; the grouping of the FP32 partial
                                sums follows the lists, so a checkpoint resumes
                                bit for bit only with a fixed skin.  0
                                (default): the skin is fixed.                */
} md_config;

/*
 * The sample: n_atoms atoms of n_replicas independent replicas stored
 * back to back (replica r owns atoms replica_offset[r] .. replica_offset[r+1]-1).
 * Replicas share the configuration but have their own RNG seed, box, gas
 * volume and pulses; a replica run alone gives the same result bit for bit
 * (with list_skin_nm > 0 the list is rebuilt for all replicas when any of
 * them needs it, so forces then match a solo run to FP32 rounding of the
 * block sums, and charges still bit for bit).
 * box[3r..3r+2] > 0: periodic (minimum image; every edge >= 3 r_cut);
 * all zero: vacuum.  volume[r]: electron-gas volume (nm^3) for n_e = N_e/V.
 * fragment: LJ is excluded between atoms with equal fragment id.
 */
typedef struct md_system {
    int n_atoms;                      /* >= 1                               */
    const double* x;                  /* [3*n_atoms] AoS positions (nm)     */
    const double* v;                  /* [3*n_atoms] AoS velocities (nm/ps) */
    const uint8_t* species;           /* [n_atoms] < n_species              */
    const int32_t* fragment;          /* [n_atoms]                          */
    const uint8_t* q0;                /* [n_atoms] initial charge <= Z, or NULL (0) */
    int n_replicas;                   /* >= 1                               */
    const int32_t* replica_offset;    /* [n_replicas+1], 0 .. n_atoms       */
    const uint64_t* seed;             /* [n_replicas] Philox key            */
    const double* box;                /* [3*n_replicas]                     */
    const double* volume;             /* [n_replicas] > 0                   */
    /*
     * Bonded terms of the native structure (Sec. II.B, Eqs. 9-10; Sec. III
     * names the harmonic angle term).  All optional: n_bonds = n_angles = 0
     * (a zero-filled tail of the struct) gives none.  Readings:
     *  - a bond i-j is the Morse potential V = D_e (1 - e^{-beta (r - b_e)})^2,
     *    zero at the equilibrium distance b_e and D_e at dissociation (the
     *    printed Eq. 10 has lost the width beta and the square of the bracket);
     *  - an angle i-j-k with vertex j is V = (k_theta / 2)(theta - theta_0)^2;
     *  - each term is scaled by c = 1 - zbar/N clamped to [0, 1] (Eq. 9), zbar
     *    the summed charge of its N atoms (2 or 3) at the current charges:
     *    c = 1 for neutral atoms and 0 once their mean charge reaches 1.  c is
     *    a constant of the force (charges are integers);
     *  - a term's energy is shared equally among its atoms; distances take the
     *    minimum image of the replica's box.
     * The atoms of a term must be distinct and belong to one replica and one
     * fragment: LJ is omitted between bonded atoms while the screened Coulomb
     * stays (Sec. II.B), which the fragment rule gives.  Anything else is
     * MD_ERR_INVALID_ARG.  The library copies the arrays.
     */
    int n_bonds;                      /* >= 0                               */
    const int32_t* bonds;             /* [n_bonds][3]: i, j, bond type      */
    int n_bond_types;                 /* >= 1 when n_bonds > 0              */
    const double* bond_params;        /* [n_bond_types][3]: D_e >= 0 (kJ/mol),
                                         b_e >= 0 (nm), beta > 0 (1/nm)     */
    int n_angles;                     /* >= 0                               */
    const int32_t* angles;            /* [n_angles][4]: i, j (vertex), k, angle type */
    int n_angle_types;                /* >= 1 when n_angles > 0             */
    const double* angle_params;       /* [n_angle_types][2]: k_theta >= 0
                                         (kJ/mol/rad^2), theta_0 in [0, pi] (rad) */
} md_system;

/* One X-ray pulse (Sec. II.A: pulse energy, duration, photon energy). */
typedef struct md_pulse {
    double photon_kev;       /* must equal md_config.photon_kev              */
    double fwhm_fs;          /* > 0; the width of a flat-top pulse          */
    double fluence_ph_um2;   /* >= 0                                        */
    double t_center_fs;
    int shape;               /* MD_PULSE_*                                  */
} md_pulse;

/* State exchange (md_get_state / md_set_state).  Unused pointers may be NULL. */
enum {
    MD_FIELD_X = 1,        /* x [3n] AoS                                     */
    MD_FIELD_V = 2,        /* v [3n] AoS, at the integer step                */
    MD_FIELD_F = 4,        /* f [3n] AoS (get only)                          */
    MD_FIELD_Q = 8,        /* q [n]                                          */
    MD_FIELD_H = 16,       /* h [n] K-hole flag                              */
    MD_FIELD_PLASMA = 32,  /* n_e, e_gas_mev [R]; te_ev, kappa [R] get only  */
    MD_FIELD_COUNTS = 64,  /* event_counts [R][4] (PI, Auger, CI, REC), get only */
    MD_FIELD_STEP = 128,   /* step                                           */
    MD_FIELD_XLIST = 256,  /* x_list [3n] AoS: positions of the last list
                              build (list_skin_nm > 0; otherwise equal to x).
                              md_set_state rebuilds the list from them, so a
                              resumed run groups its sums as the original did */
    MD_FIELD_ALL = 511
};
typedef struct md_state {
    double* x;
    double* v;
    double* f;
    uint8_t* q;
    uint8_t* h;
    int64_t* n_e;
    int64_t* e_gas_mev;
    double* te_ev;
    double* kappa;
    int64_t* event_counts;
    int64_t step;
    double* x_list;
} md_state;

/* Accumulated device time of the pair kernel (md_config.profile = 1). */
typedef struct md_timing {
    double pair_ms;          /* sum of CUDA-event durations                 */
    int64_t pair_launches;
    int64_t steps;
    int64_t pair_count_last; /* in-cutoff pairs of the last evaluated step (md_get_energies) */
    int tile_warps;          /* launch shape in use                         */
    int tile_blocks_per_sm;
    int64_t list_capacity;   /* cluster-pair list entries allocated         */
    int64_t list_entries;    /* entries the last list build used            */
    int64_t list_grows;      /* times the list was enlarged on demand       */
    int64_t list_builds;     /* cell + list builds in md_step since init or
                                md_reset_timing (equals steps when the skin is 0) */
    int sort_threads;        /* cell-sort block size in use                 */
    int list_blocks_per_sm;  /* list-build blocks per SM in use             */
    int build_kernels;       /* kernels of one cell + list build in the step
                                graph (5 to 12: the scans and the sort take
                                one or several kernels by grid size)       */
    int64_t list_unbuffered_builds; /* of list_builds, those without the skin
                                (list_skin_adaptive)                         */
} md_timing;

typedef struct md_handle md_handle;

/* Create a handle: validate, copy inputs, allocate, build the first cell
 * list and the initial forces F_0(x_0, q_0).  The inputs are the sample of
 * Sec. II.A/II.D (positions, velocities, species with their nuclear charge
 * and the per-charge-state LJ sizes of Sec. II.B Eq. 11, initial charges,
 * native fragments for the LJ exclusion of Sec. II.B, the electron-gas
 * volume of Eq. 3) and the atomic data the CR model needs (cross sections,
 * Auger lifetimes, ionisation potentials, rate coefficients; Sec. II.A).
 * cfg and sys are read during the call only; *out receives the handle
 * (owned by the caller, released with md_finalize) or NULL.  Errors:
 * INVALID_ARG (inconsistent sizes, values out of range; the message names
 * the field), OOM, CUDA. */
md_status md_init(const md_config* cfg, const md_system* sys, md_handle** out);

/* Issue all later device work on this cudaStream_t (NULL = legacy default). */
md_status md_set_stream(md_handle* h, void* cuda_stream);

/* The X-ray pulse(s) of Sec. II.A that drive photo-ionisation (photon
 * energy, FWHM, fluence, centre; Sec. II.D and IV give the paper's pulse
 * shapes: Gaussian, pump and probe pulses): the fluence per step of replica
 * `replica` (-1: all) from n_pulses pulses (host array, copied), over steps
 * 0 .. max_steps-1.  Gaussian pulses integrate the normal CDF with
 * sigma_t = FWHM / (2 sqrt(2 ln 2)) over each step; flat-top pulses the
 * overlap.  Uploads the table (the only host-to-device copy of a run).
 * Errors: INVALID_ARG (bad replica, a photon energy other than the
 * cross-section table's, FWHM <= 0, negative fluence, unknown shape),
 * BAD_STATE (poisoned handle), CUDA. */
md_status md_set_pulse(md_handle* h, int replica, const md_pulse* p, int n_pulses);

/* Same table given directly: dF[n] photons/nm^2 in step n (n < n_steps <= max_steps). */
md_status md_set_pulse_table(md_handle* h, int replica, const double* dF, int n_steps);

/* Overwrite entries first_step .. first_step+n-1 of the fluence table
 * (e.g. a per-step input streamed from the host); other entries unchanged. */
md_status md_set_pulse_table_at(md_handle* h, int replica, int first_step, const double* dF, int n);

/* The fluence of one step for every replica at once: dF[r] (photons/nm^2,
 * finite, >= 0) becomes entry `step` of replica r's table, r < n_replicas,
 * in one host-to-device copy ordered on the handle's stream (the host array
 * may be reused when the call returns only if it is pinned and the stream
 * has passed the copy; pageable memory is staged by the driver).  Errors:
 * INVALID_ARG (step outside [0, max_steps), null or bad values), CUDA. */
md_status md_set_fluence_at(md_handle* h, int step, const double* dF);

/* Charge-state fractions per step for charge_mode = MD_CHARGE_TABLE (Sec.
 * II.A: the CR calculation's time-resolved fraction of each charge state of
 * every species).  frac: host array [n_rows][n_ts] (copied), n_ts = the sum
 * over species of Z_s + 1, type state (s, q) in column off_s + q with off_s
 * = sum_{s' < s} (Z_s' + 1).  Row n holds the fractions at t_n = t_start +
 * n dt; the charge update of step n reads row n + 1.  Rows n_rows ..
 * max_steps keep their previous contents (at init: every atom neutral).
 * Each species' fractions must be >= 0 and sum to 1 within 1e-9.  The
 * library stores their running sums (FP64, in charge order).  replica = -1:
 * all replicas.  Errors: INVALID_ARG (bad replica, n_rows outside
 * [1, max_steps + 1], bad fractions), BAD_STATE (charge_mode is not
 * MD_CHARGE_TABLE), CUDA. */
md_status md_set_charge_table(md_handle* h, int replica, const double* frac, int n_rows);

/* Prescribed plasma (plasma_mode = MD_PLASMA_PRESCRIBED): n_e (nm^-3) and
 * T_e (eV) for steps 0 .. n_steps-1 (n_steps <= max_steps + 1). */
md_status md_set_plasma_table(md_handle* h, int replica, const double* ne,
                              const double* te_ev, int n_steps);

/* Advance every replica by n_steps timesteps of the method: per step, the
 * velocity-Verlet half kick and drift (Sec. II.B, Eq. 12), the stochastic
 * charge update (Sec. II.A) with the plasma scalars of the previous step, the
 * free-electron reduction to the Debye length (Sec. II.A, Eq. 3), the
 * neighbour list when the buffered one is used up (cutoff from the screening,
 * Sec. II.B), the pair forces (Sec. II.A Eq. 2, Sec. II.B Eqs. 8 and 11) and
 * the second half kick.  Asynchronous on the handle's stream except for a
 * final 4-byte status read.  When the atoms crowd
 * together beyond what the cluster-pair list was sized for, the steps stop
 * after the one that needs more room, the list grows (through dev_alloc when
 * given) and the remaining steps follow: the trajectory is the same as with a
 * larger list from the start.  Errors: BAD_STATE, TABLE_END, FIXED_OVERFLOW,
 * NONFINITE, CELL_OVERFLOW, OOM, CUDA. */
md_status md_step(md_handle* h, int n_steps);

/* md_step without the final status read: enqueues n_steps timesteps on the
 * handle's stream and returns.  Errors of those steps (and the list growth
 * md_step describes) are handled by the next md_sync, md_step,
 * md_get_state, md_set_state, md_get_energies or md_get_timing.  Errors:
 * BAD_STATE, TABLE_END, INVALID_ARG, CUDA. */
md_status md_step_async(md_handle* h, int n_steps);

/* Wait for the steps enqueued by md_step_async and read their status
 * (same errors as md_step). */
md_status md_sync(md_handle* h);

/* The outputs the paper reads from a run (Sec. II.A-II.C: time-resolved
 * ion charges and K holes, free-electron count, temperature and Debye
 * screening, positions for the structure and displacement analyses, plus
 * velocities, forces and event counts): copy the requested fields (MD_FIELD_*
 * mask) to caller-owned host buffers, in the original atom order.  Synchronises the handle's stream.  After steps
 * enqueued by md_step_async, and without MD_FIELD_X or MD_FIELD_XLIST (which
 * are reordered on the host), the copies and the steps' status are read back
 * together in one host round trip (use pinned buffers for asynchronous
 * copies); if those steps raised a flag (a list that needs more room, an
 * error), md_sync's handling runs first and the fields are copied again.
 * Errors: those of md_sync, INVALID_ARG (a requested buffer is NULL), CUDA. */
md_status md_get_state(md_handle* h, md_state* out, unsigned fields);

/* Overwrite x, v, q, h, plasma counters and/or the step counter (mask;
 * caller-owned host buffers, copied); recomputes the cell list, the plasma
 * scalars of Sec. II.A Eq. 3 and the forces of Eqs. 2, 8 and 11.
 * Checkpoint/resume with md_get_state(MD_FIELD_ALL) continues bit for bit
 * (the paper has no checkpoint; the state is the one Sec. II.A-II.B evolve).
 * Errors: INVALID_ARG (a null buffer for a requested field, charges above Z,
 * non-finite values), BAD_STATE, OOM, CUDA. */
md_status md_set_state(md_handle* h, const md_state* in, unsigned fields);

/* Kinetic and cutoff-shifted potential energy per replica ([n_replicas]
 * each) and the number of in-cutoff pairs at the current state. */
md_status md_get_energies(md_handle* h, double* e_kin, double* e_pot, int64_t* n_pairs);

/* Radial distribution data for the partial structure factors of Sec. II.C
 * (Eq. 18): the number of unordered atom pairs of each species pair (a, b)
 * whose distance r (minimum image in periodic boxes) lies in bin
 * k = floor(r / dr), dr = r_max / n_bins, for r < r_max, at the current
 * positions, summed over replicas.  Each pair is counted once.  The distances
 * are those of the force evaluation: FP32 coordinates relative to the cell
 * centre on the mixed path, FP64 on the FP64 path.  A pair within rounding of
 * a bin edge may fall on either side.  counts: host array
 * [n_species][n_species][n_bins] (caller-owned), filled for a <= b and
 * mirrored.  Errors: INVALID_ARG (r_max not in (0, r_cut], n_bins not in
 * [1, 65536], null counts), BAD_STATE, CUDA. */
md_status md_rdf(md_handle* h, double r_max, int n_bins, int64_t* counts);

/* Partial structure factor of Sec. II.C, Eq. 18, from one species pair's
 * histogram (md_rdf): g_ab at the bin centres r_k is counts_k over the pairs
 * an ideal gas of the same density puts in the shell, n_a n_b / V (or
 * n_a (n_a - 1) / (2V) when same != 0) times (4 pi / 3)(r_{k+1}^3 - r_k^3).
 * Then S_ab(q) = 1 + (4 pi rho0 / q) sum_k dr r_k (g_ab(r_k) - 1) sin(q r_k),
 * with rho0 the total number density.  Host-only; q[n_q] > 0 (nm^-1), out
 * s[n_q].  Errors: INVALID_ARG (bad sizes, null pointers, q <= 0, V <= 0). */
md_status md_structure_factor(const int64_t* counts, int n_bins, double r_max, double n_a, double n_b,
                              int same, double volume, double rho0, const double* q, int n_q, double* s);

/* Fragments of the current state and their ion yields (Sec. III: the
 * fractional ion yields by mass and charge).  Reading: a fragment is a
 * connected component of the graph that joins atoms of one replica closer
 * than r_frag (0 < r_frag <= r_cut; distances as in the force evaluation,
 * FP32 on the mixed path, so a pair within rounding of r_frag may go either
 * way).  label[n_atoms] (original order, caller-owned, may be NULL): the
 * smallest atom index of the atom's fragment.  counts[n_replicas]
 * [mass_max + 1][charge_max + 1] (may be NULL): fragments per replica by mass
 * number (the sum of the atoms' mass numbers, round(md_config.mass)) and net
 * charge (the sum of their charges); larger values go to the last bin.  The
 * fractional yield of a (mass, charge) is its count over the fragments
 * counted.  Errors: INVALID_ARG (r_frag, bin counts, both outputs NULL),
 * BAD_STATE, OOM, CUDA. */
md_status md_fragments(md_handle* h, double r_frag, int mass_max, int charge_max, int32_t* label, int64_t* counts);

/* Probe records (md_config.probe_record = 1; Sec. II.C, Eq. 17): records
 * first .. first + n - 1 of one replica, record k being the state after k
 * steps (record 0: the initial state; a restored checkpoint or a grown list
 * rewrites the record of its step).  Per record and species (row-major
 * [n][n_species], caller-owned, either may be NULL): q_sum = the summed
 * charge of the replica's atoms of that species, exact; d2_sum = their summed
 * squared displacement |x - x0|^2 (nm^2) from the positions md_init was
 * given, minimum image of the replica's box, summed exactly in 2^-40 nm^2
 * fixed point (each atom's value capped at 2^23 nm^2).  Errors: BAD_STATE (records off, handle poisoned),
 * INVALID_ARG (replica, or records beyond the current step), CUDA. */
md_status md_get_probe_series(md_handle* h, int replica, int first, int n, int64_t* q_sum, double* d2_sum);

/* Probe-weighted displacement per species (Sec. II.C, Eq. 17), out[n_species]:
 * sum_k w_k d_k over records first .. first + n - 1, with d_k =
 * sqrt(d2_sum / N_s) the RMS displacement of the species, and
 * w_k = int_{t_k}^{t_k + dt} g f dt / sum over the records, t_k = t_start +
 * k dt, g the probe pulse profile (the pulses' per-step fluence; their
 * fluence cancels), f = 1 - zbar_s / Z_s the fraction of bound electrons,
 * zbar_s = q_sum / N_s constant over a step (charges change at step ends).
 * A species without atoms, or with no weight left (f = 0 throughout), gives
 * 0.  Errors: those of md_get_probe_series, and INVALID_ARG for bad pulses. */
md_status md_probe_displacement(md_handle* h, int replica, int first, int n, const md_pulse* probe, int n_pulses,
                                double* out);

md_status md_get_timing(md_handle* h, md_timing* out);
md_status md_reset_timing(md_handle* h);

/* Last error message of the handle (or, when h is NULL, of the last failed
 * md_init, md_pulse_table, md_philox, md_fma_peak or md_forces_noalloc on
 * this thread). */
const char* md_last_error(const md_handle* h);

/* Release the handle and its device memory.  NULL is a no-op. */
void md_finalize(md_handle* h);

/* Host-only: the per-step fluence table md_set_pulse would upload
 * (out[n_steps]); dt_fs is the timestep in fs.  Needs no GPU. */
md_status md_pulse_table(const md_pulse* p, int n_pulses, double t_start_fs, double dt_fs,
                         int n_steps, double* out);

/* Diagnostic: the device Philox4x32-10 (Salmon et al., SC'11) used by the
 * charge update, out[4i..4i+3] = Philox(d_ctr4[4i..4i+3], key = seed), on
 * device buffers d_ctr4/d_out (n blocks) and the given stream. */
md_status md_philox(uint64_t seed, const uint32_t* d_ctr4, int64_t n, uint32_t* d_out,
                    void* cuda_stream);

/* Measurement: the throughput of the FP32 (precision MD_PREC_MIXED) or FP64
 * (MD_PREC_FP64) fused multiply-add pipe of the current device, the
 * denominator of the force kernel's roofline (the paper has no counterpart).
 * One launch of blocks_per_sm x (SM count) blocks of 256 threads, each thread
 * running 8 independent FMA chains for iters x 16 steps, timed with CUDA
 * events on cuda_stream (synchronous).  *flops_per_s = 2 x FMAs / time
 * (an FMA counts as two operations); *seconds (may be NULL) = the kernel's
 * time.  Errors: INVALID_ARG for iters < 1, blocks_per_sm outside 1..64 or a
 * bad precision; CUDA for a failed launch (message in md_last_error(NULL)). */
md_status md_fma_peak(int precision, int64_t iters, int blocks_per_sm, double* flops_per_s, double* seconds,
                      void* cuda_stream);

/*
 * Allocation-free force evaluation (the paper has no counterpart; this is a
 * convenience of the library).  For callers that cannot allocate device
 * memory -- a plug-in inside a host program that owns the device memory
 * budget, a memory-capped process, an inner loop that must keep the device
 * footprint fixed -- it computes the screened Coulomb + screened LJ forces of
 * one configuration using only a fixed scratch area compiled into the
 * library (a file-scope __device__ array of about 11 MB, held by every GPU
 * that loads the library until the process exits).  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Limits: n_atoms <= MD_NOALLOC_MAX_ATOMS; a periodic box needs at most
 * MD_NOALLOC_MAX_CELLS cells of edge >= r_cut; larger inputs are rejected
 * with MD_ERR_INVALID_ARG (message in md_last_error(NULL)).  The cluster-pair
 * list holds 48 entries per cluster (liquid water at r_cut = 1.2 nm needs
 * about 31); a denser configuration returns MD_ERR_CELL_OVERFLOW.
 * Inputs: device pointers d_x [3n] AoS positions (nm), d_species [n],
 * d_q [n] charges, d_fragment [n] (LJ excluded within a fragment); the screening
 * kappa = 1/lambda_D (nm^-1, 0 = bare Coulomb) and the species tables on the host.
 * Every atom needs species[i] < n_species and q[i] <= z[species[i]]; the
 * device arrays are checked on the device, and an atom that breaks this makes
 * the call return MD_ERR_INVALID_ARG (its forces are then not meaningful).
 * Output: d_f [3n] AoS forces (kJ/mol/nm), device memory owned by the caller.
 * The result equals md_init (same sample, kappa_fixed = kappa, charges
 * frozen) followed by md_get_state(MD_FIELD_F).
 * The first call on a device looks up the scratch area's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  The address is kept for the life of the process; a
 * cudaDeviceReset on that device invalidates it, so do not call this entry
 * point after resetting a device.  All calls share the one scratch area, which keeps the
 * last call's contents: every call resets what must start at zero, and calls
 * that overlap on the GPU (different streams or threads) race -- serialise
 * them.  The call is synchronous with respect to `cuda_stream` (it reads a
 * 4-byte status back).
 */
#define MD_NOALLOC_MAX_ATOMS 16384
#define MD_NOALLOC_MAX_CELLS 4096
typedef struct md_forces_input {
    int n_atoms;
    const double* d_x;
    const uint8_t* d_species;
    const uint8_t* d_q;
    const int32_t* d_fragment;
    double box[3];               /* periodic box (all zero: vacuum)          */
    double kappa;
    double r_cut;
    double coulomb_f;
    int precision;               /* MD_PREC_MIXED or MD_PREC_FP64            */
    int n_species;
    int z[MD_MAX_SPECIES];
    double lj_sigma0[MD_MAX_SPECIES];
    double lj_eps0[MD_MAX_SPECIES];
} md_forces_input;
md_status md_forces_noalloc(const md_forces_input* in, double* d_f, void* cuda_stream);

/* Library version string. */
const char* md_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MD_GB300_H */
