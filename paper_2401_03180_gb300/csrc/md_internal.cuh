// Internal device-side definitions of the GB300 ionising-MD library.
// Not part of the C ABI (include/md.h is).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace mdg {

// Atoms are grouped in clusters of 8 consecutive slots of the cell-sorted
// order; a warp processes one super-cluster of up to K_SC i-clusters against
// one neighbour cell at a time.
constexpr int kClusterSize = 8;
constexpr int kSuperClusters = 8;     // K_SC
constexpr int kHalfShell = 14;        // self cell + 13 neighbour cells
constexpr int kSCAtoms = kSuperClusters * kClusterSize;   // atom slots of a super-cluster
constexpr int kChunk = 8;             // cluster-pair list entries per force work item
constexpr int kListMinPerCluster = 32;   // initial pair-list entries per cluster
constexpr int kMaxSpecies = 8;
constexpr int kMaxTS = 128;
constexpr int kNEtab = 16 * 40;       // e^{-k/16} table, lambda < 40
constexpr int kRepWindow = 8;         // replicas per CTA kept in shared memory
constexpr double kFixScale = 4294967296.0;        // 2^32
constexpr double kFixInv = 1.0 / 4294967296.0;
constexpr double kFixLimit = 4.611686018427388e18;  // 2^62 (overflow guard)
constexpr double kEvKJmol = 96.48533212;          // kJ/mol per eV
constexpr double kLn2 = 0.69314718055994530942;   // ln 2 (scales the LJ table's c12 column)
constexpr double kPi = 3.14159265358979323846;
constexpr int kChargeTable = 1;                  // MD_CHARGE_TABLE
constexpr float kBBoxMargin = 1e-4f;               // nm, slack of the cluster prefilter
constexpr int kScanCtasMax = 1024;                 // CTAs of the multi-CTA scans (cells, super-clusters)

// device error bits (mirrored to md_status by the host)
enum : unsigned {
    ERR_OVERFLOW = 1u,
    ERR_NONFINITE = 2u,
    ERR_CELL = 4u,
    ERR_TABLE_END = 8u,
    ERR_LIST = 16u,             // cluster-pair list capacity exceeded
    ERR_INPUT = 32u,            // a species index or charge out of range in device-side input
};

// Cluster-pair list entry: x = j-cluster, y = half-shell index of the
// j-cluster's cell | kEntryExcl when an i-atom and a j-atom may share a
// fragment, (z, w) = column-major 64-bit mask of the super-cluster's atom
// slots (bit a*8 + k: atom a of i-cluster k) that may interact with the
// j-cluster.
using PairEntry = uint4;
constexpr unsigned kEntryExcl = 0x100u;

struct Grid {                // cell grid of one replica (rebuilt every step)
    double origin[3];        // lower corner (nm)
    double edge[3];          // cell edge per dimension, >= r_cut
    double inv_edge[3];
    double box[3];           // periodic box lengths (0 for vacuum)
    float edge_f[3];
    int dims[3];
    int cell_off;            // first global cell index of the replica
    int cell_cap;            // cells reserved for the replica
    int periodic;
};

// Hybrid ion-sphere / Debye electrostatics of one charge state q at the
// plasma state of a step (Sec. II.A, Eqs. 4-7; reading in include/md.h):
// phi(r) = q/r + c1 - c2 r^2 for r < rp, G e^{-kappa r}/r for r >= rp.
constexpr int kHybQ = 33;    // charge states 0 .. MD_MAX_Z
struct HybQ {
    double G;                // Debye-form amplitude (q g(q)); q when there is no ion sphere
    double rp;               // transition radius r' (nm); 0: no ion sphere
    double c1;               // constant of the ion-sphere form
    double phirc;            // phi(r_cut), the energy shift
    float Gf, rpf, c1f, phircf;
};
struct HybRep {              // per replica
    double c2;               // -2 pi n_e / 3 (the same for every q)
    double rpm2;             // (max r' over the charge states present)^2
    float c2f, rpm2f;
};

// The current cluster-pair list's radius (adaptive Verlet buffer): the step
// kernel decides each rebuild and the radius of the next list; the cell grid,
// the list kernels and the force kernel read it.
// Break-even from the measured costs on the 2 M-atom droplet: a buffered step
// costs the force kernel on the trimmed list plus (build + trimming pass) / L
// for lists of L steps, an unbuffered one the force kernel on the r_cut list
// plus a build; the two meet at L = 3.  Taking the skin back waits for twice
// that, estimated from the one-step displacement (straight-line motion, which
// overestimates the lifetime of accelerating atoms).
constexpr int kAdaptOffLife = 3;   // a buffered list that lived fewer steps: drop the skin
constexpr int kAdaptOnLife = 6;    // unbuffered, and a buffered list would last this long: take it back
struct ListCtl {
    float rlist_f;           // r_cut (+ skin) of the current list
    float half_skin2;        // (skin/2)^2 of the current list; 0: rebuilt every step
    double r_list;
    int buffered;            // 1: the current list carries the skin
    int since_build;         // steps since the last build
    long long unbuffered_builds;
};

struct RepState {            // plasma and bookkeeping of one replica
    long long n_e;           // free electrons
    long long e_gas;         // gas energy, meV
    long long counts[4];     // PI, Auger, CI, REC events so far
    double te_ev;            // T_e used by the rate tables
    double n_dens;           // n_e (nm^-3)
    double kappa;            // 1/lambda_D (nm^-1) from Eq. 3
    double ne_dt;            // n_e * dt
    double wt;               // Te-grid interpolation weight
    int it0;                 // Te-grid interval
    float kappa_f;           // screening used by the pair forces
    double kappa_force;      // same in double
};

struct RepAccum {            // per-step sums of one replica
    long long dNe;
    long long dE;
    long long counts[4];
    unsigned long long bmin[3];  // ordered encodings of doubles
    unsigned long long bmax[3];
};

// Everything a kernel may touch.  Passed by value.
struct Params {
    int n_atoms, n_rep, n_species, n_ts, n_te, max_steps;
    int n_ts_lj;             // type states of the species present (LJ table side)
    int cell_cap_total, slot_cap, cluster_cap, sc_cap;
    int precision, cr_enabled, plasma_mode;
    int screening;           // MD_SCREEN_*
    int langevin;            // 1: electron-ion coupling (some langevin_g > 0)
    int charge_mode;         // MD_CHARGE_*
    int z_max;               // largest nuclear charge of the species present
    double dt, r_cut, rc2, kappa_fixed, te_floor, four_pi_f, coulomb_f, inv_dte;
    float rc2_f, rc_f;
    double r_list;           // r_cut + Verlet skin: cell edge and list cutoff (fixed skin)
    float rlist_f;
    float half_skin2;        // (skin/2)^2; 0: rebuild every step
    ListCtl* lc;             // adaptive skin: the current list's radius (else null: the values above)

    // atoms, original order
    double *x, *y, *z, *vx, *vy, *vz;
    uint8_t *species, *q, *h;
    int *frag, *rep, *local_id, *slot_of, *atom_cell, *atom_rank;

    // species / type-state tables
    const double* hdtm;      // [n_species] 0.5 dt / m
    const float* hdtm_f;     // [n_species] (float)(0.5 dt / m 2^-32): the mixed path's half kick per fixed-point unit
    const double* mass;      // [n_species]
    const int* zs;           // [n_species]
    const int* ts_off;       // [n_species + 1]
    const int* lj_ts_off;    // [n_species] LJ table row of (species, q = 0)
    const double* auger_dt;  // [n_species]
    const double* sigma_pi;  // [n_ts][2]
    const double* k_ci;      // [n_ts][n_te]
    const double* k_rec;     // [n_ts][n_te]
    const long long* ip_mev;     // [n_ts]
    const long long* e_pi_mev;   // [n_ts][2]
    const long long* e_auger_mev;// [n_species]
    const double* etab;      // [kNEtab]
    const double* inv12;     // [13] 1/m
    const float2* lj_f;      // [n_ts_lj][n_ts_lj] (-6 c6, -ln2 c12)
    const double2* lj_d;     // [n_ts_lj][n_ts_lj] (-6 c6, -ln2 c12)

    // replicas
    Grid* grid;              // grid for the next cell build (step kernel output)
    Grid* grid_b;            // grid of the last build (list, forces, refresh); may alias grid
    RepState* rs;
    RepAccum* acc;
    HybQ* hq;                // [n_rep][kHybQ] (hybrid screening only, else null)
    HybRep* hrep;            // [n_rep]
    const double* lgv_g;     // [n_species] electron-ion coupling (nm^3/ps)
    double2* lgv;            // [n_rep][kMaxSpecies] (c, sigma) of the Langevin update of the next step
    double* qcum;            // [n_rep][max_steps + 1][n_ts] running sums of the charge-state fractions
    const unsigned long long* seed;
    const double* dF;        // [n_rep][max_steps]
    const double* pres_ne;   // [n_rep][max_steps + 1]
    const double* pres_te;
    const double* volume;
    const int* rep_off;      // [n_rep + 1]

    // cell list
    int* cell_count;         // [cell_cap_total]
    int* cell_start;         // [cell_cap_total + 1] unpadded
    int* cell_pstart;        // [cell_cap_total + 1] padded (multiples of 8)
    unsigned long long* tmp_key;  // [n_atoms] (sub-cell key << 32 | atom)
    int* sc_cell;            // [sc_cap]
    int* sc_first;           // [sc_cap] first cluster
    int* sc_ncl;             // [sc_cap] clusters in the super-cluster
    int* counters;           // [0] n_sc, [1] n_slots, [2] work, [3] ticket, [4] big cells, [6] list entries, [7] chunks
    int* big_cells;          // [cell_cap_total] cells too large for the one-warp sort (counters[4] of them)
    int* list_cnt;           // [sc_cap * kHalfShell] entries of each super-cluster in each half-shell cell
    int* sc_tot;             // [sc_cap] entries per super-cluster
    int* sc_eoff;            // [sc_cap] first entry of each super-cluster
    int* sc_coff;            // [sc_cap] first chunk of each super-cluster
    int* scan_tmp;           // [kScanCtasMax * 3] per-CTA sums and bases of the multi-CTA scans
    PairEntry* pl;           // [pl_cap] cluster-pair list (j-cluster, half-shell index, i-atom mask)
    int4* pl_chunk;          // [chunk_cap] (SC, first entry, entries, replica)
    int pl_cap, chunk_cap;

    // packed, cell-sorted arrays (slot order)
    float4* xq;              // (x, y, z) relative to the cell centre, q
    double4_32a* xq64;
    int2* tf;                // (type state, fragment)
    int* atom_of;            // slot -> atom (-1: padding)
    double4_32a* cl_cen;     // per cluster: centre of its cell at the build (x, y, z, -)
    double *xr, *yr, *zr;    // positions at the last build (Verlet skin only, else null)
    unsigned* maxd2;         // max over atoms of |x - x_build|^2 this step (float bits)
    int* builds;             // [0] list builds by the step graph, [1] last step rebuilt
    cudaGraphConditionalHandle cond;   // IF node of the step graph (Verlet skin only)
    float4* bb_lo;           // per cluster, relative to its cell centre
    float4* bb_hi;
    int2* bb_frag;           // min/max fragment of the cluster
    long long *fx, *fy, *fz, *epot;   // fixed-point sums per slot

    // bonded terms of the native structure (Sec. II.B, Eqs. 9-10); none when both counts are 0
    int n_bonds, n_angles;
    const int4* bonds;       // [n_bonds] (i, j, type, 0), atoms in original order
    const int4* angles;      // [n_angles] (i, j = vertex, k, type)
    const double* bond_pd;   // [bond types][3] D_e, b_e, beta
    const double* angle_pd;  // [angle types][2] k_theta, theta_0
    const float* bond_pf;    // FP32 copies of the two tables
    const float* angle_pf;

    // probe records (Sec. II.C, Eq. 17); null when off
    const double *x0, *y0, *z0;   // initial positions, original order
    long long* probe;        // [n_rep][max_steps + 1][n_species][3]: sum q; sum |x - x0|^2 in 2^-40 nm^2, high and low 32 bits
    long long* pair_count;   // in-cutoff pairs (energy pass)

    // run state
    unsigned* err;
    long long* step;
    int* kick_full;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ordered_bits(double v)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered(unsigned long long u)
{
    u = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
    return __longlong_as_double((long long)u);
}
__host__ __device__ __forceinline__ unsigned long long ordered_bits_host(double v)
{
    union { double d; unsigned long long u; } c;
    c.d = v;
    unsigned long long u = c.u;
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// Comparisons of doubles on their bit patterns, in the integer pipe (FP64
// issues at 2 lanes per SM per clock on GB300).  For non-NaN operands they
// give exactly the FP64 comparisons; -0.0 counts as zero.
//
// beyond_half(d, L), L > 0 normal: +1 when d > L/2, -1 when d < -L/2, else 0.
__device__ __forceinline__ int beyond_half(double d, double L)
{
    const long long b = __double_as_longlong(d);
    const long long half = __double_as_longlong(L) - (1ll << 52);   // bits of L/2
    if ((b & 0x7fffffffffffffffll) <= half) return 0;
    return b < 0 ? -1 : 1;
}
// x < 0 (x not -0.0) and x >= L for L > 0.
__device__ __forceinline__ bool below_zero(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool at_or_above(double x, double L)
{
    return __double_as_longlong(x) >= __double_as_longlong(L);
}

// The 13 half-shell neighbour offsets plus the cell itself (index 0).
__host__ __device__ __forceinline__ void half_shell(int nb, int& dx, int& dy, int& dz)
{
    // enumerate (dx,dy,dz) with dz>0, or dz==0 && dy>0, or dz==dy==0 && dx>0
    if (nb == 0) { dx = dy = dz = 0; return; }
    int k = nb - 1;               // 0..12
    if (k < 1) { dx = 1; dy = 0; dz = 0; return; }
    k -= 1;                       // 0..11
    if (k < 3) { dx = k - 1; dy = 1; dz = 0; return; }
    k -= 3;                       // 0..8
    dx = k % 3 - 1; dy = k / 3 - 1; dz = 1;
}

// Packed record of atom i in a slot of the cell centred at cen: coordinates
// relative to the centre (minimum image when periodic: between list builds an
// atom may have been wrapped across the box), charge, LJ type state, fragment;
// the slot's force sums are cleared.  Used by the build and by the refresh
// between builds, so both round identically.  Returns the relative position
// rounded to FP32 (the precision of the cluster bounding boxes).
__device__ __forceinline__ float4 pack_record(const Params& p, int slot, const double xi[3], const double cen[3],
                                              int periodic, const double box[3], int sp, int qi, int fr)
{
    double d[3] = {xi[0] - cen[0], xi[1] - cen[1], xi[2] - cen[2]};
    if (periodic)
        for (int k = 0; k < 3; ++k) {
            const int o = beyond_half(d[k], box[k]);
            if (o > 0) d[k] -= box[k];
            else if (o < 0) d[k] += box[k];
        }
    if (p.precision == 0) p.xq[slot] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)qi);
    else p.xq64[slot] = make_double4_32a(d[0], d[1], d[2], (double)qi);
    p.tf[slot] = make_int2(p.lj_ts_off[sp] + qi, fr);
    p.fx[slot] = 0; p.fy[slot] = 0; p.fz[slot] = 0; p.epot[slot] = 0;
    return make_float4((float)d[0], (float)d[1], (float)d[2], 0.0f);
}
__device__ __forceinline__ float4 pack_slot(const Params& p, int slot, int i, const double cen[3], const Grid& g)
{
    const double xi[3] = {p.x[i], p.y[i], p.z[i]};
    return pack_record(p, slot, xi, cen, g.periodic, g.box, p.species[i], p.q[i], p.frag[i]);
}

// Radius and half skin of the current list (adaptive or fixed).
__device__ __forceinline__ float list_rlist_f(const Params& p) { return p.lc ? p.lc->rlist_f : p.rlist_f; }
__device__ __forceinline__ double list_rlist(const Params& p) { return p.lc ? p.lc->r_list : p.r_list; }
__device__ __forceinline__ float list_half_skin2(const Params& p) { return p.lc ? p.lc->half_skin2 : p.half_skin2; }

// Launch helpers implemented in the .cu files.
void launch_step_a(const Params& p, int mode, cudaStream_t s, int grid_atoms);
// launch_cells and launch_pair_list return the number of kernels they launched
int launch_cells(const Params& p, cudaStream_t s, int grid_atoms, int grid_cells, int sort_threads);
int launch_pair_list(const Params& p, cudaStream_t s, int blocks);
void launch_pair_forces(const Params& p, cudaStream_t s, bool energy, int blocks, int warps);
void launch_velocity_out(const Params& p, double* d_v_out, cudaStream_t s);
void launch_energy(const Params& p, double* d_ekin, long long* d_epot, cudaStream_t s);
void launch_philox(unsigned long long seed, const uint32_t* ctr, long long n, uint32_t* out,
                   cudaStream_t s);
void launch_force_out(const Params& p, double* d_f_out, cudaStream_t s);
void launch_refresh(const Params& p, cudaStream_t s);
void launch_rdf(const Params& p, cudaStream_t s, int blocks, int n_bins, double r_max, unsigned long long* hist);
void launch_probe(const Params& p, cudaStream_t s, bool rewrite);
void launch_frag_link(const Params& p, cudaStream_t s, int blocks, double r_frag, int* parent);
void launch_frag_init(const Params& p, cudaStream_t s, int* parent, int* mass, int* charge);
void launch_frag_count(const Params& p, cudaStream_t s, const int* parent, int* label, int* mass, int* charge,
                       const int* mass_number, int mass_max, int charge_max, unsigned long long* counts);
int pair_max_blocks_per_sm(bool fp64, bool energy, bool hyb, int warps, int n_ts);
// message returned by md_last_error(NULL) (host side)
void set_global_error(const std::string& msg);

// modes of launch_step_a
enum : int {
    STEP_KICK_DRIFT = 1,     // velocity kick + position drift
    STEP_CR = 2,             // collisional-radiative charge update
    STEP_ADVANCE = 4,        // bump the step counter at the end
    STEP_SETCOND = 8,        // decide the rebuild and set the graph condition
};

}  // namespace mdg
