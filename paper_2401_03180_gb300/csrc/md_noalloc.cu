// md_forces_noalloc: a force evaluation that allocates no memory.
//
// Some callers cannot allocate device memory: a plug-in running inside a
// host program that owns the whole device memory budget through its own
// pool, a process whose memory is capped so that a new cudaMalloc would fail
// or would have to wait for the pool to shrink, or an inner loop of another
// code that must not change the device footprint between its own steps.  This
// entry point serves them: all the scratch it needs (cell list, packed
// coordinates, fixed-point force sums, grid and screening bookkeeping) lives
// in one file-scope __device__ array of a fixed, modest size
// (MD_NOALLOC_MAX_ATOMS atoms, MD_NOALLOC_MAX_CELLS cells; about 11 MB) that
// every GPU loading the library holds until the process exits.  The caller
// passes inputs and the output buffer; nothing is allocated.
//
// It runs the same kernels as a handle's initial force evaluation (cell
// build, pair forces, read-out), so its forces equal those of md_init +
// md_get_state(MD_FIELD_F) on the same input.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "md.h"
#include "md_internal.cuh"

using namespace mdg;

namespace {

constexpr int kNaMax = MD_NOALLOC_MAX_ATOMS;
constexpr int kNcMax = MD_NOALLOC_MAX_CELLS;
constexpr int kSlotCap = kNaMax + 7 * kNcMax + 8;
constexpr int kClusterCap = kSlotCap / kClusterSize + 1;
constexpr int kPlCap = 48 * kClusterCap;                  // cluster-pair list entries
constexpr int kChunkCap = kClusterCap + kPlCap / kChunk + 1;
constexpr int kTabMax = MD_MAX_TYPE_STATES * MD_MAX_TYPE_STATES;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Scratch layout (byte offsets), fixed at compile time.
struct Layout {
    size_t x, y, z, vx, vy, vz, species, q, h, frag, rep, local_id, slot_of, atom_cell, atom_rank;
    size_t zs, ts_off, hdtm, mass, auger, volume, rep_off, lj;
    size_t grid, rs, acc, cell_count, cell_start, cell_pstart, tmp_key, sc_cell, sc_first, sc_ncl;
    size_t counters, list_cnt, sc_tot, sc_eoff, sc_coff, scan_tmp, big_cells, xq, tf, atom_of, bb_lo, bb_hi, bb_frag, fx, fy, fz, epot, pair_count, err, step, kick;
    size_t pl, pl_chunk, cl_cen;
    size_t total;
};

constexpr Layout make_layout()
{
    Layout L{};
    size_t o = 0;
    auto take = [&o](size_t bytes) { const size_t at = o; o += align256(bytes); return at; };
    L.x = take(8 * kNaMax); L.y = take(8 * kNaMax); L.z = take(8 * kNaMax);
    L.vx = take(8 * kNaMax); L.vy = take(8 * kNaMax); L.vz = take(8 * kNaMax);
    L.species = take(kNaMax); L.q = take(kNaMax); L.h = take(kNaMax);
    L.frag = take(4 * kNaMax); L.rep = take(4 * kNaMax); L.local_id = take(4 * kNaMax);
    L.slot_of = take(4 * kNaMax); L.atom_cell = take(4 * kNaMax); L.atom_rank = take(4 * kNaMax);
    L.zs = take(4 * kMaxSpecies); L.ts_off = take(4 * (kMaxSpecies + 1));
    L.hdtm = take(8 * kMaxSpecies); L.mass = take(8 * kMaxSpecies); L.auger = take(8 * kMaxSpecies);
    L.volume = take(8); L.rep_off = take(8);
    L.lj = take(16 * (size_t)kTabMax);                       // float2 or double2 entries
    L.grid = take(sizeof(Grid)); L.rs = take(sizeof(RepState)); L.acc = take(16 * sizeof(RepAccum));
    L.cell_count = take(4 * kNcMax); L.cell_start = take(4 * (kNcMax + 1)); L.cell_pstart = take(4 * (kNcMax + 1));
    L.tmp_key = take(8 * kNaMax);
    L.sc_cell = take(4 * kClusterCap); L.sc_first = take(4 * kClusterCap); L.sc_ncl = take(4 * kClusterCap);
    L.counters = take(4 * 8);
    L.list_cnt = take(4 * (size_t)kClusterCap * kHalfShell);
    L.sc_tot = take(4 * kClusterCap);
    L.sc_eoff = take(4 * kClusterCap); L.sc_coff = take(4 * kClusterCap);
    L.scan_tmp = take(4 * 3 * kScanCtasMax);
    L.big_cells = take(4 * kNcMax);
    L.xq = take(32 * (size_t)kSlotCap);                      // float4 or double4_32a
    L.tf = take(8 * (size_t)kSlotCap); L.atom_of = take(4 * (size_t)kSlotCap);
    L.bb_lo = take(16 * (size_t)kClusterCap); L.bb_hi = take(16 * (size_t)kClusterCap);
    L.bb_frag = take(8 * (size_t)kClusterCap);
    L.fx = take(8 * (size_t)kSlotCap); L.fy = take(8 * (size_t)kSlotCap); L.fz = take(8 * (size_t)kSlotCap);
    L.epot = take(8 * (size_t)kSlotCap);
    L.pair_count = take(8); L.err = take(4); L.step = take(8); L.kick = take(4);
    L.pl = take(sizeof(PairEntry) * (size_t)kPlCap); L.pl_chunk = take(16 * (size_t)kChunkCap);
    L.cl_cen = take(32 * (size_t)kClusterCap);
    L.total = o;
    return L;
}

constexpr Layout kL = make_layout();

// The scratch array itself.  In host code `g_md_scratch` names a host-side
// stand-in, not device memory: its device address is obtained once per device
// with cudaGetSymbolAddress and passed to the kernels.
__device__ __align__(256) unsigned char g_md_scratch[kL.total];

unsigned char* g_base[64] = {nullptr};   // device address of the scratch, per device

md_status fail(md_status s, const std::string& m)
{
    set_global_error(m);   // read back through md_last_error(NULL)
    return s;
}

// Reset of the per-call state and the copy of the caller's atoms into the
// scratch layout (structure-of-arrays, one replica).  The species and charge
// arrays live on the device, so they are checked here: an atom whose species
// index is not below n_species or whose charge exceeds its species' Z raises
// ERR_INPUT (the call then returns MD_ERR_INVALID_ARG) and is stored as a
// neutral atom of species 0, so that every later table lookup stays in bounds.
// The error word is cleared on the stream before this kernel runs.
__global__ void k_noalloc_prepare(Params p, const double* __restrict__ x, const uint8_t* __restrict__ sp,
                                  const uint8_t* __restrict__ q, const int32_t* __restrict__ fr, int slot_cap,
                                  int cell_cap)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = p.n_atoms;
    if (t < n) {
        p.x[t] = x[3 * t + 0];
        p.y[t] = x[3 * t + 1];
        p.z[t] = x[3 * t + 2];
        p.vx[t] = 0.0; p.vy[t] = 0.0; p.vz[t] = 0.0;
        int st = sp[t], qt = q[t];
        if (st >= p.n_species || qt > p.zs[st]) {
            atomicOr(p.err, ERR_INPUT);
            st = 0;
            qt = 0;
        }
        p.species[t] = (uint8_t)st;
        p.q[t] = (uint8_t)qt;
        p.h[t] = 0;
        p.frag[t] = fr[t];
        p.rep[t] = 0;
        p.local_id[t] = t;
        p.slot_of[t] = 0;
    }
    if (t < slot_cap) {
        p.atom_of[t] = t < n ? t : -1;     // the first cell assignment walks atoms in input order
        p.fx[t] = 0; p.fy[t] = 0; p.fz[t] = 0; p.epot[t] = 0;
    }
    if (t < cell_cap) p.cell_count[t] = 0;
    if (t < 16) {
        RepAccum& a = p.acc[t];
        a.dNe = 0; a.dE = 0;
        for (int k = 0; k < 4; ++k) a.counts[k] = 0;
        for (int d = 0; d < 3; ++d) { a.bmin[d] = ~0ull; a.bmax[d] = 0ull; }
    }
    if (t == 0) {
        for (int k = 0; k < 8; ++k) p.counters[k] = 0;
        p.counters[1] = n;
        *p.step = 0;
        *p.kick_full = 0;
        *p.pair_count = 0;
        RepState st{};
        p.rs[0] = st;
    }
}

}  // namespace

extern "C" md_status md_forces_noalloc(const md_forces_input* in, double* d_f, void* stream_ptr)
{
    const cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    if (!in || !d_f) return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: null input or output");
    const int n = in->n_atoms;
    if (n < 1 || n > kNaMax)
        return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: n_atoms must be in [1, " + std::to_string(kNaMax) + "]");
    if (!in->d_x || !in->d_species || !in->d_q || !in->d_fragment)
        return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: device input arrays missing");
    if (!(in->r_cut > 0) || !(in->kappa >= 0) || !(in->coulomb_f > 0))
        return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: r_cut, coulomb_f must be > 0 and kappa >= 0");
    if (in->precision != MD_PREC_MIXED && in->precision != MD_PREC_FP64)
        return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: bad precision");
    if (in->n_species < 1 || in->n_species > MD_MAX_SPECIES)
        return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: n_species out of range");
    int ts_off[MD_MAX_SPECIES + 1] = {0};
    for (int k = 0; k < in->n_species; ++k) {
        if (in->z[k] < 1 || in->z[k] > MD_MAX_Z) return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: Z out of range");
        ts_off[k + 1] = ts_off[k] + in->z[k] + 1;
    }
    const int nts = ts_off[in->n_species];
    if (nts > MD_MAX_TYPE_STATES) return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: too many type states");
    Grid g{};
    const bool periodic = in->box[0] > 0 || in->box[1] > 0 || in->box[2] > 0;
    g.periodic = periodic ? 1 : 0;
    g.cell_off = 0;
    if (periodic) {
        long long prod = 1;
        for (int d = 0; d < 3; ++d) {
            if (!(in->box[d] >= 3.0 * in->r_cut))
                return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: periodic box edges must be >= 3 r_cut");
            const int m = std::max(3, std::min((int)std::floor(in->box[d] / in->r_cut), 1024));
            g.dims[d] = m; g.edge[d] = in->box[d] / m; g.inv_edge[d] = 1.0 / g.edge[d];
            g.edge_f[d] = (float)g.edge[d]; g.box[d] = in->box[d]; g.origin[d] = 0.0;
            prod *= m;
        }
        if (prod > kNcMax)
            return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: box needs more than " + std::to_string(kNcMax) + " cells");
        g.cell_cap = (int)prod;
    } else {
        for (int d = 0; d < 3; ++d) {
            g.dims[d] = 1; g.edge[d] = in->r_cut; g.inv_edge[d] = 1.0 / in->r_cut;
            g.edge_f[d] = (float)in->r_cut; g.box[d] = 0.0; g.origin[d] = 0.0;
        }
        g.cell_cap = kNcMax;
    }

    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail(MD_ERR_CUDA, "md_forces_noalloc: no usable current device");
    if (!g_base[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_md_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(MD_ERR_CUDA, std::string("md_forces_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_base[dev] = static_cast<unsigned char*>(ptr);
    }
    unsigned char* B = g_base[dev];

    Params P{};
    P.n_atoms = n; P.n_rep = 1; P.n_species = in->n_species; P.n_ts = nts; P.n_ts_lj = nts; P.n_te = 2; P.max_steps = 1;
    P.cell_cap_total = g.cell_cap;
    P.slot_cap = n + 7 * g.cell_cap + 8;
    P.cluster_cap = P.slot_cap / kClusterSize + 1;
    P.sc_cap = P.cluster_cap;
    P.precision = in->precision; P.cr_enabled = 0; P.plasma_mode = 0;
    P.dt = 0.0; P.r_cut = in->r_cut; P.rc2 = in->r_cut * in->r_cut; P.kappa_fixed = in->kappa;
    P.te_floor = 1.0; P.coulomb_f = in->coulomb_f; P.four_pi_f = 4.0 * M_PI * in->coulomb_f; P.inv_dte = 1.0;
    P.rc_f = (float)in->r_cut; P.rc2_f = P.rc_f * P.rc_f;
    P.r_list = in->r_cut; P.rlist_f = P.rc_f; P.half_skin2 = 0.0f;
    P.x = (double*)(B + kL.x); P.y = (double*)(B + kL.y); P.z = (double*)(B + kL.z);
    P.vx = (double*)(B + kL.vx); P.vy = (double*)(B + kL.vy); P.vz = (double*)(B + kL.vz);
    P.species = B + kL.species; P.q = B + kL.q; P.h = B + kL.h;
    P.frag = (int*)(B + kL.frag); P.rep = (int*)(B + kL.rep); P.local_id = (int*)(B + kL.local_id);
    P.slot_of = (int*)(B + kL.slot_of); P.atom_cell = (int*)(B + kL.atom_cell); P.atom_rank = (int*)(B + kL.atom_rank);
    P.zs = (const int*)(B + kL.zs); P.ts_off = (const int*)(B + kL.ts_off); P.lj_ts_off = P.ts_off;
    P.hdtm = (const double*)(B + kL.hdtm); P.mass = (const double*)(B + kL.mass);
    P.auger_dt = (const double*)(B + kL.auger); P.volume = (const double*)(B + kL.volume);
    P.rep_off = (const int*)(B + kL.rep_off);
    P.lj_f = (const float2*)(B + kL.lj); P.lj_d = (const double2*)(B + kL.lj);
    P.grid = (Grid*)(B + kL.grid); P.rs = (RepState*)(B + kL.rs); P.acc = (RepAccum*)(B + kL.acc);
    P.cell_count = (int*)(B + kL.cell_count); P.cell_start = (int*)(B + kL.cell_start);
    P.cell_pstart = (int*)(B + kL.cell_pstart); P.tmp_key = (unsigned long long*)(B + kL.tmp_key);
    P.sc_cell = (int*)(B + kL.sc_cell); P.sc_first = (int*)(B + kL.sc_first); P.sc_ncl = (int*)(B + kL.sc_ncl);
    P.counters = (int*)(B + kL.counters);
    P.list_cnt = (int*)(B + kL.list_cnt); P.sc_tot = (int*)(B + kL.sc_tot);
    P.sc_eoff = (int*)(B + kL.sc_eoff); P.sc_coff = (int*)(B + kL.sc_coff);
    P.scan_tmp = (int*)(B + kL.scan_tmp);
    P.big_cells = (int*)(B + kL.big_cells);
    P.xq = (float4*)(B + kL.xq); P.xq64 = (double4_32a*)(B + kL.xq);
    P.tf = (int2*)(B + kL.tf); P.atom_of = (int*)(B + kL.atom_of);
    P.bb_lo = (float4*)(B + kL.bb_lo); P.bb_hi = (float4*)(B + kL.bb_hi); P.bb_frag = (int2*)(B + kL.bb_frag);
    P.fx = (long long*)(B + kL.fx); P.fy = (long long*)(B + kL.fy); P.fz = (long long*)(B + kL.fz);
    P.epot = (long long*)(B + kL.epot); P.pair_count = (long long*)(B + kL.pair_count);
    P.err = (unsigned*)(B + kL.err); P.step = (long long*)(B + kL.step); P.kick_full = (int*)(B + kL.kick);
    P.pl = (PairEntry*)(B + kL.pl); P.pl_chunk = (int4*)(B + kL.pl_chunk);
    P.pl_cap = kPlCap; P.chunk_cap = kChunkCap;
    P.cl_cen = (double4_32a*)(B + kL.cl_cen);
    P.grid_b = P.grid;                 // one build: the build grid is the grid
    P.xr = P.yr = P.zr = nullptr;
    P.maxd2 = nullptr; P.builds = nullptr; P.cond = 0;

    // host-built tables: LJ per pair of type states (sigma scaled by 1 - q/Z,
    // arithmetic-mean sigma, geometric-mean epsilon), offsets, the grid
    std::vector<double> sig(nts), eps(nts);
    for (int k = 0; k < in->n_species; ++k)
        for (int qq = 0; qq <= in->z[k]; ++qq) {
            sig[ts_off[k] + qq] = in->lj_sigma0[k] * (1.0 - (double)qq / (double)in->z[k]);
            eps[ts_off[k] + qq] = in->lj_eps0[k];
        }
    std::vector<double2> tab_d((size_t)nts * nts);
    std::vector<float2> tab_f((size_t)nts * nts);
    for (int a = 0; a < nts; ++a)
        for (int b = 0; b < nts; ++b) {
            const double sg = 0.5 * (sig[a] + sig[b]);
            const double ep = std::sqrt(eps[a] * eps[b]);
            const double s6 = sg * sg * sg * sg * sg * sg;
            const double c6 = 4.0 * ep * s6, c12 = c6 * s6;
            tab_d[(size_t)a * nts + b] = make_double2(-6.0 * c6, -kLn2 * c12);   // pair kernels take (-6 c6, -ln2 c12)
            tab_f[(size_t)a * nts + b] = make_float2((float)(-6.0 * c6), (float)(-kLn2 * c12));
        }
    const int zs[MD_MAX_SPECIES] = {in->z[0], in->z[1], in->z[2], in->z[3], in->z[4], in->z[5], in->z[6], in->z[7]};
    const double one = 1.0;
    const int rep_off[2] = {0, n};
#define NA_CU(call)                                                                                 \
    do {                                                                                            \
        const cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    if (in->precision == MD_PREC_MIXED)
        NA_CU(cudaMemcpyAsync(B + kL.lj, tab_f.data(), tab_f.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    else
        NA_CU(cudaMemcpyAsync(B + kL.lj, tab_d.data(), tab_d.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(B + kL.zs, zs, sizeof(zs), cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(B + kL.ts_off, ts_off, sizeof(ts_off), cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(B + kL.volume, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(B + kL.rep_off, rep_off, sizeof(rep_off), cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(B + kL.grid, &g, sizeof(Grid), cudaMemcpyHostToDevice, s));

    NA_CU(cudaMemsetAsync(P.err, 0, sizeof(unsigned), s));
    const int span = std::max(P.slot_cap, std::max(n, g.cell_cap));
    k_noalloc_prepare<<<(span + 255) / 256, 256, 0, s>>>(P, in->d_x, in->d_species, in->d_q, in->d_fragment,
                                                          P.slot_cap, g.cell_cap);
    int n_sm = 0;
    NA_CU(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int warps = 8;
    const int blocks = n_sm * pair_max_blocks_per_sm(in->precision == MD_PREC_FP64, false, false, warps, nts);
    launch_step_a(P, 0, s, (n + 255) / 256);                           // grid and screening
    launch_cells(P, s, (n + 255) / 256, std::max(1, std::min(g.cell_cap, n_sm * 8)), 1024);
    launch_pair_list(P, s, std::max(1, std::min((P.sc_cap + 7) / 8, 8 * n_sm)));
    launch_pair_forces(P, s, false, blocks, warps);
    launch_force_out(P, d_f, s);
    NA_CU(cudaGetLastError());
    unsigned h_err = 0;
    NA_CU(cudaMemcpyAsync(&h_err, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
#undef NA_CU
    if (h_err & ERR_INPUT)
        return fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: a species index >= n_species or a charge > Z in the device input");
    if (h_err & ERR_OVERFLOW) return fail(MD_ERR_FIXED_OVERFLOW, "force beyond the 64-bit fixed-point range");
    if (h_err & ERR_NONFINITE) return fail(MD_ERR_NONFINITE, "non-finite input position");
    if (h_err & ERR_CELL) return fail(MD_ERR_CELL_OVERFLOW, "cell-list capacity exceeded");
    if (h_err & ERR_LIST) return fail(MD_ERR_CELL_OVERFLOW, "cluster-pair list capacity exceeded");
    if (h_err) return fail(MD_ERR_CUDA, "unexpected device error flag");
    return MD_OK;
}
