// Host side of the C ABI (include/md.h): validation, host-built tables,
// device memory, the per-step CUDA graph, state exchange and diagnostics.
// Compiled with -ffp-contract=off: the pulse table feeds the charge update,
// which must match the CPU oracle bit for bit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "md.h"
#include "md_internal.cuh"

using namespace mdg;

struct md_handle {
    md_config cfg{};
    std::string err;
    int N = 0, R = 0, NS = 0, NTS = 0, NTS_LJ = 0, NTE = 0;
    int n_sm = 0;
    std::vector<int> z, ts_off, lj_ts_off, rep_off;
    std::vector<Grid> grid0;
    Params P{};
    std::vector<void*> allocs;
    cudaStream_t stream = nullptr;       // caller's stream (NULL = legacy default)
    cudaStream_t cap_stream = nullptr;   // private stream used for graph capture
    cudaStream_t body_stream = nullptr;  // captures the bodies of the rebuild IF node
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec_multi = nullptr;   // kMultiSteps consecutive steps in one graph (not in profile mode)
    cudaEvent_t ev_pair0 = nullptr, ev_pair1 = nullptr;   // captured into the graph
    cudaGraph_t graph = nullptr;                          // kept for event-node updates
    cudaGraphNode_t node_ev0 = nullptr, node_ev1 = nullptr;
    std::vector<cudaEvent_t> prof_pool;                   // [2 * kProfPool] pair-kernel events
    int prof_next = 0;                                    // pairs in flight
    long long list_grows = 0;
    int grid_atoms = 1, grid_cells = 1, sort_threads = 1024;
    int pair_blocks = 1, pair_warps = 8, list_blocks = 1, list_bps = 8;
    int build_kernels = 0;               // kernels of one cell + list build in the step graph
    long long host_step = 0;             // steps enqueued
    long long pending = 0;               // enqueued steps whose status is not read yet
    bool poisoned = false;
    unsigned* h_err = nullptr;           // pinned
    RepState* h_rs = nullptr;            // pinned [R] copy of the replicas' state (md_get_state)
    double pair_ms = 0.0;
    long long pair_launches = 0, steps = 0, last_pairs = 0;
    double* d_scratch = nullptr;         // [3N] doubles for state exchange
    double* d_ekin = nullptr;
    long long* d_epot = nullptr;
    std::vector<long long> n_of_species;   // [R][NS] atoms per replica and species
};

namespace {

constexpr int kProfPool = 256;   // pair-kernel event pairs in flight (profile mode)
constexpr int kMultiSteps = 8;   // steps per launch of the multi-step graph

thread_local std::string g_init_error;

md_status fail(md_handle* h, md_status s, const std::string& msg)
{
    if (h) h->err = msg;
    else g_init_error = msg;
    return s;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(h, MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
md_status dalloc(md_handle* h, T** p, size_t count)
{
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    bytes = (bytes + 255) / 256 * 256;
    void* ptr = nullptr;
    if (h->cfg.dev_alloc) {
        ptr = h->cfg.dev_alloc(bytes, h->cfg.alloc_ctx);
        if (!ptr) return fail(h, MD_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    } else {
        cudaError_t e = cudaMalloc(&ptr, bytes);
        if (e != cudaSuccess)
            return fail(h, MD_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    h->allocs.push_back(ptr);
    *p = static_cast<T*>(ptr);
    return MD_OK;
}

#define DALLOC(ptr, n)                               \
    do {                                             \
        md_status s_ = dalloc(h, &(ptr), (size_t)(n)); \
        if (s_ != MD_OK) return s_;                  \
    } while (0)

// Per-step fluence of a list of pulses (photons/nm^2 in [t_n, t_{n+1}]).
void pulse_table_host(const md_pulse* pulses, int n_pulses, double t_start_fs, double dt_fs,
                      int n_steps, double* out)
{
    for (int n = 0; n < n_steps; ++n) {
        double ta = t_start_fs + (double)n * dt_fs;
        double tb = t_start_fs + (double)(n + 1) * dt_fs;
        double acc = 0.0;
        for (int k = 0; k < n_pulses; ++k) {
            const md_pulse& P = pulses[k];
            double fwhm = P.fwhm_fs, flu = P.fluence_ph_um2 * 1e-6, t0 = P.t_center_fs;
            double frac;
            if (P.shape == MD_PULSE_GAUSSIAN) {
                // normal CDF difference, sigma_t = FWHM / (2 sqrt(2 ln 2)); erfc taken on the
                // side of the centre where it does not cancel
                double sig = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
                double s = sig * std::sqrt(2.0);
                double za = (ta - t0) / s, zb = (tb - t0) / s;
                if (za >= 0.0) frac = 0.5 * (std::erfc(za) - std::erfc(zb));
                else if (zb <= 0.0) frac = 0.5 * (std::erfc(-zb) - std::erfc(-za));
                else frac = 1.0 - 0.5 * (std::erfc(-za) + std::erfc(zb));
            } else {
                double lo = t0 - 0.5 * fwhm, hi = t0 + 0.5 * fwhm;
                double a = ta > lo ? ta : lo;
                double b = tb < hi ? tb : hi;
                frac = b > a ? (b - a) / fwhm : 0.0;
            }
            acc = acc + flu * frac;
        }
        out[n] = acc;
    }
}

// The status of device error flags already read (nonzero flags poison the handle).
md_status flags_status(md_handle* h, unsigned e)
{
    if (!e) return MD_OK;
    h->poisoned = true;
    if (e & ERR_NONFINITE) return fail(h, MD_ERR_NONFINITE, "non-finite position or velocity");
    if (e & ERR_OVERFLOW) return fail(h, MD_ERR_FIXED_OVERFLOW, "force or energy beyond the 64-bit fixed-point range");
    if (e & ERR_CELL) return fail(h, MD_ERR_CELL_OVERFLOW, "cell-list capacity exceeded");
    if (e & ERR_TABLE_END) return fail(h, MD_ERR_TABLE_END, "stepped past the pulse table");
    return fail(h, MD_ERR_CUDA, "unknown device error flag");
}

md_status check_device_flags(md_handle* h)
{
    CU(cudaMemcpyAsync(h->h_err, h->P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return flags_status(h, *h->h_err);
}

// Whether the next force evaluation happens at the positions of the list build
// (then it may drop i-clusters with no pair within r_cut + skin from the list).
void set_build_step(md_handle* h, cudaStream_t s, bool at_build)
{
    cudaMemsetAsync(h->P.builds + 1, at_build ? 0x01 : 0x00, sizeof(int), s);   // nonzero / zero
}

// Adaptive skin: the next list carries the skin again (init and restores);
// the count of unbuffered builds is kept.
cudaError_t reset_list_ctl(md_handle* h)
{
    const Params& P = h->P;
    ListCtl c{};
    c.rlist_f = P.rlist_f;
    c.half_skin2 = P.half_skin2;
    c.r_list = P.r_list;
    c.buffered = 1;
    c.since_build = 0;
    return cudaMemcpy(P.lc, &c, offsetof(ListCtl, unbuffered_builds), cudaMemcpyHostToDevice);
}

// Cell list + cluster-pair list + forces at the current positions/charges
// (no time advance).
void enqueue_rebuild(md_handle* h, cudaStream_t s, bool energy)
{
    launch_step_a(h->P, 0, s, h->grid_atoms);
    launch_cells(h->P, s, h->grid_atoms, h->grid_cells, h->sort_threads);
    launch_pair_list(h->P, s, h->list_blocks);
    set_build_step(h, s, true);   // forces at the build positions: the list may be pruned
    launch_pair_forces(h->P, s, energy, h->pair_blocks, h->pair_warps);
    launch_probe(h->P, s, true);
}

// Cell + list build at the positions held in xr/yr/zr (a checkpoint's list
// positions), then the packed records and forces at the current positions.
void enqueue_rebuild_from_ref(md_handle* h, cudaStream_t s)
{
    Params& P = h->P;
    const size_t nb = (size_t)h->N * sizeof(double);
    double* cur[3] = {P.x, P.y, P.z};
    double* ref[3] = {P.xr, P.yr, P.zr};
    for (int d = 0; d < 3; ++d) {
        cudaMemcpyAsync(h->d_scratch + (size_t)d * h->N, cur[d], nb, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(cur[d], ref[d], nb, cudaMemcpyDeviceToDevice, s);
    }
    launch_step_a(P, 0, s, h->grid_atoms);
    launch_cells(P, s, h->grid_atoms, h->grid_cells, h->sort_threads);
    launch_pair_list(P, s, h->list_blocks);
    // a force pass at the build positions trims the entries' masks as the step
    // of the original build did (its forces are discarded; the trimmed atoms
    // only add exact zeros, so the forces below are the same either way)
    set_build_step(h, s, true);
    launch_pair_forces(P, s, false, h->pair_blocks, h->pair_warps);
    for (int d = 0; d < 3; ++d)
        cudaMemcpyAsync(cur[d], h->d_scratch + (size_t)d * h->N, nb, cudaMemcpyDeviceToDevice, s);
    launch_refresh(P, s);
    set_build_step(h, s, false);  // forces away from the build positions: no pruning
    launch_pair_forces(P, s, false, h->pair_blocks, h->pair_warps);
    launch_probe(P, s, true);
}

void enqueue_step(md_handle* h, cudaStream_t s, bool events)
{
    int mode = STEP_KICK_DRIFT | STEP_ADVANCE | (h->cfg.cr_enabled ? STEP_CR : 0);
    launch_step_a(h->P, mode, s, h->grid_atoms);
    h->build_kernels = launch_cells(h->P, s, h->grid_atoms, h->grid_cells, h->sort_threads) +
                       launch_pair_list(h->P, s, h->list_blocks);
    // external event nodes: the events are recorded on every graph replay
    if (events) cudaEventRecordWithFlags(h->ev_pair0, s, cudaEventRecordExternal);
    launch_pair_forces(h->P, s, false, h->pair_blocks, h->pair_warps);
    if (events) cudaEventRecordWithFlags(h->ev_pair1, s, cudaEventRecordExternal);
    launch_probe(h->P, s, false);
}

// Device error flags without acting on them.
md_status read_flags(md_handle* h, unsigned* e)
{
    CU(cudaMemcpyAsync(h->h_err, h->P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    *e = *h->h_err;
    return MD_OK;
}

void dfree(md_handle* h, void* ptr)
{
    for (size_t k = 0; k < h->allocs.size(); ++k)
        if (h->allocs[k] == ptr) {
            h->allocs.erase(h->allocs.begin() + (long)k);
            break;
        }
    if (h->cfg.dev_free) h->cfg.dev_free(ptr, h->cfg.alloc_ctx);
    else cudaFree(ptr);
}

// (Re)size the cluster-pair list for `entries` entries.
md_status size_list(md_handle* h, long long entries)
{
    Params& P = h->P;
    if (entries > (1LL << 30)) return fail(h, MD_ERR_INVALID_ARG, "cluster-pair list too large");
    if (P.pl) dfree(h, P.pl);
    if (P.pl_chunk) dfree(h, P.pl_chunk);
    P.pl = nullptr;
    P.pl_chunk = nullptr;
    P.pl_cap = (int)entries;
    P.chunk_cap = P.sc_cap + P.pl_cap / kChunk + 1;
    md_status st = dalloc(h, &P.pl, (size_t)P.pl_cap);
    if (st != MD_OK) return st;
    return dalloc(h, &P.pl_chunk, (size_t)P.chunk_cap);
}

// Rebuild at the current state.  A cluster-pair list overflow (the system got
// denser) grows the list to twice the entries needed and rebuilds.
md_status rebuild_checked(md_handle* h, bool* grown, bool from_ref = false)
{
    if (grown) *grown = false;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (from_ref) enqueue_rebuild_from_ref(h, h->stream);
        else enqueue_rebuild(h, h->stream, false);
        CU(cudaGetLastError());
        unsigned e = 0;
        md_status st = read_flags(h, &e);
        if (st != MD_OK) return st;
        if (e != ERR_LIST) return check_device_flags(h);
        int need[2] = {0, 0};
        CU(cudaMemcpy(need, h->P.counters + 6, sizeof(need), cudaMemcpyDeviceToHost));
        st = size_list(h, std::max<long long>(2LL * need[0], 2LL * h->P.pl_cap));
        if (st != MD_OK) return st;
        CU(cudaMemset(h->P.err, 0, sizeof(unsigned)));
        h->list_grows += 1;
        if (grown) *grown = true;
    }
    return fail(h, MD_ERR_CELL_OVERFLOW, "cluster-pair list could not be sized");
}

// Step with a Verlet-buffered list: the step kernel re-packs every atom's
// record in its slot, decides whether the list is used up and sets the
// condition of an IF node whose body is the cell + list build; the forces
// follow.
md_status capture_buffered_step(md_handle* h, bool events)
{
    cudaStream_t s = h->cap_stream;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle hc;
    CU(cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault));
    h->P.cond = hc;
    const int mode = STEP_KICK_DRIFT | STEP_ADVANCE | STEP_SETCOND | (h->cfg.cr_enabled ? STEP_CR : 0);
    launch_step_a(h->P, mode, s, h->grid_atoms);
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    CU(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp));
    cudaGraph_t rebuild = cp.conditional.phGraph_out[0];
    CU(cudaStreamBeginCaptureToGraph(h->body_stream, rebuild, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    h->build_kernels = launch_cells(h->P, h->body_stream, h->grid_atoms, h->grid_cells, h->sort_threads) +
                       launch_pair_list(h->P, h->body_stream, h->list_blocks);
    CU(cudaStreamEndCapture(h->body_stream, &rebuild));
    CU(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
    if (events) cudaEventRecordWithFlags(h->ev_pair0, s, cudaEventRecordExternal);
    launch_pair_forces(h->P, s, false, h->pair_blocks, h->pair_warps);
    if (events) cudaEventRecordWithFlags(h->ev_pair1, s, cudaEventRecordExternal);
    launch_probe(h->P, s, false);
    return MD_OK;
}

// kMultiSteps consecutive steps in one graph (each step with its own rebuild
// IF node and conditional handle), so that md_step(n) issues n / kMultiSteps
// graph launches; the steps are those of the single-step graph, in order.
md_status capture_multi(md_handle* h)
{
    if (h->exec_multi) {
        cudaGraphExecDestroy(h->exec_multi);
        h->exec_multi = nullptr;
    }
    if (h->cfg.profile) return MD_OK;   // profile mode re-points per-step event nodes: one step per launch
    CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < kMultiSteps; ++k) {
        md_status st = MD_OK;
        if (h->cfg.list_skin_nm > 0) st = capture_buffered_step(h, false);
        else enqueue_step(h, h->cap_stream, false);
        if (st != MD_OK) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(h->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            return st;
        }
    }
    cudaGraph_t g = nullptr;
    CU(cudaStreamEndCapture(h->cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&h->exec_multi, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return MD_OK;
}

md_status capture_graph(md_handle* h)
{
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    if (h->graph) {
        cudaGraphDestroy(h->graph);
        h->graph = nullptr;
    }
    CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    if (h->cfg.list_skin_nm > 0) {
        md_status st = capture_buffered_step(h, h->cfg.profile != 0);
        if (st != MD_OK) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(h->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            return st;
        }
    } else {
        enqueue_step(h, h->cap_stream, h->cfg.profile != 0);
    }
    CU(cudaStreamEndCapture(h->cap_stream, &h->graph));
    if (h->cfg.profile) {
        // the two event-record nodes around the pair kernel: each launch points
        // them at a fresh pair of events from the pool
        size_t n = 0;
        CU(cudaGraphGetNodes(h->graph, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        CU(cudaGraphGetNodes(h->graph, nodes.data(), &n));
        h->node_ev0 = h->node_ev1 = nullptr;
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            CU(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            CU(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            if (ev == h->ev_pair0) h->node_ev0 = nd;
            if (ev == h->ev_pair1) h->node_ev1 = nd;
        }
        if (!h->node_ev0 || !h->node_ev1) return fail(h, MD_ERR_CUDA, "profile event nodes not found in the step graph");
    }
    cudaError_t e = cudaGraphInstantiate(&h->exec, h->graph, 0);
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return capture_multi(h);
}

// Pair-kernel times of the launched steps (profile mode).
md_status drain_profile(md_handle* h)
{
    if (h->prof_next == 0) return MD_OK;
    CU(cudaEventSynchronize(h->prof_pool[2 * (h->prof_next - 1) + 1]));
    for (int k = 0; k < h->prof_next; ++k) {
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, h->prof_pool[2 * k], h->prof_pool[2 * k + 1]));
        h->pair_ms += ms;
    }
    h->pair_launches += h->prof_next;
    h->prof_next = 0;
    return MD_OK;
}

// Choose the launch shapes by timing (results are identical for every shape:
// the fixed-point sums and the list's layout do not depend on them): first the
// cell sort's block size and the list build's blocks per SM (a full cell +
// list build at the current positions, which leaves the same list), then the
// force kernel's warps per block and blocks per SM.  Axes pinned in md_config
// are left alone.
md_status autotune(md_handle* h)
{
    const bool fp64 = h->cfg.precision == MD_PREC_FP64;
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    auto timed = [&](auto&& launch, float* out) -> md_status {
        float tot = 0.0f;
        for (int rep = 0; rep < 4; ++rep) {
            CU(cudaEventRecord(a, h->stream));
            launch();
            CU(cudaEventRecord(b, h->stream));
            CU(cudaEventSynchronize(b));
            float ms = 0.0f;
            CU(cudaEventElapsedTime(&ms, a, b));
            if (rep) tot += ms;
        }
        *out = tot;
        return MD_OK;
    };
    {
        const int st_c[] = {256, 1024};
        const int lb_c[] = {2, 4, 8, 16};
        float best = 1e30f;
        int bs = h->sort_threads, bl = h->list_bps;
        for (int st : st_c) {
            if (h->cfg.sort_threads && st != h->cfg.sort_threads) continue;
            for (int lb : lb_c) {
                if (h->cfg.list_blocks_per_sm && lb != h->cfg.list_blocks_per_sm) continue;
                const int lblocks =
                    (int)std::max(1LL, std::min(((long long)h->P.sc_cap + 7) / 8, (long long)lb * h->n_sm));
                float ms = 0.0f;
                md_status s = timed([&]() {
                    launch_cells(h->P, h->stream, h->grid_atoms, h->grid_cells, st);
                    launch_pair_list(h->P, h->stream, lblocks);
                }, &ms);
                if (s != MD_OK) return s;
                if (ms < best) { best = ms; bs = st; bl = lb; }
            }
        }
        h->sort_threads = bs;
        h->list_bps = bl;
        h->list_blocks = (int)std::max(1LL, std::min(((long long)h->P.sc_cap + 7) / 8, (long long)bl * h->n_sm));
    }
    float best = 1e30f;
    int bw = h->pair_warps, bb = h->pair_blocks;
    const int warps_c[] = {4, 8, 12};
    for (int w : warps_c) {
        if (fp64 && w > 8) continue;   // the FP64 kernel takes up to 256 threads per block
        if (h->cfg.pair_warps && w != h->cfg.pair_warps) continue;
        int maxb = pair_max_blocks_per_sm(fp64, false, h->P.screening != 0, w, h->NTS_LJ);
        for (int bps = 1; bps <= maxb; ++bps) {
            if (h->cfg.pair_blocks_per_sm && bps != h->cfg.pair_blocks_per_sm) continue;
            const int blocks = bps * h->n_sm;
            float ms = 0.0f;
            md_status s = timed([&]() {
                // reset the work counter only (the list stays; forces are rebuilt afterwards)
                cudaMemsetAsync(h->P.counters + 2, 0, sizeof(int), h->stream);
                launch_pair_forces(h->P, h->stream, false, blocks, w);
            }, &ms);
            if (s != MD_OK) return s;
            if (ms < best) {
                best = ms;
                bw = w; bb = blocks;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->pair_warps = bw;
    h->pair_blocks = bb;
    return MD_OK;
}

// The bonded terms of md_system: counts, parameter tables, and atoms that are
// distinct, in range, and in one replica and one fragment.
md_status validate_bonded(const md_system* s)
{
    md_handle* h = nullptr;
    if (s->n_bonds < 0 || s->n_angles < 0) return fail(h, MD_ERR_INVALID_ARG, "n_bonds and n_angles must be >= 0");
    if ((long long)s->n_bonds + s->n_angles > (1LL << 30)) return fail(h, MD_ERR_INVALID_ARG, "too many bonded terms");
    if (s->n_bonds > 0 && (!s->bonds || !s->bond_params || s->n_bond_types < 1))
        return fail(h, MD_ERR_INVALID_ARG, "bonds need the bonds array and n_bond_types >= 1 parameter rows");
    if (s->n_angles > 0 && (!s->angles || !s->angle_params || s->n_angle_types < 1))
        return fail(h, MD_ERR_INVALID_ARG, "angles need the angles array and n_angle_types >= 1 parameter rows");
    if (s->n_bonds == 0 && s->n_angles == 0) return MD_OK;
    for (int t = 0; t < (s->n_bonds > 0 ? s->n_bond_types : 0); ++t) {
        const double* b = s->bond_params + 3 * t;
        if (!(b[0] >= 0 && b[0] < 1e9) || !(b[1] >= 0 && b[1] < 1e3) || !(b[2] > 0 && b[2] < 1e6))
            return fail(h, MD_ERR_INVALID_ARG, "bond parameters must be finite with D_e >= 0, b_e >= 0, beta > 0");
    }
    for (int t = 0; t < (s->n_angles > 0 ? s->n_angle_types : 0); ++t) {
        const double* a = s->angle_params + 2 * t;
        if (!(a[0] >= 0 && a[0] < 1e9) || !(a[1] >= 0 && a[1] <= 3.141592653589793))
            return fail(h, MD_ERR_INVALID_ARG, "angle parameters must have 0 <= k_theta < 1e9 and theta_0 in [0, pi]");
    }
    const int N = s->n_atoms;
    std::vector<int> rep(N);
    for (int r = 0; r < s->n_replicas; ++r)
        for (int i = s->replica_offset[r]; i < s->replica_offset[r + 1]; ++i) rep[i] = r;
    auto same = [&](int a, int b) { return rep[a] == rep[b] && s->fragment[a] == s->fragment[b]; };
    for (int t = 0; t < s->n_bonds; ++t) {
        const int* b = s->bonds + 3 * t;
        if (b[0] < 0 || b[0] >= N || b[1] < 0 || b[1] >= N || b[0] == b[1])
            return fail(h, MD_ERR_INVALID_ARG, "bond " + std::to_string(t) + ": atoms out of range or equal");
        if (b[2] < 0 || b[2] >= s->n_bond_types)
            return fail(h, MD_ERR_INVALID_ARG, "bond " + std::to_string(t) + ": type out of range");
        if (!same(b[0], b[1]))
            return fail(h, MD_ERR_INVALID_ARG, "bond " + std::to_string(t) + ": atoms in different replicas or fragments");
    }
    for (int t = 0; t < s->n_angles; ++t) {
        const int* a = s->angles + 4 * t;
        for (int k = 0; k < 3; ++k)
            if (a[k] < 0 || a[k] >= N) return fail(h, MD_ERR_INVALID_ARG, "angle " + std::to_string(t) + ": atom out of range");
        if (a[0] == a[1] || a[1] == a[2] || a[0] == a[2])
            return fail(h, MD_ERR_INVALID_ARG, "angle " + std::to_string(t) + ": atoms must be distinct");
        if (a[3] < 0 || a[3] >= s->n_angle_types)
            return fail(h, MD_ERR_INVALID_ARG, "angle " + std::to_string(t) + ": type out of range");
        if (!same(a[0], a[1]) || !same(a[1], a[2]))
            return fail(h, MD_ERR_INVALID_ARG, "angle " + std::to_string(t) + ": atoms in different replicas or fragments");
    }
    return MD_OK;
}

md_status validate(const md_config* c, const md_system* s)
{
    md_handle* h = nullptr;
    md_status st_bonded = MD_OK;
    if (!c || !s) return fail(h, MD_ERR_INVALID_ARG, "null config or system");
    if (!(c->dt_ps > 0) || !(c->r_cut > 0) || !(c->r_cut < 1e3))
        return fail(h, MD_ERR_INVALID_ARG, "dt_ps and r_cut must be positive");
    if (!(c->list_skin_nm >= 0) || !(c->list_skin_nm <= c->r_cut))
        return fail(h, MD_ERR_INVALID_ARG, "list_skin_nm must be in [0, r_cut]");
    if (c->list_skin_adaptive != 0 && c->list_skin_adaptive != 1)
        return fail(h, MD_ERR_INVALID_ARG, "list_skin_adaptive must be 0 or 1");
    if (c->precision != MD_PREC_MIXED && c->precision != MD_PREC_FP64)
        return fail(h, MD_ERR_INVALID_ARG, "precision must be MD_PREC_MIXED or MD_PREC_FP64");
    if (c->plasma_mode != MD_PLASMA_BOOKKEEPING && c->plasma_mode != MD_PLASMA_PRESCRIBED)
        return fail(h, MD_ERR_INVALID_ARG, "bad plasma_mode");
    if (c->screening != MD_SCREEN_DEBYE && c->screening != MD_SCREEN_HYBRID)
        return fail(h, MD_ERR_INVALID_ARG, "screening must be MD_SCREEN_DEBYE or MD_SCREEN_HYBRID");
    for (int k = 0; k < MD_MAX_SPECIES; ++k)
        if (!(c->langevin_g[k] >= 0.0) || !(c->langevin_g[k] < 1e30))
            return fail(h, MD_ERR_INVALID_ARG, "langevin_g must be finite and >= 0");
    if (c->charge_mode != MD_CHARGE_RATES && c->charge_mode != MD_CHARGE_TABLE)
        return fail(h, MD_ERR_INVALID_ARG, "charge_mode must be MD_CHARGE_RATES or MD_CHARGE_TABLE");
    if (c->max_steps < 1) return fail(h, MD_ERR_INVALID_ARG, "max_steps must be >= 1");
    if (!(c->te_floor_ev > 0)) return fail(h, MD_ERR_INVALID_ARG, "te_floor_ev must be > 0");
    if (!(c->coulomb_f > 0)) return fail(h, MD_ERR_INVALID_ARG, "coulomb_f must be > 0");
    if (c->n_species < 1 || c->n_species > MD_MAX_SPECIES)
        return fail(h, MD_ERR_INVALID_ARG, "n_species out of range");
    int nts = 0;
    for (int k = 0; k < c->n_species; ++k) {
        if (c->z[k] < 1 || c->z[k] > MD_MAX_Z) return fail(h, MD_ERR_INVALID_ARG, "Z out of range");
        if (!(c->mass[k] > 0)) return fail(h, MD_ERR_INVALID_ARG, "masses must be positive");
        if (!(c->lj_sigma0[k] >= 0) || !(c->lj_eps0[k] >= 0))
            return fail(h, MD_ERR_INVALID_ARG, "LJ parameters must be >= 0");
        nts += c->z[k] + 1;
    }
    if (nts > MD_MAX_TYPE_STATES) return fail(h, MD_ERR_INVALID_ARG, "too many type states");
    if (c->n_te < 2 || !(c->dte_ev > 0)) return fail(h, MD_ERR_INVALID_ARG, "Te grid needs n_te >= 2, dte_ev > 0");
    if (!c->sigma_pi || !c->k_ci || !c->k_rec || !c->ip_mev || !c->e_pi_mev || !c->e_auger_mev)
        return fail(h, MD_ERR_INVALID_ARG, "CR tables missing");
    if ((c->dev_alloc == nullptr) != (c->dev_free == nullptr))
        return fail(h, MD_ERR_INVALID_ARG, "dev_alloc and dev_free must be given together");
    if (c->list_reserve < 0 || c->list_reserve > 4096)
        return fail(h, MD_ERR_INVALID_ARG, "list_reserve must be in [0, 4096]");
    if (c->pair_warps != 0 && c->pair_warps != 4 && c->pair_warps != 8 &&
        !(c->pair_warps == 12 && c->precision == MD_PREC_MIXED))
        return fail(h, MD_ERR_INVALID_ARG, "pair_warps must be 0, 4, 8 or 12 (12: mixed precision only)");
    if (c->pair_blocks_per_sm < 0 || c->pair_blocks_per_sm > 64)
        return fail(h, MD_ERR_INVALID_ARG, "pair_blocks_per_sm must be in [0, 64]");
    if (c->sort_threads != 0 && c->sort_threads != 256 && c->sort_threads != 1024)
        return fail(h, MD_ERR_INVALID_ARG, "sort_threads must be 0, 256 or 1024");
    if (c->list_blocks_per_sm < 0 || c->list_blocks_per_sm > 16)
        return fail(h, MD_ERR_INVALID_ARG, "list_blocks_per_sm must be in [0, 16]");
    if (s->n_atoms < 1) return fail(h, MD_ERR_INVALID_ARG, "n_atoms must be >= 1");
    if (!s->x || !s->v || !s->species || !s->fragment || !s->replica_offset || !s->seed || !s->box ||
        !s->volume)
        return fail(h, MD_ERR_INVALID_ARG, "system arrays missing");
    if (s->n_replicas < 1 || s->n_replicas > s->n_atoms)
        return fail(h, MD_ERR_INVALID_ARG, "n_replicas out of range");
    if (s->replica_offset[0] != 0 || s->replica_offset[s->n_replicas] != s->n_atoms)
        return fail(h, MD_ERR_INVALID_ARG, "replica_offset must run from 0 to n_atoms");
    for (int r = 0; r < s->n_replicas; ++r) {
        if (s->replica_offset[r + 1] <= s->replica_offset[r])
            return fail(h, MD_ERR_INVALID_ARG, "every replica needs at least one atom");
        if (!(s->volume[r] > 0)) return fail(h, MD_ERR_INVALID_ARG, "volume must be > 0");
        const double* L = s->box + 3 * r;
        bool per = L[0] > 0 || L[1] > 0 || L[2] > 0;
        if (per) {
            for (int d = 0; d < 3; ++d)
                if (!(L[d] >= 3.0 * (c->r_cut + c->list_skin_nm)))
                    return fail(h, MD_ERR_INVALID_ARG, "periodic box edges must all be >= 3 (r_cut + list_skin_nm)");
        }
    }
    st_bonded = validate_bonded(s);
    if (st_bonded != MD_OK) return st_bonded;
    for (int i = 0; i < s->n_atoms; ++i) {
        if (s->species[i] >= c->n_species) return fail(h, MD_ERR_INVALID_ARG, "species index out of range");
        if (s->q0 && s->q0[i] > c->z[s->species[i]]) return fail(h, MD_ERR_INVALID_ARG, "q0 above Z");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(s->x[3 * i + d]) || !std::isfinite(s->v[3 * i + d]))
                return fail(h, MD_ERR_INVALID_ARG, "non-finite input position or velocity");
    }
    return MD_OK;
}

}  // namespace

void mdg::set_global_error(const std::string& msg) { g_init_error = msg; }

// Runs one entry point's body; host memory exhaustion (or any other C++
// exception) becomes a status instead of crossing the C ABI.
template <class F>
static md_status guarded(md_handle* h, F&& f)
{
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return fail(h, MD_ERR_OOM, "host memory exhausted");
    } catch (const std::exception& e) {
        return fail(h, MD_ERR_CUDA, std::string("internal error: ") + e.what());
    } catch (...) {
        return fail(h, MD_ERR_CUDA, "internal error");
    }
}

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* md_version(void) { return "gb300-ionising-md 0.1 (sm_103a)"; }

const char* md_last_error(const md_handle* h)
{
    if (!h) return g_init_error.c_str();
    return h->err.c_str();
}

static md_status md_pulse_table_body(const md_pulse* p, int n_pulses, double t_start_fs, double dt_fs, int n_steps,
                         double* out)
{
    md_handle* h = nullptr;
    if ((n_pulses > 0 && !p) || n_pulses < 0 || n_steps < 0 || (n_steps > 0 && !out) || !(dt_fs > 0))
        return fail(h, MD_ERR_INVALID_ARG, "md_pulse_table: bad arguments");
    for (int k = 0; k < n_pulses; ++k)
        if (!(p[k].fwhm_fs > 0) || !(p[k].fluence_ph_um2 >= 0) ||
            (p[k].shape != MD_PULSE_GAUSSIAN && p[k].shape != MD_PULSE_FLAT_TOP))
            return fail(h, MD_ERR_INVALID_ARG, "md_pulse_table: bad pulse");
    pulse_table_host(p, n_pulses, t_start_fs, dt_fs, n_steps, out);
    return MD_OK;
}

md_status md_pulse_table(const md_pulse* p, int n_pulses, double t_start_fs, double dt_fs, int n_steps,
                         double* out)
{
    return guarded(nullptr, [&]() { return md_pulse_table_body(p, n_pulses, t_start_fs, dt_fs, n_steps, out); });
}

static md_status init_impl(md_handle* h, const md_config* cfg, const md_system* sys);

static md_status md_init_body(const md_config* cfg, const md_system* sys, md_handle** out)
{
    if (out) *out = nullptr;
    if (!out) return fail(nullptr, MD_ERR_INVALID_ARG, "out is null");
    md_status st = validate(cfg, sys);
    if (st != MD_OK) return st;
    md_handle* h = new md_handle();
    st = init_impl(h, cfg, sys);
    if (st != MD_OK) {
        g_init_error = h->err;
        md_finalize(h);
        return st;
    }
    *out = h;
    return MD_OK;
}

md_status md_init(const md_config* cfg, const md_system* sys, md_handle** out)
{
    return guarded(nullptr, [&]() { return md_init_body(cfg, sys, out); });
}

static md_status init_impl(md_handle* h, const md_config* cfg, const md_system* sys)
{
    h->cfg = *cfg;
    const md_config& c = h->cfg;
    h->N = sys->n_atoms;
    h->R = sys->n_replicas;
    h->NS = c.n_species;
    h->NTE = c.n_te;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
    CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
    CU(cudaEventCreate(&h->ev_pair0));
    CU(cudaEventCreate(&h->ev_pair1));
    if (c.profile) {
        h->prof_pool.assign(2 * kProfPool, nullptr);
        for (cudaEvent_t& ev : h->prof_pool) CU(cudaEventCreate(&ev));
    }
    CU(cudaMallocHost(&h->h_err, sizeof(unsigned)));
    CU(cudaMallocHost(&h->h_rs, (size_t)std::max(sys->n_replicas, 1) * sizeof(RepState)));

    // ---- type states and tables ----
    h->z.assign(c.z, c.z + c.n_species);
    h->ts_off.assign(h->NS + 1, 0);
    for (int s = 0; s < h->NS; ++s) h->ts_off[s + 1] = h->ts_off[s] + h->z[s] + 1;
    const int nts = h->NTS = h->ts_off[h->NS];
    // LJ per pair of type states: sigma scaled by (1 - q/Z) (Eq. 11), arithmetic-mean
    // sigma and geometric-mean epsilon, c6 = 4 eps s^6, c12 = c6 s^6.  The pair
    // table covers only the species present in the system (it is staged in shared
    // memory by the pair kernel); absent species map to row 0 and are never read.
    std::vector<char> present(h->NS, 0);
    for (int i = 0; i < sys->n_atoms; ++i) present[sys->species[i]] = 1;
    h->lj_ts_off.assign(h->NS, 0);
    int nts_lj = 0;
    for (int s = 0; s < h->NS; ++s)
        if (present[s]) {
            h->lj_ts_off[s] = nts_lj;
            nts_lj += h->z[s] + 1;
        }
    h->NTS_LJ = nts_lj;
    std::vector<double> sig_ts(nts_lj), eps_ts(nts_lj);
    for (int s = 0; s < h->NS; ++s)
        if (present[s])
            for (int q = 0; q <= h->z[s]; ++q) {
                sig_ts[h->lj_ts_off[s] + q] = c.lj_sigma0[s] * (1.0 - (double)q / (double)h->z[s]);
                eps_ts[h->lj_ts_off[s] + q] = c.lj_eps0[s];
            }
    std::vector<double2> lj_d((size_t)nts_lj * nts_lj);
    std::vector<float2> lj_f((size_t)nts_lj * nts_lj);
    for (int a = 0; a < nts_lj; ++a)
        for (int b = 0; b < nts_lj; ++b) {
            double sg = 0.5 * (sig_ts[a] + sig_ts[b]);
            double ep = std::sqrt(eps_ts[a] * eps_ts[b]);
            double s6 = sg * sg * sg * sg * sg * sg;
            double c6 = 4.0 * ep * s6, c12 = c6 * s6;
            lj_d[(size_t)a * nts_lj + b] = make_double2(-6.0 * c6, -kLn2 * c12);   // pair kernels take (-6 c6, -ln2 c12)
            lj_f[(size_t)a * nts_lj + b] = make_float2((float)(-6.0 * c6), (float)(-kLn2 * c12));
        }
    std::vector<double> etab(kNEtab), inv12(13, 0.0);
    for (int k = 0; k < kNEtab; ++k) etab[k] = std::exp(-(double)k / 16.0);
    for (int m = 1; m <= 12; ++m) inv12[m] = 1.0 / (double)m;
    std::vector<double> hdtm(h->NS), auger_dt(h->NS), mass(h->NS);
    for (int s = 0; s < h->NS; ++s) {
        hdtm[s] = (0.5 * c.dt_ps) / c.mass[s];
        auger_dt[s] = c.tau_auger_ps[s] > 0 ? c.dt_ps / c.tau_auger_ps[s] : 0.0;
        mass[s] = c.mass[s];
    }

    // ---- replica grids ----
    h->rep_off.assign(sys->replica_offset, sys->replica_offset + h->R + 1);
    h->grid0.assign(h->R, Grid{});
    const double r_list = c.r_cut + c.list_skin_nm;   // cell edge and list cutoff
    long long cells_total = 0;
    for (int r = 0; r < h->R; ++r) {
        Grid& g = h->grid0[r];
        const double* L = sys->box + 3 * r;
        g.periodic = (L[0] > 0 || L[1] > 0 || L[2] > 0) ? 1 : 0;
        if (g.periodic) {
            long long prod = 1;
            for (int d = 0; d < 3; ++d) {
                int n = (int)std::floor(L[d] / r_list);
                n = std::max(3, std::min(n, 1024));
                g.dims[d] = n;
                g.edge[d] = L[d] / n;
                g.inv_edge[d] = 1.0 / g.edge[d];
                g.edge_f[d] = (float)g.edge[d];
                g.origin[d] = 0.0;
                g.box[d] = L[d];
                prod *= n;
            }
            g.cell_cap = (int)prod;
        } else {
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (int i = h->rep_off[r]; i < h->rep_off[r + 1]; ++i)
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::min(lo[d], sys->x[3 * i + d]);
                    hi[d] = std::max(hi[d], sys->x[3 * i + d]);
                }
            long long prod = 1;
            for (int d = 0; d < 3; ++d) {
                long long n = std::max(1LL, (long long)std::floor((hi[d] - lo[d]) / r_list));
                prod *= n;
                g.dims[d] = 1;
                g.edge[d] = r_list;
                g.inv_edge[d] = 1.0 / r_list;
                g.edge_f[d] = (float)r_list;
                g.origin[d] = lo[d];
                g.box[d] = 0.0;
            }
            // room for the sample to expand 4x in cell count before cells grow
            long long cap = std::max(64LL, 4 * prod);
            cap = std::min(cap, (long long)(1 << 22));
            g.cell_cap = (int)cap;
        }
        g.cell_off = (int)cells_total;
        cells_total += g.cell_cap;
    }
    if (cells_total > (1LL << 26)) return fail(h, MD_ERR_INVALID_ARG, "cell grid too large");
    const int C = (int)cells_total;
    const long long slot_cap = (long long)h->N + 7LL * C + 8;
    if (slot_cap > (1LL << 30)) return fail(h, MD_ERR_INVALID_ARG, "system too large");

    // ---- device memory ----
    Params& P = h->P;
    P.n_atoms = h->N; P.n_rep = h->R; P.n_species = h->NS; P.n_ts = nts; P.n_te = h->NTE;
    P.n_ts_lj = h->NTS_LJ;
    P.max_steps = c.max_steps;
    P.cell_cap_total = C;
    P.slot_cap = (int)slot_cap;
    P.cluster_cap = P.slot_cap / kClusterSize + 1;
    P.sc_cap = P.cluster_cap;
    P.precision = c.precision; P.cr_enabled = c.cr_enabled; P.plasma_mode = c.plasma_mode;
    P.dt = c.dt_ps; P.r_cut = c.r_cut; P.rc2 = c.r_cut * c.r_cut; P.kappa_fixed = c.kappa_fixed;
    P.te_floor = c.te_floor_ev; P.coulomb_f = c.coulomb_f;
    P.screening = c.screening;
    P.z_max = 0;
    for (int k = 0; k < c.n_species; ++k) P.z_max = std::max(P.z_max, c.z[k]);
    P.four_pi_f = 4.0 * M_PI * c.coulomb_f;
    P.inv_dte = 1.0 / c.dte_ev;
    P.rc_f = (float)c.r_cut;
    P.r_list = r_list;
    P.rlist_f = (float)r_list;
    P.half_skin2 = (float)(0.25 * c.list_skin_nm * c.list_skin_nm);
    P.rc2_f = P.rc_f * P.rc_f;
    const int N = h->N, R = h->R, NS = h->NS;
    DALLOC(P.x, N); DALLOC(P.y, N); DALLOC(P.z, N);
    DALLOC(P.vx, N); DALLOC(P.vy, N); DALLOC(P.vz, N);
    DALLOC(P.species, N); DALLOC(P.q, N); DALLOC(P.h, N);
    DALLOC(P.frag, N); DALLOC(P.rep, N); DALLOC(P.local_id, N); DALLOC(P.slot_of, N);
    DALLOC(P.atom_cell, N); DALLOC(P.atom_rank, N);
    double *d_hdtm, *d_mass, *d_auger, *d_sigma, *d_kci, *d_krec, *d_etab, *d_inv;
    int *d_z, *d_tsoff, *d_ljtsoff;
    long long *d_ip, *d_epi, *d_eaug;
    float2* d_ljf;
    double2* d_ljd;
    DALLOC(d_hdtm, NS); DALLOC(d_mass, NS); DALLOC(d_z, NS); DALLOC(d_tsoff, NS + 1); DALLOC(d_ljtsoff, NS); DALLOC(d_auger, NS);
    DALLOC(d_sigma, 2 * nts); DALLOC(d_kci, (size_t)nts * h->NTE); DALLOC(d_krec, (size_t)nts * h->NTE);
    DALLOC(d_ip, nts); DALLOC(d_epi, 2 * nts); DALLOC(d_eaug, NS);
    DALLOC(d_etab, kNEtab); DALLOC(d_inv, 13);
    DALLOC(d_ljf, (size_t)nts_lj * nts_lj); DALLOC(d_ljd, (size_t)nts_lj * nts_lj);
    P.hdtm = d_hdtm; P.mass = d_mass; P.zs = d_z; P.ts_off = d_tsoff; P.lj_ts_off = d_ljtsoff; P.auger_dt = d_auger;
    {
        float* d_hf;
        DALLOC(d_hf, NS);
        std::vector<float> hf(NS);
        for (int sp = 0; sp < NS; ++sp) hf[sp] = (float)(hdtm[sp] * kFixInv);
        CU(cudaMemcpy(d_hf, hf.data(), NS * sizeof(float), cudaMemcpyHostToDevice));
        P.hdtm_f = d_hf;
    }
    P.sigma_pi = d_sigma; P.k_ci = d_kci; P.k_rec = d_krec; P.ip_mev = d_ip; P.e_pi_mev = d_epi;
    P.e_auger_mev = d_eaug; P.etab = d_etab; P.inv12 = d_inv; P.lj_f = d_ljf; P.lj_d = d_ljd;
    unsigned long long* d_seed;
    double *d_dF, *d_pne, *d_pte, *d_vol;
    int* d_repoff;
    DALLOC(P.grid, R); DALLOC(P.rs, R); DALLOC(P.acc, (size_t)R * 16);
    if (c.screening == MD_SCREEN_HYBRID) {
        DALLOC(P.hq, (size_t)R * kHybQ);
        DALLOC(P.hrep, R);
    }
    P.charge_mode = c.charge_mode;
    if (c.charge_mode == MD_CHARGE_TABLE) {
        // every atom neutral until a table is set: running sums of 1 everywhere
        const size_t n = (size_t)R * (c.max_steps + 1) * nts;
        DALLOC(P.qcum, n);
        std::vector<double> ones(n, 1.0);
        CU(cudaMemcpy(P.qcum, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    }
    P.langevin = 0;
    for (int k = 0; k < c.n_species; ++k)
        if (c.langevin_g[k] > 0.0) P.langevin = 1;
    if (P.langevin) {
        double* d_g;
        DALLOC(d_g, kMaxSpecies);
        DALLOC(P.lgv, (size_t)R * kMaxSpecies);
        CU(cudaMemcpy(d_g, c.langevin_g, sizeof(double) * std::min(kMaxSpecies, MD_MAX_SPECIES), cudaMemcpyHostToDevice));
        P.lgv_g = d_g;
    }
    P.n_bonds = sys->n_bonds;
    P.n_angles = sys->n_angles;
    P.bonds = nullptr; P.angles = nullptr;
    P.bond_pd = nullptr; P.angle_pd = nullptr; P.bond_pf = nullptr; P.angle_pf = nullptr;
    if (sys->n_bonds > 0) {
        std::vector<int4> b(sys->n_bonds);
        for (int t = 0; t < sys->n_bonds; ++t)
            b[t] = make_int4(sys->bonds[3 * t], sys->bonds[3 * t + 1], sys->bonds[3 * t + 2], 0);
        const int nt = 3 * sys->n_bond_types;
        std::vector<float> pf(sys->bond_params, sys->bond_params + nt);
        int4* d_b; double* d_pd; float* d_pf;
        DALLOC(d_b, b.size()); DALLOC(d_pd, nt); DALLOC(d_pf, nt);
        CU(cudaMemcpy(d_b, b.data(), b.size() * sizeof(int4), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_pd, sys->bond_params, nt * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_pf, pf.data(), nt * sizeof(float), cudaMemcpyHostToDevice));
        P.bonds = d_b; P.bond_pd = d_pd; P.bond_pf = d_pf;
    }
    if (sys->n_angles > 0) {
        const int nt = 2 * sys->n_angle_types;
        std::vector<float> pf(sys->angle_params, sys->angle_params + nt);
        int4* d_a; double* d_pd; float* d_pf;
        DALLOC(d_a, (size_t)sys->n_angles); DALLOC(d_pd, nt); DALLOC(d_pf, nt);
        CU(cudaMemcpy(d_a, sys->angles, (size_t)sys->n_angles * sizeof(int4), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_pd, sys->angle_params, nt * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_pf, pf.data(), nt * sizeof(float), cudaMemcpyHostToDevice));
        P.angles = d_a; P.angle_pd = d_pd; P.angle_pf = d_pf;
    }
    DALLOC(d_seed, R); DALLOC(d_dF, (size_t)R * c.max_steps);
    DALLOC(d_pne, (size_t)R * (c.max_steps + 1)); DALLOC(d_pte, (size_t)R * (c.max_steps + 1));
    DALLOC(d_vol, R); DALLOC(d_repoff, R + 1);
    P.seed = d_seed; P.dF = d_dF; P.pres_ne = d_pne; P.pres_te = d_pte; P.volume = d_vol; P.rep_off = d_repoff;
    DALLOC(P.cell_count, C); DALLOC(P.cell_start, C + 1); DALLOC(P.cell_pstart, C + 1);
    DALLOC(P.tmp_key, N);
    DALLOC(P.sc_cell, P.sc_cap); DALLOC(P.sc_first, P.sc_cap); DALLOC(P.sc_ncl, P.sc_cap);
    DALLOC(P.counters, 8);
    DALLOC(P.list_cnt, (size_t)P.sc_cap * kHalfShell);
    DALLOC(P.sc_tot, P.sc_cap); DALLOC(P.sc_eoff, P.sc_cap); DALLOC(P.sc_coff, P.sc_cap);
    DALLOC(P.scan_tmp, 3 * kScanCtasMax);
    DALLOC(P.big_cells, C);
    P.pl = nullptr;
    P.pl_chunk = nullptr;
    {
        const int reserve = c.list_reserve > 0 ? c.list_reserve : kListMinPerCluster;
        md_status st0 = size_list(h, (long long)reserve * P.cluster_cap);
        if (st0 != MD_OK) return st0;
    }
    if (c.precision == MD_PREC_MIXED) { DALLOC(P.xq, P.slot_cap); P.xq64 = nullptr; }
    else { DALLOC(P.xq64, P.slot_cap); P.xq = nullptr; }
    DALLOC(P.tf, P.slot_cap); DALLOC(P.atom_of, P.slot_cap);
    DALLOC(P.bb_lo, P.cluster_cap); DALLOC(P.bb_hi, P.cluster_cap); DALLOC(P.bb_frag, P.cluster_cap);
    DALLOC(P.fx, P.slot_cap); DALLOC(P.fy, P.slot_cap); DALLOC(P.fz, P.slot_cap); DALLOC(P.epot, P.slot_cap);
    DALLOC(P.pair_count, 1);
    DALLOC(P.err, 1); DALLOC(P.step, 1); DALLOC(P.kick_full, 1);
    DALLOC(h->d_scratch, 3 * (size_t)N);
    DALLOC(P.cl_cen, P.cluster_cap);
    DALLOC(P.maxd2, 1);
    DALLOC(P.builds, 2);
    P.lc = nullptr;
    if (c.list_skin_nm > 0) {
        DALLOC(P.grid_b, R);
        DALLOC(P.xr, N); DALLOC(P.yr, N); DALLOC(P.zr, N);
        if (c.list_skin_adaptive) DALLOC(P.lc, 1);
    } else {
        P.grid_b = P.grid;   // rebuilt every step: the build grid is the grid
        P.xr = P.yr = P.zr = nullptr;
    }
    P.cond = 0;
    DALLOC(h->d_ekin, R); DALLOC(h->d_epot, R);

    // ---- uploads (synchronous, init only) ----
    {
        std::vector<double> tmp(N);
        double* dst[6] = {P.x, P.y, P.z, P.vx, P.vy, P.vz};
        for (int k = 0; k < 6; ++k) {
            const double* src = k < 3 ? sys->x : sys->v;
            for (int i = 0; i < N; ++i) tmp[i] = src[3 * i + (k % 3)];
            CU(cudaMemcpy(dst[k], tmp.data(), N * sizeof(double), cudaMemcpyHostToDevice));
        }
        CU(cudaMemcpy(P.species, sys->species, N, cudaMemcpyHostToDevice));
        h->n_of_species.assign((size_t)R * NS, 0);
        for (int r = 0; r < R; ++r)
            for (int i = h->rep_off[r]; i < h->rep_off[r + 1]; ++i) h->n_of_species[(size_t)r * NS + sys->species[i]] += 1;
        P.x0 = P.y0 = P.z0 = nullptr;
        P.probe = nullptr;
        if (c.probe_record) {
            double *d_x0, *d_y0, *d_z0;
            DALLOC(d_x0, N); DALLOC(d_y0, N); DALLOC(d_z0, N);
            CU(cudaMemcpy(d_x0, P.x, N * sizeof(double), cudaMemcpyDeviceToDevice));
            CU(cudaMemcpy(d_y0, P.y, N * sizeof(double), cudaMemcpyDeviceToDevice));
            CU(cudaMemcpy(d_z0, P.z, N * sizeof(double), cudaMemcpyDeviceToDevice));
            P.x0 = d_x0; P.y0 = d_y0; P.z0 = d_z0;
            const size_t nrec = (size_t)R * (c.max_steps + 1) * NS * 3;
            DALLOC(P.probe, nrec);
            CU(cudaMemset(P.probe, 0, nrec * sizeof(long long)));
        }
        std::vector<uint8_t> q0(N, 0);
        if (sys->q0) std::copy(sys->q0, sys->q0 + N, q0.begin());
        CU(cudaMemcpy(P.q, q0.data(), N, cudaMemcpyHostToDevice));
        CU(cudaMemset(P.h, 0, N));
        CU(cudaMemcpy(P.frag, sys->fragment, N * sizeof(int), cudaMemcpyHostToDevice));
        std::vector<int> rep(N), loc(N);
        std::vector<RepState> rs(R);
        for (int r = 0; r < R; ++r) {
            rs[r] = RepState{};
            for (int i = h->rep_off[r]; i < h->rep_off[r + 1]; ++i) {
                rep[i] = r;
                loc[i] = i - h->rep_off[r];
                rs[r].n_e += q0[i];
            }
        }
        CU(cudaMemcpy(P.rep, rep.data(), N * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(P.local_id, loc.data(), N * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(P.rs, rs.data(), R * sizeof(RepState), cudaMemcpyHostToDevice));
        std::vector<RepAccum> acc((size_t)R * 16);
        for (auto& a : acc) {
            a = RepAccum{};
            for (int d = 0; d < 3; ++d) { a.bmin[d] = ~0ull; a.bmax[d] = 0ull; }
        }
        CU(cudaMemcpy(P.acc, acc.data(), acc.size() * sizeof(RepAccum), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(P.grid, h->grid0.data(), R * sizeof(Grid), cudaMemcpyHostToDevice));
        if (P.grid_b != P.grid)
            CU(cudaMemcpy(P.grid_b, h->grid0.data(), R * sizeof(Grid), cudaMemcpyHostToDevice));
        CU(cudaMemset(P.maxd2, 0, sizeof(unsigned)));
        CU(cudaMemset(P.builds, 0, 2 * sizeof(int)));
        if (P.lc) {
            CU(cudaMemset(P.lc, 0, sizeof(ListCtl)));
            CU(reset_list_ctl(h));
        }
        CU(cudaMemcpy(d_seed, sys->seed, R * sizeof(unsigned long long), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_vol, sys->volume, R * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_repoff, h->rep_off.data(), (R + 1) * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemset(d_dF, 0, (size_t)R * c.max_steps * sizeof(double)));
        CU(cudaMemset(d_pne, 0, (size_t)R * (c.max_steps + 1) * sizeof(double)));
        CU(cudaMemset(d_pte, 0, (size_t)R * (c.max_steps + 1) * sizeof(double)));
        CU(cudaMemcpy(d_hdtm, hdtm.data(), NS * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_mass, mass.data(), NS * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_z, h->z.data(), NS * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_tsoff, h->ts_off.data(), (NS + 1) * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_ljtsoff, h->lj_ts_off.data(), NS * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_auger, auger_dt.data(), NS * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_sigma, c.sigma_pi, 2 * nts * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_kci, c.k_ci, (size_t)nts * h->NTE * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_krec, c.k_rec, (size_t)nts * h->NTE * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_ip, c.ip_mev, nts * sizeof(long long), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_epi, c.e_pi_mev, 2 * nts * sizeof(long long), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_eaug, c.e_auger_mev, NS * sizeof(long long), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_etab, etab.data(), kNEtab * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_inv, inv12.data(), 13 * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_ljf, lj_f.data(), lj_f.size() * sizeof(float2), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_ljd, lj_d.data(), lj_d.size() * sizeof(double2), cudaMemcpyHostToDevice));
        CU(cudaMemset(P.cell_count, 0, C * sizeof(int)));
        CU(cudaMemset(P.counters, 0, 8 * sizeof(int)));
        {
            // the first cell assignment walks atoms in input order
            std::vector<int> ident(P.slot_cap, -1);
            for (int i = 0; i < N; ++i) ident[i] = i;
            CU(cudaMemcpy(P.atom_of, ident.data(), P.slot_cap * sizeof(int), cudaMemcpyHostToDevice));
            CU(cudaMemcpy(P.counters + 1, &N, sizeof(int), cudaMemcpyHostToDevice));
        }
        CU(cudaMemset(P.err, 0, sizeof(unsigned)));
        CU(cudaMemset(P.step, 0, sizeof(long long)));
        CU(cudaMemset(P.kick_full, 0, sizeof(int)));
        CU(cudaMemset(P.slot_of, 0, N * sizeof(int)));
        CU(cudaMemset(P.fx, 0, P.slot_cap * sizeof(long long)));
        CU(cudaMemset(P.fy, 0, P.slot_cap * sizeof(long long)));
        CU(cudaMemset(P.fz, 0, P.slot_cap * sizeof(long long)));
        CU(cudaMemset(P.pair_count, 0, sizeof(long long)));
    }
    h->grid_atoms = (N + 255) / 256;
    h->grid_cells = std::max(1, std::min(C, h->n_sm * 8));
    // many cells per SM: small CTAs keep more (latency-bound) cells in flight
    h->sort_threads = c.sort_threads ? c.sort_threads : (C >= 4 * h->n_sm ? 256 : 1024);
    {
        // the shape with the most resident warps per SM (8-warp blocks on a tie):
        // with many LJ type states the per-block table limits 8-warp blocks
        const bool fp64 = c.precision == MD_PREC_FP64;
        if (c.pair_warps) {
            h->pair_warps = c.pair_warps;
        } else {
            h->pair_warps = 8;
            int best = 8 * pair_max_blocks_per_sm(fp64, false, c.screening != 0, 8, h->NTS_LJ);
            if (!fp64) {
                const int w12 = 12 * pair_max_blocks_per_sm(fp64, false, c.screening != 0, 12, h->NTS_LJ);
                if (w12 > best) h->pair_warps = 12;
            }
        }
        const int maxb = pair_max_blocks_per_sm(fp64, false, c.screening != 0, h->pair_warps, h->NTS_LJ);
        if (c.pair_blocks_per_sm > maxb)
            return fail(h, MD_ERR_INVALID_ARG, "pair_blocks_per_sm exceeds the " + std::to_string(maxb) +
                                                   " blocks of " + std::to_string(h->pair_warps) +
                                                   " warps an SM holds for this system");
        h->pair_blocks = h->n_sm * (c.pair_blocks_per_sm ? c.pair_blocks_per_sm : maxb);
    }
    // list kernels: one warp per super-cluster (or per group of its cells), 8 warps per block
    h->list_bps = c.list_blocks_per_sm ? c.list_blocks_per_sm : 8;
    h->list_blocks = (int)std::max(1LL, std::min(((long long)P.sc_cap + 7) / 8, (long long)h->list_bps * h->n_sm));
    CU(cudaDeviceSynchronize());

    // ---- initial cell list, cluster-pair list and forces F_0 ----
    md_status st = rebuild_checked(h, nullptr);
    if (st != MD_OK) return st;
    if (c.list_reserve == 0) {
        // headroom: twice the entries the initial configuration needs
        int need = 0;
        CU(cudaMemcpy(&need, P.counters + 6, sizeof(int), cudaMemcpyDeviceToHost));
        if (2LL * need > P.pl_cap) {
            st = size_list(h, 2LL * need);
            if (st != MD_OK) return st;
            st = rebuild_checked(h, nullptr);
            if (st != MD_OK) return st;
        }
    }
    if (c.autotune) {
        st = autotune(h);
        if (st != MD_OK) return st;
        st = rebuild_checked(h, nullptr);
        if (st != MD_OK) return st;
    }
    return capture_graph(h);
}

void md_finalize(md_handle* h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->exec_multi) cudaGraphExecDestroy(h->exec_multi);
    for (void* p : h->allocs) {
        if (h->cfg.dev_free) h->cfg.dev_free(p, h->cfg.alloc_ctx);
        else cudaFree(p);
    }
    if (h->ev_pair0) cudaEventDestroy(h->ev_pair0);
    if (h->ev_pair1) cudaEventDestroy(h->ev_pair1);
    for (cudaEvent_t ev : h->prof_pool)
        if (ev) cudaEventDestroy(ev);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->body_stream) cudaStreamDestroy(h->body_stream);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->h_rs) cudaFreeHost(h->h_rs);
    delete h;
}

md_status md_set_stream(md_handle* h, void* stream)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    h->stream = static_cast<cudaStream_t>(stream);
    return MD_OK;
}

static md_status check_replica(md_handle* h, int replica)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    if (replica < -1 || replica >= h->R) return fail(h, MD_ERR_INVALID_ARG, "replica out of range");
    return MD_OK;
}

static md_status md_set_pulse_body(md_handle* h, int replica, const md_pulse* p, int n_pulses)
{
    md_status st = check_replica(h, replica);
    if (st != MD_OK) return st;
    if (n_pulses < 0 || (n_pulses > 0 && !p)) return fail(h, MD_ERR_INVALID_ARG, "bad pulse list");
    for (int k = 0; k < n_pulses; ++k) {
        if (std::fabs(p[k].photon_kev - h->cfg.photon_kev) > 1e-9 * std::max(1.0, h->cfg.photon_kev))
            return fail(h, MD_ERR_INVALID_ARG, "pulse photon energy differs from the cross-section table");
        if (!(p[k].fwhm_fs > 0) || !(p[k].fluence_ph_um2 >= 0) ||
            (p[k].shape != MD_PULSE_GAUSSIAN && p[k].shape != MD_PULSE_FLAT_TOP))
            return fail(h, MD_ERR_INVALID_ARG, "bad pulse parameters");
    }
    std::vector<double> tab(h->cfg.max_steps);
    pulse_table_host(p, n_pulses, h->cfg.t_start_fs, h->cfg.dt_ps * 1000.0, h->cfg.max_steps, tab.data());
    return md_set_pulse_table(h, replica, tab.data(), h->cfg.max_steps);
}

md_status md_set_pulse(md_handle* h, int replica, const md_pulse* p, int n_pulses)
{
    return guarded(h, [&]() { return md_set_pulse_body(h, replica, p, n_pulses); });
}

static md_status md_set_pulse_table_body(md_handle* h, int replica, const double* dF, int n_steps)
{
    md_status st = check_replica(h, replica);
    if (st != MD_OK) return st;
    if (n_steps < 0 || n_steps > h->cfg.max_steps || (n_steps > 0 && !dF))
        return fail(h, MD_ERR_INVALID_ARG, "n_steps must be in [0, max_steps]");
    for (int n = 0; n < n_steps; ++n)
        if (!(dF[n] >= 0) || !std::isfinite(dF[n])) return fail(h, MD_ERR_INVALID_ARG, "fluence must be finite and >= 0");
    const int r0 = replica < 0 ? 0 : replica, r1 = replica < 0 ? h->R : replica + 1;
    for (int r = r0; r < r1; ++r) {
        double* dst = const_cast<double*>(h->P.dF) + (size_t)r * h->cfg.max_steps;
        CU(cudaMemcpyAsync(dst, dF, n_steps * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        if (n_steps < h->cfg.max_steps)
            CU(cudaMemsetAsync(dst + n_steps, 0, (h->cfg.max_steps - n_steps) * sizeof(double), h->stream));
    }
    CU(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status md_set_pulse_table(md_handle* h, int replica, const double* dF, int n_steps)
{
    return guarded(h, [&]() { return md_set_pulse_table_body(h, replica, dF, n_steps); });
}

static md_status md_set_pulse_table_at_body(md_handle* h, int replica, int first_step, const double* dF, int n)
{
    md_status st = check_replica(h, replica);
    if (st != MD_OK) return st;
    if (first_step < 0 || n < 0 || first_step + n > h->cfg.max_steps || (n > 0 && !dF))
        return fail(h, MD_ERR_INVALID_ARG, "range outside [0, max_steps)");
    for (int k = 0; k < n; ++k)
        if (!(dF[k] >= 0) || !std::isfinite(dF[k])) return fail(h, MD_ERR_INVALID_ARG, "fluence must be finite and >= 0");
    const int r0 = replica < 0 ? 0 : replica, r1 = replica < 0 ? h->R : replica + 1;
    for (int r = r0; r < r1; ++r) {
        double* dst = const_cast<double*>(h->P.dF) + (size_t)r * h->cfg.max_steps + first_step;
        CU(cudaMemcpyAsync(dst, dF, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    return MD_OK;
}

md_status md_set_pulse_table_at(md_handle* h, int replica, int first_step, const double* dF, int n)
{
    return guarded(h, [&]() { return md_set_pulse_table_at_body(h, replica, first_step, dF, n); });
}

md_status md_set_fluence_at(md_handle* h, int step, const double* dF)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (step < 0 || step >= h->cfg.max_steps || !dF) return fail(h, MD_ERR_INVALID_ARG, "step outside [0, max_steps)");
    for (int r = 0; r < h->R; ++r)
        if (!(dF[r] >= 0) || !std::isfinite(dF[r])) return fail(h, MD_ERR_INVALID_ARG, "fluence must be finite and >= 0");
    // column `step` of the [replica][max_steps] table: one strided copy
    double* dst = const_cast<double*>(h->P.dF) + step;
    CU(cudaMemcpy2DAsync(dst, (size_t)h->cfg.max_steps * sizeof(double), dF, sizeof(double), sizeof(double),
                         (size_t)h->R, cudaMemcpyHostToDevice, h->stream));
    return MD_OK;
}

static md_status md_set_charge_table_body(md_handle* h, int replica, const double* frac, int n_rows)
{
    md_status st = check_replica(h, replica);
    if (st != MD_OK) return st;
    if (h->cfg.charge_mode != MD_CHARGE_TABLE) return fail(h, MD_ERR_BAD_STATE, "charge_mode is not MD_CHARGE_TABLE");
    if (!frac || n_rows < 1 || n_rows > h->cfg.max_steps + 1)
        return fail(h, MD_ERR_INVALID_ARG, "n_rows must be in [1, max_steps + 1]");
    const int nts = h->NTS;
    std::vector<double> cum((size_t)n_rows * nts);
    for (int n = 0; n < n_rows; ++n)
        for (int s = 0; s < h->NS; ++s) {
            double acc = 0.0;
            for (int k = h->ts_off[s]; k < h->ts_off[s + 1]; ++k) {
                const double f = frac[(size_t)n * nts + k];
                if (!(f >= 0.0) || !(f <= 1.0)) return fail(h, MD_ERR_INVALID_ARG, "fractions must be in [0, 1]");
                acc = acc + f;
                cum[(size_t)n * nts + k] = acc;
            }
            if (!(std::fabs(acc - 1.0) <= 1e-9))
                return fail(h, MD_ERR_INVALID_ARG, "the fractions of a species must sum to 1 (row " + std::to_string(n) + ")");
        }
    const int r0 = replica < 0 ? 0 : replica, r1 = replica < 0 ? h->R : replica + 1;
    const size_t stride = (size_t)(h->cfg.max_steps + 1) * nts;
    for (int r = r0; r < r1; ++r)
        CU(cudaMemcpyAsync(h->P.qcum + r * stride, cum.data(), cum.size() * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status md_set_charge_table(md_handle* h, int replica, const double* frac, int n_rows)
{
    return guarded(h, [&]() { return md_set_charge_table_body(h, replica, frac, n_rows); });
}

static md_status md_set_plasma_table_body(md_handle* h, int replica, const double* ne, const double* te, int n_steps)
{
    md_status st = check_replica(h, replica);
    if (st != MD_OK) return st;
    if (n_steps < 1 || n_steps > h->cfg.max_steps + 1 || !ne || !te)
        return fail(h, MD_ERR_INVALID_ARG, "n_steps must be in [1, max_steps + 1]");
    const int r0 = replica < 0 ? 0 : replica, r1 = replica < 0 ? h->R : replica + 1;
    const size_t stride = (size_t)h->cfg.max_steps + 1;
    for (int r = r0; r < r1; ++r) {
        CU(cudaMemcpyAsync(const_cast<double*>(h->P.pres_ne) + r * stride, ne, n_steps * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemcpyAsync(const_cast<double*>(h->P.pres_te) + r * stride, te, n_steps * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
    }
    // the scalars of the current step change with the table: recompute them
    launch_step_a(h->P, 0, h->stream, h->grid_atoms);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status md_set_plasma_table(md_handle* h, int replica, const double* ne, const double* te, int n_steps)
{
    return guarded(h, [&]() { return md_set_plasma_table_body(h, replica, ne, te, n_steps); });
}

namespace {

md_status launch_steps(md_handle* h, int n)
{
    int k = 0;
    if (h->exec_multi)
        for (; k + kMultiSteps <= n; k += kMultiSteps) CU(cudaGraphLaunch(h->exec_multi, h->stream));
    for (; k < n; ++k) {
        if (h->cfg.profile) {
            if (h->prof_next == kProfPool) {
                md_status st = drain_profile(h);
                if (st != MD_OK) return st;
            }
            const int j = h->prof_next++;
            CU(cudaGraphExecEventRecordNodeSetEvent(h->exec, h->node_ev0, h->prof_pool[2 * j]));
            CU(cudaGraphExecEventRecordNodeSetEvent(h->exec, h->node_ev1, h->prof_pool[2 * j + 1]));
        }
        CU(cudaGraphLaunch(h->exec, h->stream));
    }
    h->host_step += n;
    h->pending += n;
    return MD_OK;
}

}  // namespace

static md_status md_step_async_body(md_handle* h, int n_steps)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    if (n_steps < 0) return fail(h, MD_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (h->host_step + n_steps > h->cfg.max_steps)
        return fail(h, MD_ERR_TABLE_END, "step " + std::to_string(h->host_step + n_steps) +
                                             " is past max_steps = " + std::to_string(h->cfg.max_steps));
    return launch_steps(h, n_steps);
}

md_status md_step_async(md_handle* h, int n_steps)
{
    return guarded(h, [&]() { return md_step_async_body(h, n_steps); });
}

static md_status md_sync_body(md_handle* h)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    while (true) {
        unsigned e = 0;
        md_status st = read_flags(h, &e);
        if (st != MD_OK) return st;
        if (e != ERR_LIST) {
            h->steps += h->pending;
            h->pending = 0;
            st = flags_status(h, e);
            if (st != MD_OK) return st;
            return drain_profile(h);
        }
        // The list of some step overflowed: the state stopped after that step's
        // kick, drift and charge update, and the steps after it did nothing.
        // Grow the list, compute the forces of that step, launch the rest again.
        long long dstep = 0;
        CU(cudaMemcpy(&dstep, h->P.step, sizeof(long long), cudaMemcpyDeviceToHost));
        const long long first = h->host_step - h->pending;
        const long long adv = dstep - first;
        if (adv < 1 || adv > h->pending) return fail(h, MD_ERR_CUDA, "inconsistent step counter after a list overflow");
        const int rest = (int)(h->pending - adv);
        h->steps += adv;
        h->host_step = dstep;
        h->pending = 0;
        CU(cudaMemset(h->P.err, 0, sizeof(unsigned)));
        st = rebuild_checked(h, nullptr);
        if (st != MD_OK) return st;
        st = capture_graph(h);
        if (st != MD_OK) return st;
        st = launch_steps(h, rest);
        if (st != MD_OK) return st;
    }
}

md_status md_sync(md_handle* h)
{
    return guarded(h, [&]() { return md_sync_body(h); });
}

static md_status md_step_body(md_handle* h, int n_steps)
{
    md_status st = md_step_async(h, n_steps);
    if (st != MD_OK) return st;
    return md_sync(h);
}

md_status md_step(md_handle* h, int n_steps)
{
    return guarded(h, [&]() { return md_step_body(h, n_steps); });
}

// The copies of md_get_state that need no host-side reordering (velocities,
// forces, charges, K holes, the replicas' plasma state into pinned memory),
// enqueued on the handle's stream.
static md_status get_state_async(md_handle* h, md_state* out, unsigned fields)
{
    const int N = h->N, R = h->R;
    if (fields & MD_FIELD_V) {
        if (!out->v) return fail(h, MD_ERR_INVALID_ARG, "v buffer missing");
        launch_velocity_out(h->P, h->d_scratch, h->stream);
        CU(cudaMemcpyAsync(out->v, h->d_scratch, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    if (fields & MD_FIELD_F) {
        if (!out->f) return fail(h, MD_ERR_INVALID_ARG, "f buffer missing");
        launch_force_out(h->P, h->d_scratch, h->stream);
        CU(cudaMemcpyAsync(out->f, h->d_scratch, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    if (fields & MD_FIELD_Q) {
        if (!out->q) return fail(h, MD_ERR_INVALID_ARG, "q buffer missing");
        CU(cudaMemcpyAsync(out->q, h->P.q, N, cudaMemcpyDeviceToHost, h->stream));
    }
    if (fields & MD_FIELD_H) {
        if (!out->h) return fail(h, MD_ERR_INVALID_ARG, "h buffer missing");
        CU(cudaMemcpyAsync(out->h, h->P.h, N, cudaMemcpyDeviceToHost, h->stream));
    }
    if (fields & (MD_FIELD_PLASMA | MD_FIELD_COUNTS))
        CU(cudaMemcpyAsync(h->h_rs, h->P.rs, R * sizeof(RepState), cudaMemcpyDeviceToHost, h->stream));
    return MD_OK;
}

// The plasma fields from the pinned copy of the replicas' state (after the
// stream has been synchronised).
static void unpack_rep_state(md_handle* h, md_state* out, unsigned fields)
{
    if (!(fields & (MD_FIELD_PLASMA | MD_FIELD_COUNTS))) return;
    const RepState* rs = h->h_rs;
    for (int r = 0; r < h->R; ++r) {
        if (fields & MD_FIELD_PLASMA) {
            if (out->n_e) out->n_e[r] = rs[r].n_e;
            if (out->e_gas_mev) out->e_gas_mev[r] = rs[r].e_gas;
            if (out->te_ev) out->te_ev[r] = rs[r].te_ev;
            if (out->kappa) out->kappa[r] = rs[r].kappa;
        }
        if ((fields & MD_FIELD_COUNTS) && out->event_counts)
            for (int k = 0; k < 4; ++k) out->event_counts[4 * r + k] = rs[r].counts[k];
    }
}

static md_status md_get_state_body(md_handle* h, md_state* out, unsigned fields)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (!out) return fail(h, MD_ERR_INVALID_ARG, "null state");
    // Fields copied without host-side reordering, after steps still in flight:
    // the copies and the error flags are read in one round trip.  Any flag
    // set (a list overflow, an error) falls back to md_sync and copies again.
    const unsigned host_side = MD_FIELD_X | MD_FIELD_XLIST;
    if (h->pending && !h->poisoned && !(fields & host_side)) {
        md_status st = get_state_async(h, out, fields);
        if (st != MD_OK) return st;
        CU(cudaMemcpyAsync(h->h_err, h->P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        if (*h->h_err == 0) {
            h->steps += h->pending;
            h->pending = 0;
            st = drain_profile(h);
            if (st != MD_OK) return st;
            unpack_rep_state(h, out, fields);
            if (fields & MD_FIELD_STEP) out->step = h->host_step;
            return MD_OK;
        }
    }
    if (h->pending && !h->poisoned) {
        md_status st_ = md_sync(h);
        if (st_ != MD_OK) return st_;
    }
    const int N = h->N;
    CU(cudaStreamSynchronize(h->stream));
    std::vector<double> tmp;
    if (fields & MD_FIELD_X) {
        if (!out->x) return fail(h, MD_ERR_INVALID_ARG, "x buffer missing");
        tmp.resize(N);
        double* src[3] = {h->P.x, h->P.y, h->P.z};
        for (int d = 0; d < 3; ++d) {
            CU(cudaMemcpy(tmp.data(), src[d], N * sizeof(double), cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i) out->x[3 * i + d] = tmp[i];
        }
    }
    {
        md_status st = get_state_async(h, out, fields);
        if (st != MD_OK) return st;
        CU(cudaStreamSynchronize(h->stream));
        unpack_rep_state(h, out, fields);
    }
    if (fields & MD_FIELD_STEP) out->step = h->host_step;
    if (fields & MD_FIELD_XLIST) {
        if (!out->x_list) return fail(h, MD_ERR_INVALID_ARG, "x_list buffer missing");
        tmp.resize(N);
        const bool buffered = h->P.xr != nullptr;
        double* src[3] = {buffered ? h->P.xr : h->P.x, buffered ? h->P.yr : h->P.y, buffered ? h->P.zr : h->P.z};
        for (int d = 0; d < 3; ++d) {
            CU(cudaMemcpy(tmp.data(), src[d], N * sizeof(double), cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i) out->x_list[3 * i + d] = tmp[i];
        }
    }
    CU(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status md_get_state(md_handle* h, md_state* out, unsigned fields)
{
    return guarded(h, [&]() { return md_get_state_body(h, out, fields); });
}

static md_status md_set_state_body(md_handle* h, const md_state* in, unsigned fields)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (!in) return fail(h, MD_ERR_INVALID_ARG, "null state");
    if (h->pending && !h->poisoned) {
        md_status st_ = md_sync(h);
        if (st_ != MD_OK) return st_;
    }
    const int N = h->N, R = h->R;
    CU(cudaStreamSynchronize(h->stream));
    // bring velocities to the integer step with the current forces first
    launch_velocity_out(h->P, h->d_scratch, h->stream);
    {
        std::vector<double> v(3 * (size_t)N), tmp(N);
        CU(cudaMemcpyAsync(v.data(), h->d_scratch, v.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        const double* vs = (fields & MD_FIELD_V) ? in->v : v.data();
        if ((fields & MD_FIELD_V) && !in->v) return fail(h, MD_ERR_INVALID_ARG, "v buffer missing");
        double* dst[3] = {h->P.vx, h->P.vy, h->P.vz};
        for (int d = 0; d < 3; ++d) {
            for (int i = 0; i < N; ++i) {
                tmp[i] = vs[3 * i + d];
                if (!std::isfinite(tmp[i])) return fail(h, MD_ERR_INVALID_ARG, "non-finite velocity");
            }
            CU(cudaMemcpy(dst[d], tmp.data(), N * sizeof(double), cudaMemcpyHostToDevice));
        }
    }
    if (fields & MD_FIELD_X) {
        if (!in->x) return fail(h, MD_ERR_INVALID_ARG, "x buffer missing");
        std::vector<double> tmp(N);
        double* dst[3] = {h->P.x, h->P.y, h->P.z};
        for (int d = 0; d < 3; ++d) {
            for (int i = 0; i < N; ++i) {
                tmp[i] = in->x[3 * i + d];
                if (!std::isfinite(tmp[i])) return fail(h, MD_ERR_INVALID_ARG, "non-finite position");
            }
            CU(cudaMemcpy(dst[d], tmp.data(), N * sizeof(double), cudaMemcpyHostToDevice));
        }
    }
    if (fields & MD_FIELD_Q) {
        if (!in->q) return fail(h, MD_ERR_INVALID_ARG, "q buffer missing");
        std::vector<uint8_t> sp(N);
        CU(cudaMemcpy(sp.data(), h->P.species, N, cudaMemcpyDeviceToHost));
        for (int i = 0; i < N; ++i)
            if (in->q[i] > h->z[sp[i]]) return fail(h, MD_ERR_INVALID_ARG, "q above Z");
        CU(cudaMemcpy(h->P.q, in->q, N, cudaMemcpyHostToDevice));
    }
    if (fields & MD_FIELD_H) {
        if (!in->h) return fail(h, MD_ERR_INVALID_ARG, "h buffer missing");
        for (int i = 0; i < N; ++i)
            if (in->h[i] > 1) return fail(h, MD_ERR_INVALID_ARG, "h must be 0 or 1");
        CU(cudaMemcpy(h->P.h, in->h, N, cudaMemcpyHostToDevice));
    }
    if (fields & (MD_FIELD_PLASMA | MD_FIELD_COUNTS)) {
        std::vector<RepState> rs(R);
        CU(cudaMemcpy(rs.data(), h->P.rs, R * sizeof(RepState), cudaMemcpyDeviceToHost));
        for (int r = 0; r < R; ++r) {
            if (fields & MD_FIELD_PLASMA) {
                if (!in->n_e || !in->e_gas_mev) return fail(h, MD_ERR_INVALID_ARG, "plasma buffers missing");
                if (in->n_e[r] < 0 || in->e_gas_mev[r] < 0) return fail(h, MD_ERR_INVALID_ARG, "negative plasma counter");
                rs[r].n_e = in->n_e[r];
                rs[r].e_gas = in->e_gas_mev[r];
            }
            if ((fields & MD_FIELD_COUNTS) && in->event_counts)
                for (int k = 0; k < 4; ++k) rs[r].counts[k] = in->event_counts[4 * r + k];
        }
        CU(cudaMemcpy(h->P.rs, rs.data(), R * sizeof(RepState), cudaMemcpyHostToDevice));
    }
    if (fields & MD_FIELD_STEP) {
        if (in->step < 0 || in->step > h->cfg.max_steps) return fail(h, MD_ERR_INVALID_ARG, "step out of range");
        h->host_step = in->step;
        CU(cudaMemcpy(h->P.step, &in->step, sizeof(long long), cudaMemcpyHostToDevice));
    }
    CU(cudaMemset(h->P.kick_full, 0, sizeof(int)));
    CU(cudaMemset(h->P.err, 0, sizeof(unsigned)));
    h->poisoned = false;
    bool from_ref = false;
    if (fields & MD_FIELD_XLIST) {
        if (!in->x_list) return fail(h, MD_ERR_INVALID_ARG, "x_list buffer missing");
        if (h->P.xr) {   // buffered list: rebuild it where the checkpointed run built it
            std::vector<double> tmp(N);
            double* dst[3] = {h->P.xr, h->P.yr, h->P.zr};
            for (int d = 0; d < 3; ++d) {
                for (int i = 0; i < N; ++i) {
                    tmp[i] = in->x_list[3 * i + d];
                    if (!std::isfinite(tmp[i])) return fail(h, MD_ERR_INVALID_ARG, "non-finite list position");
                }
                CU(cudaMemcpy(dst[d], tmp.data(), N * sizeof(double), cudaMemcpyHostToDevice));
            }
            from_ref = true;
        }
    }
    if (h->P.lc) CU(reset_list_ctl(h));   // the restored list carries the skin
    bool grown = false;
    md_status st = rebuild_checked(h, &grown, from_ref);
    if (st != MD_OK) return st;
    return grown ? capture_graph(h) : MD_OK;
}

md_status md_set_state(md_handle* h, const md_state* in, unsigned fields)
{
    return guarded(h, [&]() { return md_set_state_body(h, in, fields); });
}

static md_status md_rdf_body(md_handle* h, double r_max, int n_bins, int64_t* counts)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (!counts) return fail(h, MD_ERR_INVALID_ARG, "null counts");
    if (!(r_max > 0.0) || r_max > h->cfg.r_cut) return fail(h, MD_ERR_INVALID_ARG, "r_max must be in (0, r_cut]");
    if (n_bins < 1 || n_bins > 65536) return fail(h, MD_ERR_INVALID_ARG, "n_bins must be in [1, 65536]");
    if (h->pending && !h->poisoned) {
        md_status st_ = md_sync(h);
        if (st_ != MD_OK) return st_;
    }
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    const int ns = h->NS;
    const size_t nh = (size_t)ns * ns * n_bins;
    unsigned long long* d_hist = nullptr;
    md_status st = dalloc(h, &d_hist, nh);
    if (st != MD_OK) return st;
    // the list of the last build covers every pair within r_cut at the current
    // positions, and the packed records hold the current positions
    CU(cudaMemsetAsync(d_hist, 0, nh * sizeof(unsigned long long), h->stream));
    CU(cudaMemsetAsync(h->P.counters + 2, 0, sizeof(int), h->stream));
    launch_rdf(h->P, h->stream, h->n_sm * 4, n_bins, r_max, d_hist);
    CU(cudaMemsetAsync(h->P.counters + 2, 0, sizeof(int), h->stream));
    CU(cudaGetLastError());
    std::vector<unsigned long long> tmp(nh);
    CU(cudaMemcpyAsync(tmp.data(), d_hist, nh * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    dfree(h, d_hist);
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b)
            for (int k = 0; k < n_bins; ++k) {
                const int lo = std::min(a, b), hi = std::max(a, b);
                counts[((size_t)a * ns + b) * n_bins + k] = (int64_t)tmp[((size_t)lo * ns + hi) * n_bins + k];
            }
    return MD_OK;
}

md_status md_rdf(md_handle* h, double r_max, int n_bins, int64_t* counts)
{
    return guarded(h, [&]() { return md_rdf_body(h, r_max, n_bins, counts); });
}

static md_status md_fragments_body(md_handle* h, double r_frag, int mass_max, int charge_max, int32_t* label, int64_t* counts)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (!(r_frag > 0.0) || r_frag > h->cfg.r_cut) return fail(h, MD_ERR_INVALID_ARG, "r_frag must be in (0, r_cut]");
    if (mass_max < 0 || mass_max > 1000000 || charge_max < 0 || charge_max > 100000 || (!label && !counts))
        return fail(h, MD_ERR_INVALID_ARG, "mass_max, charge_max out of range or no output");
    const size_t nc = (size_t)h->R * (mass_max + 1) * (charge_max + 1);
    if (nc > ((size_t)1 << 28)) return fail(h, MD_ERR_INVALID_ARG, "count array too large");
    if (h->pending && !h->poisoned) {
        md_status st_ = md_sync(h);
        if (st_ != MD_OK) return st_;
    }
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    const int N = h->N;
    int *d_parent = nullptr, *d_label = nullptr, *d_mass = nullptr, *d_charge = nullptr;
    unsigned long long* d_counts = nullptr;
    md_status st = dalloc(h, &d_parent, N);
    if (st == MD_OK) st = dalloc(h, &d_label, N);
    if (st == MD_OK) st = dalloc(h, &d_mass, N);
    if (st == MD_OK) st = dalloc(h, &d_charge, N);
    if (st == MD_OK) st = dalloc(h, &d_counts, nc);
    auto release = [&]() {
        for (void* ptr : {(void*)d_parent, (void*)d_label, (void*)d_mass, (void*)d_charge, (void*)d_counts})
            if (ptr) dfree(h, ptr);
    };
    if (st != MD_OK) {
        release();
        return st;
    }
    int an[kMaxSpecies] = {0};
    for (int k = 0; k < h->NS; ++k) an[k] = (int)std::lround(h->cfg.mass[k]);   // mass numbers
    // the list of the last build covers every pair within r_cut at the current
    // positions, and the packed records hold the current positions
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemsetAsync(d_counts, 0, nc * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        launch_frag_init(h->P, s, d_parent, d_mass, d_charge);
        e = cudaMemsetAsync(h->P.counters + 2, 0, sizeof(int), s);
    }
    if (e == cudaSuccess) {
        launch_frag_link(h->P, s, h->n_sm * 4, r_frag, d_parent);
        e = cudaMemsetAsync(h->P.counters + 2, 0, sizeof(int), s);
    }
    if (e == cudaSuccess) {
        launch_frag_count(h->P, s, d_parent, d_label, d_mass, d_charge, an, mass_max, charge_max, d_counts);
        e = cudaGetLastError();
    }
    std::vector<unsigned long long> tmp(counts ? nc : 0);
    if (e == cudaSuccess && label)
        e = cudaMemcpyAsync(label, d_label, (size_t)N * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && counts)
        e = cudaMemcpyAsync(tmp.data(), d_counts, nc * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release();
    if (e != cudaSuccess) return fail(h, MD_ERR_CUDA, std::string("md_fragments: ") + cudaGetErrorString(e));
    for (size_t k = 0; k < tmp.size(); ++k) counts[k] = (int64_t)tmp[k];
    return check_device_flags(h);
}

md_status md_fragments(md_handle* h, double r_frag, int mass_max, int charge_max, int32_t* label, int64_t* counts)
{
    return guarded(h, [&]() { return md_fragments_body(h, r_frag, mass_max, charge_max, label, counts); });
}

static md_status md_get_probe_series_body(md_handle* h, int replica, int first, int n, int64_t* q_sum, double* d2_sum)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (!h->P.probe) return fail(h, MD_ERR_BAD_STATE, "probe records are off (md_config.probe_record = 0)");
    if (h->pending && !h->poisoned) {
        md_status st_ = md_sync(h);
        if (st_ != MD_OK) return st_;
    }
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    if (replica < 0 || replica >= h->R) return fail(h, MD_ERR_INVALID_ARG, "replica out of range");
    if (first < 0 || n < 1 || (long long)first + n - 1 > h->host_step || (!q_sum && !d2_sum))
        return fail(h, MD_ERR_INVALID_ARG, "records first .. first + n - 1 must lie in 0 .. the current step");
    const int ns = h->NS;
    std::vector<long long> tmp((size_t)n * ns * 3);
    const size_t off = 3 * (((size_t)replica * (h->cfg.max_steps + 1) + (size_t)first) * ns);
    CU(cudaMemcpyAsync(tmp.data(), h->P.probe + off, tmp.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < (size_t)n * ns; ++k) {
        if (q_sum) q_sum[k] = tmp[3 * k];
        // high and low 32-bit parts of the 2^-40 nm^2 fixed-point sum
        if (d2_sum) d2_sum[k] = (double)tmp[3 * k + 1] * 0.00390625 + (double)tmp[3 * k + 2] * 9.094947017729282e-13;
    }
    return MD_OK;
}

md_status md_get_probe_series(md_handle* h, int replica, int first, int n, int64_t* q_sum, double* d2_sum)
{
    return guarded(h, [&]() { return md_get_probe_series_body(h, replica, first, n, q_sum, d2_sum); });
}

static md_status md_probe_displacement_body(md_handle* h, int replica, int first, int n, const md_pulse* probe, int n_pulses,
                                double* out)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (!out || !probe || n_pulses < 1) return fail(h, MD_ERR_INVALID_ARG, "probe pulses and out are required");
    for (int k = 0; k < n_pulses; ++k)
        if (!(probe[k].fwhm_fs > 0) || !(probe[k].fluence_ph_um2 >= 0) ||
            (probe[k].shape != MD_PULSE_GAUSSIAN && probe[k].shape != MD_PULSE_FLAT_TOP))
            return fail(h, MD_ERR_INVALID_ARG, "bad probe pulse");
    const int ns = h->NS;
    std::vector<int64_t> qs((size_t)n > 0 ? (size_t)n * ns : 1);
    std::vector<double> d2((size_t)n > 0 ? (size_t)n * ns : 1);
    md_status st = md_get_probe_series(h, replica, first, n, qs.data(), d2.data());
    if (st != MD_OK) return st;
    // Eq. 17: w_k = int_{t_k}^{t_k + dt} g f / int g f, f constant over a step
    std::vector<double> G(n);
    const double dt_fs = h->cfg.dt_ps * 1000.0;
    pulse_table_host(probe, n_pulses, h->cfg.t_start_fs + first * dt_fs, dt_fs, n, G.data());
    for (int s = 0; s < ns; ++s) {
        const double na = (double)h->n_of_species[(size_t)replica * ns + s];
        out[s] = 0.0;
        if (!(na > 0)) continue;
        double tot = 0.0, acc = 0.0;
        for (int k = 0; k < n; ++k) {
            const double f = 1.0 - ((double)qs[(size_t)k * ns + s] / na) / (double)h->z[s];
            const double gf = G[k] * f;
            tot += gf;
            acc += gf * std::sqrt(d2[(size_t)k * ns + s] / na);
        }
        out[s] = tot > 0 ? acc / tot : 0.0;
    }
    return MD_OK;
}

md_status md_probe_displacement(md_handle* h, int replica, int first, int n, const md_pulse* probe, int n_pulses,
                                double* out)
{
    return guarded(h, [&]() { return md_probe_displacement_body(h, replica, first, n, probe, n_pulses, out); });
}

static md_status md_structure_factor_body(const int64_t* counts, int n_bins, double r_max, double n_a, double n_b, int same,
                              double volume, double rho0, const double* q, int n_q, double* s)
{
    if (!counts || !q || !s || n_bins < 1 || n_q < 1 || !(r_max > 0.0) || !(volume > 0.0) || !(rho0 >= 0.0))
        return fail(nullptr, MD_ERR_INVALID_ARG, "bad arguments to md_structure_factor");
    const double dr = r_max / n_bins;
    const double pairs = same ? 0.5 * n_a * (n_a - 1.0) : n_a * n_b;
    if (!(pairs > 0.0)) return fail(nullptr, MD_ERR_INVALID_ARG, "no pairs for this species pair");
    std::vector<double> rk(n_bins), gk(n_bins);
    for (int k = 0; k < n_bins; ++k) {
        const double r0 = k * dr, r1 = (k + 1) * dr;
        const double shell = 4.0 * kPi / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0);
        rk[k] = 0.5 * (r0 + r1);
        gk[k] = (double)counts[k] / (pairs / volume * shell);
    }
    for (int j = 0; j < n_q; ++j) {
        if (!(q[j] > 0.0)) return fail(nullptr, MD_ERR_INVALID_ARG, "q must be > 0");
        double acc = 0.0;
        for (int k = 0; k < n_bins; ++k) acc += rk[k] * (gk[k] - 1.0) * std::sin(q[j] * rk[k]);
        s[j] = 1.0 + 4.0 * kPi * rho0 / q[j] * acc * dr;
    }
    return MD_OK;
}

md_status md_structure_factor(const int64_t* counts, int n_bins, double r_max, double n_a, double n_b, int same,
                              double volume, double rho0, const double* q, int n_q, double* s)
{
    return guarded(nullptr, [&]() { return md_structure_factor_body(counts, n_bins, r_max, n_a, n_b, same, volume, rho0, q, n_q, s); });
}

static md_status md_get_energies_body(md_handle* h, double* e_kin, double* e_pot, int64_t* n_pairs)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (h->pending && !h->poisoned) {
        md_status st_ = md_sync(h);
        if (st_ != MD_OK) return st_;
    }
    if (h->poisoned) return fail(h, MD_ERR_BAD_STATE, "handle is in an error state: " + h->err);
    const int R = h->R;
    CU(cudaMemsetAsync(h->P.pair_count, 0, sizeof(long long), h->stream));
    // the current list and packed records (re-packed from the same state), so
    // the forces come out bit-identical
    launch_refresh(h->P, h->stream);
    set_build_step(h, h->stream, false);
    launch_pair_forces(h->P, h->stream, true, h->pair_blocks, h->pair_warps);
    launch_energy(h->P, h->d_ekin, h->d_epot, h->stream);
    CU(cudaGetLastError());
    std::vector<double> ek(R);
    std::vector<long long> ep(R);
    long long np = 0;
    CU(cudaMemcpyAsync(ek.data(), h->d_ekin, R * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(ep.data(), h->d_epot, R * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&np, h->P.pair_count, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    md_status st = check_device_flags(h);
    if (st != MD_OK) return st;
    for (int r = 0; r < R; ++r) {
        if (e_kin) e_kin[r] = ek[r];
        if (e_pot) e_pot[r] = (double)ep[r] * kFixInv;
    }
    if (n_pairs) *n_pairs = np;
    h->last_pairs = np;
    return MD_OK;
}

md_status md_get_energies(md_handle* h, double* e_kin, double* e_pot, int64_t* n_pairs)
{
    return guarded(h, [&]() { return md_get_energies_body(h, e_kin, e_pot, n_pairs); });
}

md_status md_get_timing(md_handle* h, md_timing* out)
{
    if (!h || !out) return fail(h, MD_ERR_INVALID_ARG, "null argument");
    if (h->pending && !h->poisoned) {
        md_status st = md_sync(h);
        if (st != MD_OK) return st;
    }
    out->pair_ms = h->pair_ms;
    out->pair_launches = h->pair_launches;
    out->steps = h->steps;
    out->pair_count_last = h->last_pairs;
    out->tile_warps = h->pair_warps;
    out->tile_blocks_per_sm = h->pair_blocks / std::max(1, h->n_sm);
    out->list_capacity = h->P.pl_cap;
    int used = 0;
    CU(cudaMemcpy(&used, h->P.counters + 6, sizeof(int), cudaMemcpyDeviceToHost));
    out->list_entries = used;
    out->list_grows = h->list_grows;
    out->sort_threads = h->sort_threads;
    out->list_blocks_per_sm = h->list_bps;
    out->build_kernels = h->build_kernels;
    if (h->cfg.list_skin_nm > 0) {
        int b = 0;
        CU(cudaMemcpy(&b, h->P.builds, sizeof(int), cudaMemcpyDeviceToHost));
        out->list_builds = b;
    } else {
        out->list_builds = h->steps;
    }
    out->list_unbuffered_builds = 0;
    if (h->P.lc) {
        long long u = 0;
        CU(cudaMemcpy(&u, reinterpret_cast<char*>(h->P.lc) + offsetof(ListCtl, unbuffered_builds), sizeof(u),
                      cudaMemcpyDeviceToHost));
        out->list_unbuffered_builds = u;
    }
    return MD_OK;
}

md_status md_reset_timing(md_handle* h)
{
    if (!h) return fail(nullptr, MD_ERR_INVALID_ARG, "null handle");
    if (h->pending && !h->poisoned) {
        md_status st = md_sync(h);
        if (st != MD_OK) return st;
    }
    h->pair_ms = 0.0;
    h->pair_launches = 0;
    h->steps = 0;
    CU(cudaMemset(h->P.builds, 0, sizeof(int)));
    if (h->P.lc)
        CU(cudaMemset(reinterpret_cast<char*>(h->P.lc) + offsetof(ListCtl, unbuffered_builds), 0, sizeof(long long)));
    return MD_OK;
}

md_status md_philox(uint64_t seed, const uint32_t* d_ctr4, int64_t n, uint32_t* d_out, void* stream)
{
    md_handle* h = nullptr;
    if (n < 0 || (n > 0 && (!d_ctr4 || !d_out))) return fail(h, MD_ERR_INVALID_ARG, "md_philox: bad arguments");
    launch_philox(seed, d_ctr4, n, d_out, static_cast<cudaStream_t>(stream));
    CU(cudaGetLastError());
    return MD_OK;
}

}  // extern "C"
