// Cell-list neighbour build (every step, or when the Verlet skin is used up).  The paper's cutoff is chosen
// from the screening (Sec. II.B); here every replica gets a grid of cells of
// edge >= r_cut, atoms are counted per cell, the cells are scanned, and each
// cell is sorted deterministically (3D Hilbert index of a 16^3 sub-grid, then
// atom index) into a padded slot range that is a multiple of the 8-atom
// cluster size; runs of 8 consecutive atoms along the Hilbert curve are
// compact, near-cubic clusters.  The
// packed arrays hold FP32 (or FP64) coordinates relative to the cell centre,
// the charge, the type state and the fragment, plus one bounding box per
// cluster for the pair kernel's prefilter.
#include <algorithm>

#include "md_internal.cuh"

namespace mdg {

constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 1024;
constexpr int kSortMax = 2048;       // keys per cell kept in shared memory (larger cells sort from global memory)
constexpr int kSmallCell = 256;      // cells up to this many atoms are sorted by one warp
constexpr int kScanCellsMulti = 16384;   // grids of at least this many cells are scanned by many CTAs
constexpr int kSmallWarps = 8;       // warps per block of the one-warp-per-cell sort

__device__ __forceinline__ int cell_coord(double x, double origin, double inv_edge, int n)
{
    double u = (x - origin) * inv_edge;
    int c = (u >= 0.0) ? (int)u : 0;   // NaN and negatives -> 0
    return c < n ? c : n - 1;
}

// Index of cell (x, y, z) of a 2^kHilBits grid along the 3D Hilbert curve
// (Skilling's transpose algorithm, "Programming the Hilbert curve", AIP Conf.
// Proc. 707, 2004: undo the excess work, Gray-encode, interleave the bits).
constexpr int kHilBits = 4;
__device__ __forceinline__ unsigned hilbert3(unsigned x0, unsigned x1, unsigned x2)
{
    unsigned X[3] = {x0, x1, x2};
#pragma unroll
    for (unsigned Q = 1u << (kHilBits - 1); Q > 1; Q >>= 1) {
        const unsigned P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const unsigned t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    unsigned t = 0;
#pragma unroll
    for (unsigned Q = 1u << (kHilBits - 1); Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    X[0] ^= t; X[1] ^= t; X[2] ^= t;
    unsigned key = 0;
#pragma unroll
    for (int b = kHilBits - 1; b >= 0; --b)
#pragma unroll
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

// Atoms are visited in the previous step's slot order, so neighbouring
// threads mostly share a cell and one atomic per (warp, cell) suffices.
__global__ void __launch_bounds__(256) k_cell_assign(Params p)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int i = s < p.counters[1] ? p.atom_of[s] : -1;
    int c = -1;
    if (i >= 0) {
        const Grid& g = p.grid[p.rep[i]];
        const int cx = cell_coord(p.x[i], g.origin[0], g.inv_edge[0], g.dims[0]);
        const int cy = cell_coord(p.y[i], g.origin[1], g.inv_edge[1], g.dims[1]);
        const int cz = cell_coord(p.z[i], g.origin[2], g.inv_edge[2], g.dims[2]);
        c = g.cell_off + cx + g.dims[0] * (cy + g.dims[1] * cz);
    }
    const unsigned grp = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(&p.cell_count[c], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c >= 0) {
        p.atom_cell[i] = c;
        p.atom_rank[i] = base + __popc(grp & ((1u << lane) - 1u));
    }
}

// Single-CTA scan over all cells: unpadded starts, padded starts, and the
// super-cluster table (cell, first cluster, cluster count).  Each warp owns a
// contiguous run of cells and reads it 32 cells at a time (coalesced): a
// first pass sums the run, a scan over the 32 warps gives each run its base,
// and a second pass scans every 32-cell group with shuffles and writes.
__device__ __forceinline__ void cell_sizes(int n, int& pad, int& nsc)
{
    pad = (n + kClusterSize - 1) / kClusterSize * kClusterSize;
    nsc = (pad / kClusterSize + kSuperClusters - 1) / kSuperClusters;
}

// One block's part of the scan: cells [lo, hi), from the running totals
// base[0..2] (atoms, padded slots, super-clusters) of the cells before lo.
// Writes the unpadded and padded starts and the super-cluster table of those
// cells and clears their counts; leaves the block's totals in s_tot / s_base
// (warp kWarps-1's base plus total).  WRITE = false: only the totals.
template <bool WRITE>
__device__ __forceinline__ void scan_cells(const Params& p, int lo, int hi, const int base[3],
                                           int (*s_tot)[3], int (*s_base)[3])
{
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int kWarps = kScanThreads / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int run = ((hi - lo + kWarps - 1) / kWarps + 31) & ~31;
    const int c_lo = min(lo + warp * run, hi), c_hi = min(c_lo + run, hi);
    int tn = 0, tp = 0, ts = 0;
    for (int c = c_lo + lane; c < c_hi; c += 32) {
        const int n = p.cell_count[c];
        int pad, nsc;
        cell_sizes(n, pad, nsc);
        tn += n; tp += pad; ts += nsc;
    }
    for (int o = 16; o; o >>= 1) {
        tn += __shfl_xor_sync(kFull, tn, o);
        tp += __shfl_xor_sync(kFull, tp, o);
        ts += __shfl_xor_sync(kFull, ts, o);
    }
    if (lane == 0) { s_tot[warp][0] = tn; s_tot[warp][1] = tp; s_tot[warp][2] = ts; }
    __syncthreads();
    if (warp == 0) {   // exclusive scan of the runs' totals
        int v[3], inc[3];
        for (int k = 0; k < 3; ++k) v[k] = inc[k] = s_tot[lane][k];
        for (int o = 1; o < 32; o <<= 1)
            for (int k = 0; k < 3; ++k) {
                const int u = __shfl_up_sync(kFull, inc[k], o);
                if (lane >= o) inc[k] += u;
            }
        for (int k = 0; k < 3; ++k) s_base[lane][k] = base[k] + inc[k] - v[k];
    }
    __syncthreads();
    if (!WRITE) return;
    int bn = s_base[warp][0], bp = s_base[warp][1], bs = s_base[warp][2];
    for (int g0 = c_lo; g0 < c_hi; g0 += 32) {
        const int c = g0 + lane;
        const int n = c < c_hi ? p.cell_count[c] : 0;
        int pad, nsc;
        cell_sizes(n, pad, nsc);
        int in_ = n, ip = pad, is = nsc;   // inclusive scans over the group
        for (int o = 1; o < 32; o <<= 1) {
            const int un = __shfl_up_sync(kFull, in_, o), up = __shfl_up_sync(kFull, ip, o), us = __shfl_up_sync(kFull, is, o);
            if (lane >= o) { in_ += un; ip += up; is += us; }
        }
        if (c < c_hi) {
            const int on = bn + in_ - n, op = bp + ip - pad, os = bs + is - nsc;
            p.cell_start[c] = on;
            p.cell_pstart[c] = op;
            const int ncl = pad / kClusterSize;
            for (int k = 0; k < nsc; ++k)
                if (os + k < p.sc_cap) {
                    p.sc_cell[os + k] = c;
                    p.sc_first[os + k] = op / kClusterSize + k * kSuperClusters;
                    p.sc_ncl[os + k] = min(kSuperClusters, ncl - k * kSuperClusters);
                }
            p.cell_count[c] = 0;     // ready for the next build
        }
        bn += __shfl_sync(kFull, in_, 31);
        bp += __shfl_sync(kFull, ip, 31);
        bs += __shfl_sync(kFull, is, 31);
    }
}

// The scan's totals: the end of the last cell, the capacity check, the counters.
__device__ __forceinline__ void scan_cells_finish(const Params& p, int on, int op, int os)
{
    const int C = p.cell_cap_total;
    p.cell_start[C] = on;
    p.cell_pstart[C] = op;
    const bool over = op > p.slot_cap || os > p.sc_cap;
    if (over) atomicOr(p.err, ERR_CELL);
    p.counters[0] = over ? 0 : os;
    p.counters[1] = over ? 0 : op;
    p.counters[2] = 0;
    p.counters[4] = 0;   // cells too large for the one-warp sort
    p.counters[6] = 0;
    p.counters[7] = 0;
}

// The grid of this build stays with the list until the next build.
__device__ __forceinline__ void keep_build_grid(const Params& p)
{
    if (p.grid_b != p.grid)
        for (int r = threadIdx.x; r < p.n_rep; r += blockDim.x) p.grid_b[r] = p.grid[r];
}

// Single-CTA scan over all cells (grids of few cells): unpadded starts, padded
// starts, and the super-cluster table (cell, first cluster, cluster count).
// Each warp owns a contiguous run of cells and reads it 32 cells at a time
// (coalesced): a first pass sums the run, a scan over the 32 warps gives each
// run its base, and a second pass scans every 32-cell group with shuffles and
// writes.
__global__ void __launch_bounds__(kScanThreads) k_cell_scan(Params p)
{
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_tot[kWarps][3], s_base[kWarps][3];
    keep_build_grid(p);
    const int zero[3] = {0, 0, 0};
    scan_cells<true>(p, 0, p.cell_cap_total, zero, s_tot, s_base);
    if (threadIdx.x == 0)
        scan_cells_finish(p, s_base[kWarps - 1][0] + s_tot[kWarps - 1][0], s_base[kWarps - 1][1] + s_tot[kWarps - 1][1],
                          s_base[kWarps - 1][2] + s_tot[kWarps - 1][2]);
}

// The same scan over many CTAs (grids of many cells), in three kernels: each
// CTA sums its range of cells; one CTA scans those sums (and finishes); each
// CTA scans its range from its base.  p.scan_tmp holds [CTA][3] sums, then
// bases.
__device__ __forceinline__ void cta_range(int n, int& lo, int& hi)
{
    const int per = ((n + (int)gridDim.x - 1) / (int)gridDim.x + 31) & ~31;
    lo = min((int)blockIdx.x * per, n);
    hi = min(lo + per, n);
}
__global__ void __launch_bounds__(kScanThreads) k_cell_scan_sums(Params p)
{
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_tot[kWarps][3], s_base[kWarps][3];
    int lo, hi;
    cta_range(p.cell_cap_total, lo, hi);
    const int zero[3] = {0, 0, 0};
    scan_cells<false>(p, lo, hi, zero, s_tot, s_base);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) p.scan_tmp[3 * blockIdx.x + k] = s_base[kWarps - 1][k] + s_tot[kWarps - 1][k];
}
__global__ void __launch_bounds__(1024) k_cell_scan_top(Params p, int n_ctas)
{
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ int s_w[32][3];
    keep_build_grid(p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int v[3] = {0, 0, 0}, inc[3];
    if ((int)threadIdx.x < n_ctas)
        for (int k = 0; k < 3; ++k) v[k] = p.scan_tmp[3 * threadIdx.x + k];
    for (int k = 0; k < 3; ++k) inc[k] = v[k];
    for (int o = 1; o < 32; o <<= 1)
        for (int k = 0; k < 3; ++k) {
            const int u = __shfl_up_sync(kFull, inc[k], o);
            if (lane >= o) inc[k] += u;
        }
    if (lane == 31)
        for (int k = 0; k < 3; ++k) s_w[warp][k] = inc[k];
    __syncthreads();
    if (warp == 0) {
        int w[3], wi[3];
        for (int k = 0; k < 3; ++k) w[k] = wi[k] = s_w[lane][k];
        for (int o = 1; o < 32; o <<= 1)
            for (int k = 0; k < 3; ++k) {
                const int u = __shfl_up_sync(kFull, wi[k], o);
                if (lane >= o) wi[k] += u;
            }
        for (int k = 0; k < 3; ++k) s_w[lane][k] = wi[k] - w[k];
        if (lane == 31) scan_cells_finish(p, wi[0], wi[1], wi[2]);
    }
    __syncthreads();
    if ((int)threadIdx.x < n_ctas)
        for (int k = 0; k < 3; ++k) p.scan_tmp[3 * threadIdx.x + k] = s_w[warp][k] + inc[k] - v[k];
}
__global__ void __launch_bounds__(kScanThreads) k_cell_scan_apply(Params p)
{
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_tot[kWarps][3], s_base[kWarps][3];
    int lo, hi;
    cta_range(p.cell_cap_total, lo, hi);
    const int base[3] = {p.scan_tmp[3 * blockIdx.x], p.scan_tmp[3 * blockIdx.x + 1], p.scan_tmp[3 * blockIdx.x + 2]};
    scan_cells<true>(p, lo, hi, base, s_tot, s_base);
}

__global__ void __launch_bounds__(256) k_cell_scatter(Params p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_atoms) return;
    const int c = p.atom_cell[i];
    const Grid& g = p.grid[p.rep[i]];
    const int local = c - g.cell_off;
    const int cx = local % g.dims[0];
    const int cy = (local / g.dims[0]) % g.dims[1];
    const int cz = local / (g.dims[0] * g.dims[1]);
    // Hilbert index of the atom's sub-cell (16 per edge)
    unsigned sub[3];
    const double xs[3] = {p.x[i], p.y[i], p.z[i]};
    const int cc[3] = {cx, cy, cz};
    for (int d = 0; d < 3; ++d) {
        const double u = (xs[d] - (g.origin[d] + cc[d] * g.edge[d])) * g.inv_edge[d] * (double)(1 << kHilBits);
        const int sv = u >= 0.0 ? (int)u : 0;
        sub[d] = (unsigned)(sv < (1 << kHilBits) - 1 ? sv : (1 << kHilBits) - 1);
    }
    const unsigned key = hilbert3(sub[0], sub[1], sub[2]);
    if (p.xr) {   // reference positions of the Verlet-buffered list
        p.xr[i] = xs[0];
        p.yr[i] = xs[1];
        p.zr[i] = xs[2];
    }
    p.tmp_key[p.cell_start[c] + p.atom_rank[i]] = ((unsigned long long)key << 32) | (unsigned)i;
}

// One CTA per cell: rank sort of the cell's keys (Hilbert index, atom), with
// up to 8 threads sharing the count of one element; then the packed arrays
// and the cluster bounding boxes.  Launched with 1,024 threads when there are
// few cells per SM (large cells, all sorted at once) and 256 when there are
// many: a cell's phases are latency-bound, and seven 256-thread CTAs per SM
// keep more cells in flight than two 1,024-thread ones.
// Order-preserving integer image of a float (for min/max with integer atomics).
__device__ __forceinline__ int ord_f(float f)
{
    const int i = __float_as_int(f);
    return i < 0 ? i ^ 0x7fffffff : i;
}
__device__ __forceinline__ float unord_f(int i) { return __int_as_float(i < 0 ? i ^ 0x7fffffff : i); }

// small_max < 0: every cell; else only the cells k_cell_sort_small listed as
// larger than it could take (p.big_cells[0 .. counters[4])).
__global__ void __launch_bounds__(kSortThreads) k_cell_sort_pack(Params p, int small_max)
{
    const int nt = blockDim.x;
    __shared__ unsigned long long s_key[kSortMax];
    // cluster boxes of a cell held in shared memory (ordered-integer min x, y, z,
    // max x, y, z, min and max fragment), built with integer atomics as the
    // atoms are packed
    __shared__ int s_bb[kSortMax / kClusterSize][8];
    if (*p.err & ERR_CELL) return;
    const int tid = threadIdx.x;
    const int n_cells = small_max < 0 ? p.cell_cap_total : p.counters[4];
    for (int ci = blockIdx.x; ci < n_cells; ci += gridDim.x) {
        const int c = small_max < 0 ? ci : p.big_cells[ci];
        const int b = p.cell_start[c];
        const int n = p.cell_start[c + 1] - b;
        const int ps = p.cell_pstart[c];
        const int npad = p.cell_pstart[c + 1] - ps;
        if (npad == 0) continue;                      // uniform across the CTA
        int rr = 0;
        {
            // replicas own contiguous cell ranges; search by cell offset
            int lo = 0, hi = p.n_rep - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.grid[mid].cell_off <= c) lo = mid; else hi = mid - 1;
            }
            rr = lo;
        }
        const Grid& g = p.grid[rr];
        const int local = c - g.cell_off;
        const int cx = local % g.dims[0];
        const int cy = (local / g.dims[0]) % g.dims[1];
        const int cz = local / (g.dims[0] * g.dims[1]);
        const double cen[3] = {g.origin[0] + (cx + 0.5) * g.edge[0],
                               g.origin[1] + (cy + 0.5) * g.edge[1],
                               g.origin[2] + (cz + 0.5) * g.edge[2]};
        const bool in_smem = n <= kSortMax;
        const unsigned long long* keys = in_smem ? s_key : p.tmp_key + b;
        const int ncl = npad / kClusterSize;
        if (in_smem) {
            for (int e = tid; e < n; e += nt) s_key[e] = p.tmp_key[b + e];
            for (int k = tid; k < ncl; k += nt) {
                s_bb[k][0] = s_bb[k][1] = s_bb[k][2] = 0x7fffffff;
                s_bb[k][3] = s_bb[k][4] = s_bb[k][5] = (int)0x80000000;
                s_bb[k][6] = 0x7fffffff;
                s_bb[k][7] = (int)0x80000000;
            }
        }
        __syncthreads();
        int tpe = 1;
        while (tpe < 8 && 2 * tpe * n <= nt) tpe *= 2;
        const int per_pass = nt / tpe;
        const int sub = tid & (tpe - 1);
        for (int base = 0; base < n; base += per_pass) {
            const int e = base + tid / tpe;
            unsigned long long ke = 0;
            int rank = 0;
            if (e < n) {
                ke = keys[e];
                for (int f = sub; f < n; f += tpe) rank += keys[f] < ke;
            }
            for (int o = 1; o < tpe; o <<= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
            if (e < n && sub == 0) {
                const int i = (int)(ke & 0xffffffffu);
                const int slot = ps + rank;
                p.atom_of[slot] = i;
                p.slot_of[i] = slot;
                const float4 v = pack_slot(p, slot, i, cen, g);
                if (in_smem) {
                    int* bb = s_bb[rank / kClusterSize];
                    atomicMin(bb + 0, ord_f(v.x)); atomicMin(bb + 1, ord_f(v.y)); atomicMin(bb + 2, ord_f(v.z));
                    atomicMax(bb + 3, ord_f(v.x)); atomicMax(bb + 4, ord_f(v.y)); atomicMax(bb + 5, ord_f(v.z));
                    const int fr = p.frag[i];
                    atomicMin(bb + 6, fr);
                    atomicMax(bb + 7, fr);
                }
            }
        }
        for (int e = n + tid; e < npad; e += nt) {     // padding: far away, no charge
            const int slot = ps + e;
            const double far = 1.0e6 + 1024.0 * (double)slot;
            p.atom_of[slot] = -1;
            if (p.precision == 0) p.xq[slot] = make_float4((float)far, 1.0e6f, 1.0e6f, 0.0f);
            else p.xq64[slot] = make_double4_32a(far, 1.0e6, 1.0e6, 0.0);
            p.tf[slot] = make_int2(0, -1 - slot);
            p.fx[slot] = 0; p.fy[slot] = 0; p.fz[slot] = 0; p.epot[slot] = 0;
        }
        __syncthreads();
        // cluster bounding boxes (real atoms only) and fragment ranges
        if (in_smem) {
            for (int k = tid; k < ncl; k += nt) {
                const int cl = ps / kClusterSize + k;
                p.cl_cen[cl] = make_double4_32a(cen[0], cen[1], cen[2], 0.0);
                p.bb_lo[cl] = make_float4(unord_f(s_bb[k][0]), unord_f(s_bb[k][1]), unord_f(s_bb[k][2]), 0.0f);
                p.bb_hi[cl] = make_float4(unord_f(s_bb[k][3]), unord_f(s_bb[k][4]), unord_f(s_bb[k][5]), 0.0f);
                p.bb_frag[cl] = make_int2(s_bb[k][6], s_bb[k][7]);
            }
            __syncthreads();
            continue;
        }
        for (int k = tid; k < ncl; k += nt) {
            float lx = 3.0e38f, ly = 3.0e38f, lz = 3.0e38f, hx = -3.0e38f, hy = -3.0e38f, hz = -3.0e38f;
            int fmin = 0x7fffffff, fmax = (int)0x80000000;
            for (int a = 0; a < kClusterSize; ++a) {
                const int slot = ps + k * kClusterSize + a;
                if (a + k * kClusterSize >= n) break;
                float vx, vy, vz;
                if (p.precision == 0) {
                    const float4 t = p.xq[slot];
                    vx = t.x; vy = t.y; vz = t.z;
                } else {
                    const double4_32a t = p.xq64[slot];
                    vx = (float)t.x; vy = (float)t.y; vz = (float)t.z;
                }
                lx = fminf(lx, vx); hx = fmaxf(hx, vx);
                ly = fminf(ly, vy); hy = fmaxf(hy, vy);
                lz = fminf(lz, vz); hz = fmaxf(hz, vz);
                const int fr = p.tf[slot].y;
                fmin = min(fmin, fr);
                fmax = max(fmax, fr);
            }
            const int cl = ps / kClusterSize + k;
            p.cl_cen[cl] = make_double4_32a(cen[0], cen[1], cen[2], 0.0);
            p.bb_lo[cl] = make_float4(lx, ly, lz, 0.0f);
            p.bb_hi[cl] = make_float4(hx, hy, hz, 0.0f);
            p.bb_frag[cl] = make_int2(fmin, fmax);
        }
        __syncthreads();
    }
}

// Cells of up to kSmallCell atoms: one warp per cell, with the same rank sort,
// packed records and cluster boxes as k_cell_sort_pack but no block barrier,
// so that many more (latency-bound) cells are in flight.  Keys and boxes live
// in the warp's share of shared memory; every lane reads the cell's keys as
// broadcasts.
__global__ void __launch_bounds__(kSmallWarps * 32) k_cell_sort_small(Params p)
{
    __shared__ unsigned long long s_key[kSmallWarps][kSmallCell];
    __shared__ int s_bb[kSmallWarps][kSmallCell / kClusterSize][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*p.err & ERR_CELL) return;
    unsigned long long* key = s_key[warp];
    for (int c = blockIdx.x * kSmallWarps + warp; c < p.cell_cap_total; c += gridDim.x * kSmallWarps) {
        const int b = p.cell_start[c];
        const int n = p.cell_start[c + 1] - b;
        const int ps = p.cell_pstart[c];
        const int npad = p.cell_pstart[c + 1] - ps;
        if (npad == 0) continue;                     // uniform across the warp
        if (n > kSmallCell) {                        // left to k_cell_sort_pack
            if (lane == 0) p.big_cells[atomicAdd(&p.counters[4], 1)] = c;
            continue;
        }
        int lo = 0, hi = p.n_rep - 1;   // replicas own contiguous cell ranges
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.grid[mid].cell_off <= c) lo = mid; else hi = mid - 1;
        }
        const Grid& g = p.grid[lo];
        const int local = c - g.cell_off;
        const int cx = local % g.dims[0];
        const int cy = (local / g.dims[0]) % g.dims[1];
        const int cz = local / (g.dims[0] * g.dims[1]);
        const double cen[3] = {g.origin[0] + (cx + 0.5) * g.edge[0],
                               g.origin[1] + (cy + 0.5) * g.edge[1],
                               g.origin[2] + (cz + 0.5) * g.edge[2]};
        const int ncl = npad / kClusterSize;
        __syncwarp();
        for (int e = lane; e < n; e += 32) key[e] = p.tmp_key[b + e];
        for (int k = lane; k < ncl; k += 32) {
            int* bb = s_bb[warp][k];
            bb[0] = bb[1] = bb[2] = 0x7fffffff;
            bb[3] = bb[4] = bb[5] = (int)0x80000000;
            bb[6] = 0x7fffffff;
            bb[7] = (int)0x80000000;
        }
        __syncwarp();
        for (int e = lane; e < n; e += 32) {
            const unsigned long long ke = key[e];
            int rank = 0;
#pragma unroll 4
            for (int f = 0; f < n; ++f) rank += key[f] < ke;
            const int i = (int)(ke & 0xffffffffu);
            const int slot = ps + rank;
            p.atom_of[slot] = i;
            p.slot_of[i] = slot;
            const float4 v = pack_slot(p, slot, i, cen, g);
            int* bb = s_bb[warp][rank / kClusterSize];
            atomicMin(bb + 0, ord_f(v.x)); atomicMin(bb + 1, ord_f(v.y)); atomicMin(bb + 2, ord_f(v.z));
            atomicMax(bb + 3, ord_f(v.x)); atomicMax(bb + 4, ord_f(v.y)); atomicMax(bb + 5, ord_f(v.z));
            const int fr = p.frag[i];
            atomicMin(bb + 6, fr);
            atomicMax(bb + 7, fr);
        }
        for (int e = n + lane; e < npad; e += 32) {     // padding: far away, no charge
            const int slot = ps + e;
            const double far = 1.0e6 + 1024.0 * (double)slot;
            p.atom_of[slot] = -1;
            if (p.precision == 0) p.xq[slot] = make_float4((float)far, 1.0e6f, 1.0e6f, 0.0f);
            else p.xq64[slot] = make_double4_32a(far, 1.0e6, 1.0e6, 0.0);
            p.tf[slot] = make_int2(0, -1 - slot);
            p.fx[slot] = 0; p.fy[slot] = 0; p.fz[slot] = 0; p.epot[slot] = 0;
        }
        __syncwarp();
        for (int k = lane; k < ncl; k += 32) {
            const int* bb = s_bb[warp][k];
            const int cl = ps / kClusterSize + k;
            p.cl_cen[cl] = make_double4_32a(cen[0], cen[1], cen[2], 0.0);
            p.bb_lo[cl] = make_float4(unord_f(bb[0]), unord_f(bb[1]), unord_f(bb[2]), 0.0f);
            p.bb_hi[cl] = make_float4(unord_f(bb[3]), unord_f(bb[4]), unord_f(bb[5]), 0.0f);
            p.bb_frag[cl] = make_int2(bb[6], bb[7]);
        }
    }
}

// Between list builds: the packed records of the current positions and
// charges in the slots of the last build (cell centres and grid of that build).
__global__ void __launch_bounds__(256) k_refresh(Params p)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot == 0) p.counters[2] = 0;   // work counter of the force kernel that follows
    if (slot >= p.counters[1]) return;
    const int i = p.atom_of[slot];
    if (i < 0) {   // padding keeps its far-away record
        p.fx[slot] = 0; p.fy[slot] = 0; p.fz[slot] = 0; p.epot[slot] = 0;
        return;
    }
    const double4_32a c = p.cl_cen[slot / kClusterSize];
    const double cen[3] = {c.x, c.y, c.z};
    pack_slot(p, slot, i, cen, p.grid_b[p.rep[i]]);
}

void launch_refresh(const Params& p, cudaStream_t s)
{
    k_refresh<<<(p.slot_cap + 255) / 256, 256, 0, s>>>(p);
}

int launch_cells(const Params& p, cudaStream_t s, int grid_atoms, int grid_cells, int sort_threads)
{
    int n = 0;
    k_cell_assign<<<(p.slot_cap + 255) / 256, 256, 0, s>>>(p);
    if (p.cell_cap_total >= kScanCellsMulti) {
        const int ctas = std::min(kScanCtasMax, (p.cell_cap_total + 1023) / 1024);
        k_cell_scan_sums<<<ctas, kScanThreads, 0, s>>>(p);
        k_cell_scan_top<<<1, 1024, 0, s>>>(p, ctas);
        k_cell_scan_apply<<<ctas, kScanThreads, 0, s>>>(p);
        n += 4;
    } else {
        k_cell_scan<<<1, kScanThreads, 0, s>>>(p);
        n += 2;
    }
    k_cell_scatter<<<grid_atoms, 256, 0, s>>>(p);
    n += 1;
    // Grids of many cells (sorted by 256-thread CTAs): cells of up to kSmallCell
    // atoms one warp each, the rest one CTA each.  Grids of few, large cells:
    // every cell one 1,024-thread CTA.
    const int small_max = sort_threads <= 256 ? kSmallCell : -1;
    if (small_max > 0) {
        k_cell_sort_small<<<grid_cells, kSmallWarps * 32, 0, s>>>(p);
        n += 1;
    }
    k_cell_sort_pack<<<grid_cells, sort_threads, 0, s>>>(p, small_max);
    return n + 1;
}

}  // namespace mdg
