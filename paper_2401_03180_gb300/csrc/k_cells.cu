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
#include "md_internal.cuh"

namespace mdg {

constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 1024;
constexpr int kSortMax = 2048;       // keys per cell kept in shared memory (larger cells sort from global memory)

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

__global__ void __launch_bounds__(kScanThreads) k_cell_scan(Params p)
{
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_tot[kWarps][3], s_base[kWarps][3];
    // the grid of this build stays with the list until the next build
    if (p.grid_b != p.grid)
        for (int r = threadIdx.x; r < p.n_rep; r += blockDim.x) p.grid_b[r] = p.grid[r];
    const int C = p.cell_cap_total;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int run = ((C + kWarps - 1) / kWarps + 31) & ~31;
    const int c_lo = min(warp * run, C), c_hi = min(c_lo + run, C);
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
        for (int k = 0; k < 3; ++k) s_base[lane][k] = inc[k] - v[k];
    }
    __syncthreads();
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
    if (threadIdx.x == 0) {
        const int on = s_base[kWarps - 1][0] + s_tot[kWarps - 1][0];
        const int op = s_base[kWarps - 1][1] + s_tot[kWarps - 1][1];
        const int os = s_base[kWarps - 1][2] + s_tot[kWarps - 1][2];
        p.cell_start[C] = on;
        p.cell_pstart[C] = op;
        const bool over = op > p.slot_cap || os > p.sc_cap;
        if (over) atomicOr(p.err, ERR_CELL);
        p.counters[0] = over ? 0 : os;
        p.counters[1] = over ? 0 : op;
        p.counters[2] = 0;
        p.counters[6] = 0;
        p.counters[7] = 0;
    }
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

__global__ void __launch_bounds__(kSortThreads) k_cell_sort_pack(Params p)
{
    const int nt = blockDim.x;
    __shared__ unsigned long long s_key[kSortMax];
    // cluster boxes of a cell held in shared memory (ordered-integer min x, y, z,
    // max x, y, z, min and max fragment), built with integer atomics as the
    // atoms are packed
    __shared__ int s_bb[kSortMax / kClusterSize][8];
    if (*p.err & ERR_CELL) return;
    const int tid = threadIdx.x;
    for (int c = blockIdx.x; c < p.cell_cap_total; c += gridDim.x) {
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

void launch_cells(const Params& p, cudaStream_t s, int grid_atoms, int grid_cells, int sort_threads)
{
    k_cell_assign<<<(p.slot_cap + 255) / 256, 256, 0, s>>>(p);
    k_cell_scan<<<1, kScanThreads, 0, s>>>(p);
    k_cell_scatter<<<grid_atoms, 256, 0, s>>>(p);
    k_cell_sort_pack<<<grid_cells, sort_threads, 0, s>>>(p);
}

}  // namespace mdg
