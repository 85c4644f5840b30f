// Cell-list neighbour build (one per step).  The paper's cutoff is chosen
// from the screening (Sec. II.B); here every replica gets a grid of cells of
// edge >= r_cut, atoms are counted per cell, the cells are scanned, and each
// cell is sorted deterministically (sub-cell Morton key, then atom index) into
// a padded slot range that is a multiple of the 8-atom cluster size.  The
// packed arrays hold FP32 (or FP64) coordinates relative to the cell centre,
// the charge, the type state and the fragment, plus one bounding box per
// cluster for the pair kernel's prefilter.
#include "md_internal.cuh"

namespace mdg {

constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 1024;
constexpr int kKdMax = 1024;         // atoms per cell ordered in shared memory

__device__ __forceinline__ int cell_coord(double x, double origin, double inv_edge, int n)
{
    double u = (x - origin) * inv_edge;
    int c = (u >= 0.0) ? (int)u : 0;   // NaN and negatives -> 0
    return c < n ? c : n - 1;
}

__device__ __forceinline__ unsigned spread3(unsigned v)   // 3 bits -> every third bit
{
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
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
// super-cluster table (cell, first cluster, cluster count).
__global__ void __launch_bounds__(kScanThreads) k_cell_scan(Params p)
{
    __shared__ int s_n[kScanThreads], s_p[kScanThreads], s_s[kScanThreads];
    const int C = p.cell_cap_total;
    const int t = threadIdx.x;
    const int chunk = (C + kScanThreads - 1) / kScanThreads;
    const int c0 = min(t * chunk, C), c1 = min(c0 + chunk, C);
    int sn = 0, sp = 0, ss = 0;
    for (int c = c0; c < c1; ++c) {
        const int n = p.cell_count[c];
        const int pad = (n + kClusterSize - 1) / kClusterSize * kClusterSize;
        const int ncl = pad / kClusterSize;
        sn += n;
        sp += pad;
        ss += (ncl + kSuperClusters - 1) / kSuperClusters;
    }
    s_n[t] = sn; s_p[t] = sp; s_s[t] = ss;
    __syncthreads();
    // Hillis-Steele inclusive scan over the per-thread sums
    for (int o = 1; o < kScanThreads; o <<= 1) {
        int an = 0, ap = 0, as = 0;
        if (t >= o) { an = s_n[t - o]; ap = s_p[t - o]; as = s_s[t - o]; }
        __syncthreads();
        s_n[t] += an; s_p[t] += ap; s_s[t] += as;
        __syncthreads();
    }
    int on = s_n[t] - sn, op = s_p[t] - sp, os = s_s[t] - ss;
    for (int c = c0; c < c1; ++c) {
        const int n = p.cell_count[c];
        const int pad = (n + kClusterSize - 1) / kClusterSize * kClusterSize;
        const int ncl = pad / kClusterSize;
        p.cell_start[c] = on;
        p.cell_pstart[c] = op;
        const int nsc = (ncl + kSuperClusters - 1) / kSuperClusters;
        for (int k = 0; k < nsc; ++k) {
            if (os + k < p.sc_cap) {
                p.sc_cell[os + k] = c;
                p.sc_first[os + k] = op / kClusterSize + k * kSuperClusters;
                p.sc_ncl[os + k] = min(kSuperClusters, ncl - k * kSuperClusters);
            }
        }
        on += n; op += pad; os += nsc;
        p.cell_count[c] = 0;     // ready for the next build
    }
    if (t == kScanThreads - 1) {
        p.cell_start[C] = on;
        p.cell_pstart[C] = op;
        const bool over = op > p.slot_cap || os > p.sc_cap;
        if (over) atomicOr(p.err, ERR_CELL);
        p.counters[0] = over ? 0 : os;
        p.counters[1] = over ? 0 : op;
        p.counters[2] = 0;
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
    // sub-cell (8 per edge) Morton key: spatially compact 8-atom clusters
    unsigned sub[3];
    const double xs[3] = {p.x[i], p.y[i], p.z[i]};
    const int cc[3] = {cx, cy, cz};
    for (int d = 0; d < 3; ++d) {
        double u = (xs[d] - (g.origin[d] + cc[d] * g.edge[d])) * g.inv_edge[d] * 8.0;
        int s = u >= 0.0 ? (int)u : 0;
        sub[d] = (unsigned)(s < 7 ? s : 7);
    }
    const unsigned key = spread3(sub[0]) | (spread3(sub[1]) << 1) | (spread3(sub[2]) << 2);
    p.tmp_key[p.cell_start[c] + p.atom_rank[i]] = ((unsigned long long)key << 32) | (unsigned)i;
}

// Segment of position e at bisection level `level` for a cell of n atoms:
// every segment longer than one cluster splits into a left part of
// ceil(len/16)*8 atoms (a whole number of clusters) and the rest.
__device__ __forceinline__ void kd_segment(int n, int level, int e, int& s, int& len)
{
    s = 0;
    len = n;
    for (int l = 0; l < level && len > kClusterSize; ++l) {
        const int left = (len + 2 * kClusterSize - 1) / (2 * kClusterSize) * kClusterSize;
        if (e < s + left) len = left;
        else { s += left; len -= left; }
    }
}

__device__ __forceinline__ int kd_levels(int n)
{
    int l = 0;
    for (int len = n; len > kClusterSize; len = (len + 2 * kClusterSize - 1) / (2 * kClusterSize) * kClusterSize) ++l;
    return l;
}

// One CTA per cell.  Atoms are ordered by recursive bisection (split each
// segment at a multiple of 8 along an axis that cycles through the cell's
// edges, longest first; ties broken by atom index) so that every run of 8
// slots is a compact, near-cubic cluster; then the packed arrays and the
// cluster bounding boxes are written.  Cells with
// more than kKdMax atoms fall back to a rank sort on (Morton sub-cell, atom).
__global__ void __launch_bounds__(kSortThreads) k_cell_sort_pack(Params p)
{
    __shared__ int s_idx[2][kKdMax];
    __shared__ float s_pos[2][3][kKdMax];
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
        int cur = 0;
        if (n <= kKdMax) {
            for (int e = tid; e < n; e += kSortThreads) {
                const int i = (int)(p.tmp_key[b + e] & 0xffffffffu);
                s_idx[0][e] = i;
                s_pos[0][0][e] = (float)(p.x[i] - cen[0]);
                s_pos[0][1][e] = (float)(p.y[i] - cen[1]);
                s_pos[0][2][e] = (float)(p.z[i] - cen[2]);
            }
            __syncthreads();
            // split axes cycle through the cell's edges, longest first
            int a0 = 0, a1 = 1, a2 = 2;
            if (g.edge[a1] > g.edge[a0]) { const int t = a0; a0 = a1; a1 = t; }
            if (g.edge[a2] > g.edge[a1]) { const int t = a1; a1 = a2; a2 = t; }
            if (g.edge[a1] > g.edge[a0]) { const int t = a0; a0 = a1; a1 = t; }
            // tpe threads share the rank count of one element
            int tpe = 1;
            while (tpe < 8 && 2 * tpe * n <= kSortThreads) tpe *= 2;
            const int per_pass = kSortThreads / tpe;
            const int sub = tid & (tpe - 1);
            const int levels = kd_levels(n);
            for (int level = 0; level < levels; ++level) {
                const int lm = level % 3;
                const int ax = lm == 0 ? a0 : (lm == 1 ? a1 : a2);
                const float* pa = s_pos[cur][ax];
                const int* ia = s_idx[cur];
                for (int base = 0; base < n; base += per_pass) {
                    const int e = base + tid / tpe;
                    int s0 = 0, len = 0, rank = 0;
                    if (e < n) {
                        kd_segment(n, level, e, s0, len);
                        if (len > kClusterSize) {
                            const float ve = pa[e];
                            const int ie = ia[e];
                            for (int f = s0 + sub; f < s0 + len; f += tpe) {
                                const float vf = pa[f];
                                rank += (vf < ve) || (vf == ve && ia[f] < ie);
                            }
                        }
                    }
                    for (int o = 1; o < tpe; o <<= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
                    if (e < n && sub == 0) {
                        const int dst = len > kClusterSize ? s0 + rank : e;
                        s_idx[cur ^ 1][dst] = ia[e];
                        s_pos[cur ^ 1][0][dst] = s_pos[cur][0][e];
                        s_pos[cur ^ 1][1][dst] = s_pos[cur][1][e];
                        s_pos[cur ^ 1][2][dst] = s_pos[cur][2][e];
                    }
                }
                __syncthreads();
                cur ^= 1;
            }
        }
        for (int e = tid; e < n; e += kSortThreads) {
            int i, pos = e;
            if (n <= kKdMax) {
                i = s_idx[cur][e];
            } else {   // fallback: rank by (Morton sub-cell, atom index) in global memory
                const unsigned long long ke = p.tmp_key[b + e];
                int rank = 0;
                for (int f = 0; f < n; ++f) rank += p.tmp_key[b + f] < ke;
                i = (int)(ke & 0xffffffffu);
                pos = rank;
            }
            const int slot = ps + pos;
            p.atom_of[slot] = i;
            p.slot_of[i] = slot;
            const int sp = p.species[i];
            const int qi = p.q[i];
            const double dx = p.x[i] - cen[0], dy = p.y[i] - cen[1], dz = p.z[i] - cen[2];
            if (p.precision == 0) p.xq[slot] = make_float4((float)dx, (float)dy, (float)dz, (float)qi);
            else p.xq64[slot] = make_double4_32a(dx, dy, dz, (double)qi);
            p.tf[slot] = make_int2(p.ts_off[sp] + qi, p.frag[i]);
            p.fx[slot] = 0; p.fy[slot] = 0; p.fz[slot] = 0; p.epot[slot] = 0;
        }
        for (int e = n + tid; e < npad; e += kSortThreads) {     // padding: far away, no charge
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
        const int ncl = npad / kClusterSize;
        for (int k = tid; k < ncl; k += kSortThreads) {
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
            p.bb_lo[cl] = make_float4(lx, ly, lz, 0.0f);
            p.bb_hi[cl] = make_float4(hx, hy, hz, 0.0f);
            p.bb_frag[cl] = make_int2(fmin, fmax);
        }
        __syncthreads();
    }
}

void launch_cells(const Params& p, cudaStream_t s, int grid_atoms, int grid_cells)
{
    k_cell_assign<<<(p.slot_cap + 255) / 256, 256, 0, s>>>(p);
    k_cell_scan<<<1, kScanThreads, 0, s>>>(p);
    k_cell_scatter<<<grid_atoms, 256, 0, s>>>(p);
    k_cell_sort_pack<<<grid_cells, kSortThreads, 0, s>>>(p);
}

}  // namespace mdg
