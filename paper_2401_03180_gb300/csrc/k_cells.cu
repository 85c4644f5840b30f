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
constexpr int kSortWarps = 8;
constexpr int kSortMax = 512;        // keys per cell kept in shared memory

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

__global__ void __launch_bounds__(256) k_cell_assign(Params p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_atoms) return;
    const Grid& g = p.grid[p.rep[i]];
    const int cx = cell_coord(p.x[i], g.origin[0], g.inv_edge[0], g.dims[0]);
    const int cy = cell_coord(p.y[i], g.origin[1], g.inv_edge[1], g.dims[1]);
    const int cz = cell_coord(p.z[i], g.origin[2], g.inv_edge[2], g.dims[2]);
    const int c = g.cell_off + cx + g.dims[0] * (cy + g.dims[1] * cz);
    p.atom_cell[i] = c;
    p.atom_rank[i] = atomicAdd(&p.cell_count[c], 1);
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

// One warp per cell: rank sort of the cell's keys, pack, bounding boxes.
__global__ void __launch_bounds__(kSortWarps * 32) k_cell_sort_pack(Params p)
{
    __shared__ unsigned long long s_key[kSortWarps][kSortMax];
    if (*p.err & ERR_CELL) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_warps = gridDim.x * kSortWarps;
    for (int c = blockIdx.x * kSortWarps + warp; c < p.cell_cap_total; c += n_warps) {
        const int b = p.cell_start[c];
        const int n = p.cell_start[c + 1] - b;
        const int ps = p.cell_pstart[c];
        const int npad = p.cell_pstart[c + 1] - ps;
        if (npad == 0) continue;
        // which replica / grid cell is this
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
        const unsigned long long* keys = in_smem ? s_key[warp] : p.tmp_key + b;
        if (in_smem)
            for (int e = lane; e < n; e += 32) s_key[warp][e] = p.tmp_key[b + e];
        __syncwarp();
        for (int e = lane; e < n; e += 32) {
            const unsigned long long ke = keys[e];
            int rank = 0;
            for (int f = 0; f < n; ++f) rank += keys[f] < ke;
            const int i = (int)(ke & 0xffffffffu);
            const int slot = ps + rank;
            p.atom_of[slot] = i;
            p.slot_of[i] = slot;
            const int s = p.species[i];
            const int qi = p.q[i];
            const double dx = p.x[i] - cen[0], dy = p.y[i] - cen[1], dz = p.z[i] - cen[2];
            if (p.precision == 0) p.xq[slot] = make_float4((float)dx, (float)dy, (float)dz, (float)qi);
            else p.xq64[slot] = make_double4_32a(dx, dy, dz, (double)qi);
            p.tf[slot] = make_int2(p.ts_off[s] + qi, p.frag[i]);
            p.fx[slot] = 0; p.fy[slot] = 0; p.fz[slot] = 0; p.epot[slot] = 0;
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
        __threadfence_block();
        // cluster bounding boxes (real atoms only) and fragment ranges
        const int ncl = npad / kClusterSize;
        for (int k = lane; k < ncl; k += 32) {
            float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
            int fmin = 0x7fffffff, fmax = (int)0x80000000;
            for (int a = 0; a < kClusterSize; ++a) {
                const int slot = ps + k * kClusterSize + a;
                if (a + k * kClusterSize >= n) break;
                float v[3];
                if (p.precision == 0) {
                    const float4 t = p.xq[slot];
                    v[0] = t.x; v[1] = t.y; v[2] = t.z;
                } else {
                    const double4_32a t = p.xq64[slot];
                    v[0] = (float)t.x; v[1] = (float)t.y; v[2] = (float)t.z;
                }
                for (int d = 0; d < 3; ++d) {
                    lo[d] = fminf(lo[d], v[d]);
                    hi[d] = fmaxf(hi[d], v[d]);
                }
                const int fr = p.tf[slot].y;
                fmin = min(fmin, fr);
                fmax = max(fmax, fr);
            }
            const int cl = ps / kClusterSize + k;
            p.bb_lo[cl] = make_float4(lo[0], lo[1], lo[2], 0.0f);
            p.bb_hi[cl] = make_float4(hi[0], hi[1], hi[2], 0.0f);
            p.bb_frag[cl] = make_int2(fmin, fmax);
        }
    }
}

void launch_cells(const Params& p, cudaStream_t s, int grid_atoms, int grid_cells)
{
    k_cell_assign<<<grid_atoms, 256, 0, s>>>(p);
    k_cell_scan<<<1, kScanThreads, 0, s>>>(p);
    k_cell_scatter<<<grid_atoms, 256, 0, s>>>(p);
    k_cell_sort_pack<<<grid_cells, kSortWarps * 32, 0, s>>>(p);
}

}  // namespace mdg
