// Short-range non-bonded forces: Debye-screened Coulomb (Sec. II.A, Eq. 2)
// plus screened LJ (Sec. II.B, Eq. 8) with charge-scaled LJ sizes (Eq. 11),
// LJ excluded inside a native fragment (Sec. II.B), cut off at r_cut with the
// energy shifted to zero there.
//
// Work decomposition (Newton's third law, every unordered pair once):
//   * atoms are cell-sorted into clusters of 8; up to 8 consecutive clusters
//     of one cell form a super-cluster (SC);
//   * a list kernel tests, per SC and half-shell cell, every j-cluster's
//     bounding box against the SC's 8 i-cluster boxes, and for the clusters
//     in range every i-atom against the j-cluster's box; each j-cluster with
//     an i-atom in range becomes an entry (j-cluster, shift, 64-bit i-atom
//     mask), contiguous per SC and cut into chunks of kChunk entries;
//   * a warp of the force kernel owns one chunk at a time (dynamic scheduling
//     through an atomic counter);
//   * the SC's atoms and per-(atom, lane row) i-force partials live in shared
//     memory; lane (tx = lane & 7, ty = lane >> 3) takes atoms ty, ty+4 of the
//     entry's j-cluster and, tile by tile, the next i-cluster whose atom tx
//     is in the mask (its own queue), so a lane column always sees the same
//     slots in the same order and the shared-memory rows it touches never
//     share a bank with another column's;
//   * at the step of a Verlet-buffered build the evaluation also tests every
//     pair against r_cut + skin and drops from the mask the i-atoms with no
//     j-atom in range (exact for the list's lifetime), and clears the entry's
//     fragment flag when no pair in range lies within one fragment;
//   * forces are summed in FP32 (or FP64) within one chunk for the i side
//     and one (SC, j-cluster) entry for the j side, then converted
//     once to 64-bit fixed point (2^-32 kJ/mol/nm): the per-atom totals are
//     exact integer sums, identical for every launch shape and schedule.
#include <algorithm>
#include <type_traits>

#include "bonded_terms.cuh"
#include "md_internal.cuh"

namespace mdg {

template <bool FP64>
struct Prec;

template <>
struct Prec<false> {
    using T = float;
    using T4 = float4;         // global packed position + charge
    using S4 = float4;         // shared-memory copy
    using C2 = float2;         // -6 c6, -ln2 c12
    static __device__ __forceinline__ T4 pos(const Params& p, int slot) { return p.xq[slot]; }
    // single MUFU operations (arguments are far from the denormal range)
    static __device__ __forceinline__ T rsq(T x)
    {
        T y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ T expneg(T x)
    {
        T y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * -1.4426950408889634f));
        return y;
    }
    static __device__ __forceinline__ T exp2_(T x)
    {
        T y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ long long fix(T v) { return __float2ll_rn(v * 4294967296.0f); }
    static __device__ __forceinline__ bool fix_ok(T v) { return fabsf(v) < 1.0737418e9f; }
    static __device__ __forceinline__ const C2* table(const Params& p) { return p.lj_f; }
    static __device__ __forceinline__ S4 mk(T a, T b, T c, T d) { return make_float4(a, b, c, d); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __fmaf_rn(a, b, c); }
};

template <>
struct Prec<true> {
    using T = double;
    using T4 = double4_32a;
    using S4 = double4_16a;
    using C2 = double2;        // -6 c6, -ln2 c12
    static __device__ __forceinline__ T4 pos(const Params& p, int slot) { return p.xq64[slot]; }
    static __device__ __forceinline__ T rsq(T x) { return rsqrt(x); }   // within 1 ulp, without a division
    static __device__ __forceinline__ T expneg(T x) { return exp(-x); }
    static __device__ __forceinline__ T exp2_(T x) { return exp2(x); }
    static __device__ __forceinline__ long long fix(T v) { return __double2ll_rn(v * 4294967296.0); }
    static __device__ __forceinline__ bool fix_ok(T v) { return fabs(v) < 1.073741824e9; }
    static __device__ __forceinline__ const C2* table(const Params& p) { return p.lj_d; }
    static __device__ __forceinline__ S4 mk(T a, T b, T c, T d) { S4 s; s.x = a; s.y = b; s.z = c; s.w = d; return s; }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __fma_rn(a, b, c); }
};

// per-warp shared-memory layout; rows kSCAtoms + tx are far-away, uncharged
// stand-ins for lane column tx once its queue of i-clusters is used up
constexpr int kFiRow = kSCAtoms + kClusterSize;   // rows per lane row of the i-force partials
template <bool FP64, bool HYB>
struct HybSmem {};
template <bool FP64>
struct HybSmem<FP64, true> {                   // hybrid electrostatics (Eqs. 4-7)
    typename Prec<FP64>::S4 ih[kFiRow];        // (f/2) G_i, (f/2) q_i, q_i of the SC atoms
    typename Prec<FP64>::T jG[kChunk * kClusterSize];    // G_j of the chunk's j-atoms
};
template <bool FP64, bool HYB>
struct WarpSmem {
    typename Prec<FP64>::S4 ix[kFiRow];        // x, y, z, f*q of the SC atoms
    int2 it[kFiRow];                           // LJ row byte offset, fragment
    typename Prec<FP64>::S4 fi[4 * kFiRow];    // [ty][atom] force (+energy)
    typename Prec<FP64>::S4 jx[kChunk * kClusterSize];   // the chunk's j-atoms, shifted: x, y, z, q
    int2 jt[kChunk * kClusterSize];                      // their LJ column byte offset, fragment
    typename Prec<FP64>::T jqk[kChunk * kClusterSize];   // their q kappa
    PairEntry ent[kChunk];                               // the chunk's list entries
    HybSmem<FP64, HYB> hy;
};

// Hybrid electrostatics of one pair (Sec. II.A, Eqs. 4-7; the reading is in
// include/md.h): an ion's potential is q/r + c1 - c2 r^2 inside its
// transition radius r' and G e^{-kappa r}/r outside, and the pair's Coulomb
// energy f (q_j phi_i + q_i phi_j) / 2.
template <typename T>
struct HybArg {
    T hGi, hqi, qi;          // (f/2) G_i, (f/2) q_i, q_i
    T Gj, Gjk;               // G_j, G_j kappa
    T kap, c2, rpm2, hf;     // kappa, c2, (largest r')^2 of the replica, f/2
    const HybQ* rows;        // the replica's charge states
};

template <bool FP64>
__device__ __forceinline__ void red_fix(long long* dst, typename Prec<FP64>::T v, unsigned* err)
{
    if (!Prec<FP64>::fix_ok(v)) {
        atomicOr(err, ERR_OVERFLOW);
        return;
    }
    atomicAdd((unsigned long long*)dst, (unsigned long long)Prec<FP64>::fix(v));
}

// One pair, d = x_i - x_j.  `ok` drops the duplicates of the self-cluster
// diagonal; with EXCL equal fragments drop the LJ part (entries known to hold
// no such pair skip the test).  qjk = q_j * kappa, kl = -kappa log2(e).  The
// LJ table holds (-6 c6, -ln2 c12), so that t = kl r serves both the
// screening factor e^{-kappa r} = 2^t and the kappa r term of the LJ force
// (kappa r = -ln2 t).  The force on i is accumulated into (fx, fy, fz), the
// force on j into (fjx, fjy, fjz); with ENERGY the cutoff-shifted pair
// energy into u.  r2o returns |d|^2.  Multiply-adds are written out so that
// each accumulation is one fused operation.
template <bool FP64, bool ENERGY, bool EXCL, bool HYB>
__device__ __forceinline__ void pair(const typename Prec<FP64>::S4& xi, int row_off, int fri,
                                     typename Prec<FP64>::T xj, typename Prec<FP64>::T yj,
                                     typename Prec<FP64>::T zj, typename Prec<FP64>::T qj,
                                     typename Prec<FP64>::T qjk, int tsj_off, int frj, bool ok,
                                     const unsigned char* __restrict__ lj_bytes,
                                     typename Prec<FP64>::T kl, typename Prec<FP64>::T rc2,
                                     typename Prec<FP64>::T& fx, typename Prec<FP64>::T& fy,
                                     typename Prec<FP64>::T& fz, typename Prec<FP64>::T& fjx,
                                     typename Prec<FP64>::T& fjy, typename Prec<FP64>::T& fjz,
                                     typename Prec<FP64>::T& u, int& npair, typename Prec<FP64>::T erc,
                                     typename Prec<FP64>::T irc, typename Prec<FP64>::T& r2o,
                                     const HybArg<typename Prec<FP64>::T>& ha)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    constexpr T kLn2 = T(0.69314718055994530942);
    const T dx = xi.x - xj, dy = xi.y - yj, dz = xi.z - zj;
    const T r2 = P::fma(dz, dz, P::fma(dy, dy, dx * dx));
    r2o = r2;
    const bool in = (r2 < rc2) && ok;
    const T rinv = in ? P::rsq(r2) : T(0);
    const typename P::C2 c = *reinterpret_cast<const typename P::C2*>(lj_bytes + row_off + tsj_off);
    const T rinv2 = rinv * rinv;
    const T rinv6 = rinv2 * rinv2 * rinv2;
    const T lj6 = (EXCL && fri == frj) ? T(0) : rinv6;   // bonded in the native structure: no LJ
    const T r = r2 * rinv;
    const T t = kl * r;                         // -kappa r log2(e)
    const T e = P::exp2_(t);                    // e^{-kappa r}
    const T An = c.y * rinv6;                   // -ln2 c12/r^6
    const T Bn = P::fma(c.x, T(-kLn2 / 6), An); // -ln2 (c12/r^6 - c6)
    const T D6 = P::fma(An, T(-12 / kLn2), c.x);  // 12 c12/r^6 - 6 c6
    const T E1 = P::fma(t, Bn, D6);             // D6 + kappa r (c12/r^6 - c6)
    // f q_i q_j (1/r + kappa); hybrid, outside both transition radii:
    // (f/2)(G_i q_j + q_i G_j)(1/r + kappa)
    const T Cc = HYB ? P::fma(ha.hGi, P::fma(qj, rinv, qjk), ha.hqi * P::fma(ha.Gj, rinv, ha.Gjk))
                     : xi.w * P::fma(qj, rinv, qjk);
    const T S = P::fma(lj6, E1, Cc);
    T fs = S * (rinv2 * e);                     // F(r)/r
    if (HYB && in && r2 < ha.rpm2) {
        // inside some ion's transition radius: each ion's -phi' from its own form
        const HybQ& Ri = ha.rows[(int)ha.qi];
        const HybQ& Rj = ha.rows[(int)qj];
        const T rpi = FP64 ? T(Ri.rp) : T(Ri.rpf), rpj = FP64 ? T(Rj.rp) : T(Rj.rpf);
        const T Gj = ha.Gj;
        const T outf = e * P::fma(ha.kap, r, T(1)) * rinv2;   // e^{-kappa r} (1 + kappa r) / r^2
        const T fc2r = T(2) * ha.hf * ha.c2 * r;                // (f/2) 2 c2 r
        const T hmi = r < rpi ? P::fma(ha.hqi, rinv2, fc2r) : ha.hGi * outf;            // (f/2)(-phi_i')
        const T hmj = r < rpj ? P::fma(ha.hf * qj, rinv2, fc2r) : (ha.hf * Gj) * outf;  // (f/2)(-phi_j')
        fs = P::fma(lj6 * E1, rinv2 * e, P::fma(qj, hmi, ha.qi * hmj) * rinv);
    }
    const T nfs = -fs;
    fx = P::fma(fs, dx, fx); fy = P::fma(fs, dy, fy); fz = P::fma(fs, dz, fz);
    fjx = P::fma(nfs, dx, fjx); fjy = P::fma(nfs, dy, fjy); fjz = P::fma(nfs, dz, fjz);
    if (ENERGY) {
        if (in) {
            const T irc6 = irc * irc * irc * irc * irc * irc;
            const T lj_on = (EXCL && fri == frj) ? T(0) : T(1);
            const T ulj = e * (lj6 * (Bn * T(-1 / kLn2))) - erc * lj_on * (c.y * T(-1 / kLn2) * irc6 + c.x * T(1.0 / 6.0)) * irc6;
            if (HYB) {
                const HybQ& Ri = ha.rows[(int)ha.qi];
                const HybQ& Rj = ha.rows[(int)qj];
                const T rpi = FP64 ? T(Ri.rp) : T(Ri.rpf), rpj = FP64 ? T(Rj.rp) : T(Rj.rpf);
                const T c1i = FP64 ? T(Ri.c1) : T(Ri.c1f), c1j = FP64 ? T(Rj.c1) : T(Rj.c1f);
                const T Gi = FP64 ? T(Ri.G) : T(Ri.Gf);
                const T pci = FP64 ? T(Ri.phirc) : T(Ri.phircf), pcj = FP64 ? T(Rj.phirc) : T(Rj.phircf);
                const T cr2 = ha.c2 * r2;
                const T phi_i = r < rpi ? ha.qi * rinv + c1i - cr2 : Gi * e * rinv;
                const T phi_j = r < rpj ? qj * rinv + c1j - cr2 : ha.Gj * e * rinv;
                u += ulj + ha.hf * (qj * (phi_i - pci) + ha.qi * (phi_j - pcj));
            } else {
                const T qq = xi.w * qj;
                u += ulj + e * qq * rinv - erc * qq * irc;
            }
            npair += 1;
        }
    }
}

// Cluster-pair list.  Every j-cluster whose bounding box comes within
// r_cut + skin of at least one of a super-cluster's (SC's) i-cluster boxes gets
// an entry (j-cluster, half-shell index, mask of the i-atoms of those clusters
// that lie within r_cut + skin of the j-cluster's box).  An SC's entries are
// contiguous, in half-shell order and by j-cluster within a cell, and cut into
// chunks of kChunk, the work items of the force kernel.  The j-clusters of an
// SC's 14 half-shell cells form one index range, swept 32 at a time with every
// lane busy (cell by cell would leave lanes idle and chain one load latency per
// cell).  Three kernels, with no block-level barrier:
//   k_list_count  a warp per (SC, part of its index range) item counts the
//                 entries of its part;
//   k_list_scan   one block sums each SC's parts and scans the totals into
//                 entry and chunk offsets (and flags a list too small for them);
//   k_list_write  a warp per item repeats the box tests in the same rounding
//                 and writes its entries from its offset (the SC's plus the
//                 counts of the SC's earlier parts); the SC's first item writes
//                 the SC's chunk descriptors.
// An SC's range is split into 1, 2, 7 or 14 parts (list_parts): as few as keep
// every warp of the grid busy, so that a system of many SCs stages each SC once
// and a small one still spreads over the GPU.
struct ListWarp {
    float4 lo[kSuperClusters], hi[kSuperClusters];   // the SC's i-cluster boxes (cell frame)
    int2 fr[kSuperClusters];                          // fragment range of each i-cluster
    float4 ip[kSCAtoms];                              // the SC's atoms, [cluster k][atom a] (write pass)
};
constexpr int kListWarps = 8;
constexpr int kScanScsMulti = 32768;   // super-cluster capacities from this size are scanned by many CTAs

// An SC's cell, in the grid of its replica.
struct ListSC {
    int sc, fc, ncl, rr, cx, cy, cz;
};
__device__ __forceinline__ ListSC list_sc(const Params& p, int sc)
{
    ListSC s;
    s.sc = sc;
    const int c = p.sc_cell[sc];
    s.fc = p.sc_first[sc];
    s.ncl = p.sc_ncl[sc];
    int lo = 0, hi = p.n_rep - 1;   // replicas own contiguous cell ranges
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.grid_b[mid].cell_off <= c) lo = mid; else hi = mid - 1;
    }
    s.rr = lo;
    const Grid& g = p.grid_b[lo];
    const int local = c - g.cell_off;
    s.cx = local % g.dims[0];
    s.cy = (local / g.dims[0]) % g.dims[1];
    s.cz = local / (g.dims[0] * g.dims[1]);
    return s;
}

// Lane nb < 14: half-shell cell nb of the SC (its first j-cluster, its number
// of j-clusters, the clusters of the cells before it, its shift into the SC
// cell's frame); *total: the SC's j-clusters over the 14 cells.
struct ListCell {
    int jr0, n, pre;
    float Dx, Dy, Dz;
};
__device__ __forceinline__ ListCell list_cells(const Params& p, const ListSC& s, int lane, int* total)
{
    ListCell c{};
    if (lane < kHalfShell) {
        const Grid& g = p.grid_b[s.rr];
        int dx, dy, dz;
        half_shell(lane, dx, dy, dz);
        int ncx = s.cx + dx, ncy = s.cy + dy, ncz = s.cz + dz;
        bool valid = true;
        if (g.periodic) {
            ncx = ncx < 0 ? ncx + g.dims[0] : (ncx >= g.dims[0] ? ncx - g.dims[0] : ncx);
            ncy = ncy < 0 ? ncy + g.dims[1] : (ncy >= g.dims[1] ? ncy - g.dims[1] : ncy);
            ncz = ncz < 0 ? ncz + g.dims[2] : (ncz >= g.dims[2] ? ncz - g.dims[2] : ncz);
        } else {
            valid = ncx >= 0 && ncy >= 0 && ncz >= 0 && ncx < g.dims[0] && ncy < g.dims[1] && ncz < g.dims[2];
        }
        if (valid) {
            const int c2 = g.cell_off + ncx + g.dims[0] * (ncy + g.dims[1] * ncz);
            c.jr0 = lane == 0 ? s.fc : p.cell_pstart[c2] / kClusterSize;
            c.n = p.cell_pstart[c2 + 1] / kClusterSize - c.jr0;
        }
        c.Dx = (float)dx * g.edge_f[0];
        c.Dy = (float)dy * g.edge_f[1];
        c.Dz = (float)dz * g.edge_f[2];
    }
    int inc = c.n;   // inclusive scan over the 14 cells
    for (int o = 1; o < 16; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    c.pre = inc - c.n;
    *total = __shfl_sync(0xffffffffu, inc, kHalfShell - 1);
    return c;
}

// The cell (nb) and j-cluster of flat index idx of the SC's range (every lane
// takes part; lanes with idx out of range get some cell, unused).
__device__ __forceinline__ void list_locate(const ListCell& c, int idx, int& nb, int& jc, float& Dx, float& Dy,
                                            float& Dz)
{
    int lo = 0;   // the last cell whose first index is <= idx (cells of no cluster are skipped)
#pragma unroll
    for (int step = 8; step; step >>= 1) {
        const int cand = min(lo + step, kHalfShell - 1);
        if (__shfl_sync(0xffffffffu, c.pre, cand) <= idx) lo = cand;
    }
    nb = lo;
    jc = __shfl_sync(0xffffffffu, c.jr0, lo) + idx - __shfl_sync(0xffffffffu, c.pre, lo);
    Dx = __shfl_sync(0xffffffffu, c.Dx, lo);
    Dy = __shfl_sync(0xffffffffu, c.Dy, lo);
    Dz = __shfl_sync(0xffffffffu, c.Dz, lo);
}

// Largest of three floats in one instruction (max selects, so this equals
// fmaxf(c, fmaxf(a, b)) for the finite operands of the box tests).
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Mask of the SC's i-clusters whose boxes come within r_cut + skin of the
// j-cluster box [jl, jh] (already shifted into the SC's frame); in the SC's own
// cell (nb = 0) only i-clusters up to the j-cluster.  Explicit roundings, so
// that the count and the write pass reach the same masks.
__device__ __forceinline__ unsigned list_test(const ListWarp& w, int nb, int fc, int ncl, int jc, float4 jl,
                                              float4 jh, float rcb2)
{
    unsigned m = 0;
    const int kmax = nb == 0 ? min(ncl, jc - fc + 1) : ncl;
#pragma unroll 2
    for (int k = 0; k < kmax; ++k) {
        const float4 il = w.lo[k], ih = w.hi[k];
        const float gx = max3f(il.x - jh.x, jl.x - ih.x, 0.0f);
        const float gy = max3f(il.y - jh.y, jl.y - ih.y, 0.0f);
        const float gz = max3f(il.z - jh.z, jl.z - ih.z, 0.0f);
        if (__fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx))) < rcb2) m |= 1u << k;
    }
    return m;
}

// Parts of an SC's index range: the fewest of 1, 2, 7, 14 with at least as
// many (SC, part) items as the grid has warps.
__device__ __forceinline__ int list_parts(int n_sc)
{
    const long long warps = (long long)gridDim.x * kListWarps;
    if ((long long)n_sc >= warps) return 1;
    if (2LL * n_sc >= warps) return 2;
    if (7LL * n_sc >= warps) return 7;
    return 14;
}

// The box of flat index idx (when idx < i1), shifted into the SC's frame.
struct ListJ {
    int nb, jc;
    unsigned m;
    float4 jl, jh;
};
__device__ __forceinline__ ListJ list_j(const Params& p, const ListWarp& w, const ListSC& s, const ListCell& c,
                                        int idx, int i1, float rcb2)
{
    ListJ j;
    float Dx, Dy, Dz;
    list_locate(c, idx, j.nb, j.jc, Dx, Dy, Dz);
    j.m = 0u;
    j.jl = j.jh = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx < i1) {
        const float4 lo = p.bb_lo[j.jc], hi = p.bb_hi[j.jc];
        j.jl = make_float4(lo.x + Dx, lo.y + Dy, lo.z + Dz, 0.0f);
        j.jh = make_float4(hi.x + Dx, hi.y + Dy, hi.z + Dz, 0.0f);
        j.m = list_test(w, j.nb, s.fc, s.ncl, j.jc, j.jl, j.jh, rcb2);
    }
    return j;
}

__global__ void __launch_bounds__(kListWarps * 32, 4) k_list_count(Params p)
{
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ ListWarp s_w[kListWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ListWarp& w = s_w[warp];
    if (*p.err & ERR_CELL) return;
    const int n_sc = p.counters[0];
    const int G = list_parts(n_sc);
    const float rcb = list_rlist_f(p) + kBBoxMargin;   // r_cut + Verlet skin
    const float rcb2 = rcb * rcb;
    for (int item = blockIdx.x * kListWarps + warp; item < n_sc * G; item += gridDim.x * kListWarps) {
        const int sc = item / G, gr = item - sc * G;
        const ListSC s = list_sc(p, sc);
        int total;
        const ListCell c = list_cells(p, s, lane, &total);
        const int i0 = (int)((long long)total * gr / G), i1 = (int)((long long)total * (gr + 1) / G);
        __syncwarp();
        if (lane < s.ncl) {
            w.lo[lane] = p.bb_lo[s.fc + lane];
            w.hi[lane] = p.bb_hi[s.fc + lane];
        }
        __syncwarp();
        int cnt = 0;
        for (int base = i0; base < i1; base += 64) {   // two batches in flight
            const ListJ ja = list_j(p, w, s, c, base + lane, i1, rcb2);
            const ListJ jb = list_j(p, w, s, c, base + 32 + lane, i1, rcb2);
            cnt += __popc(__ballot_sync(kFull, ja.m != 0u)) + __popc(__ballot_sync(kFull, jb.m != 0u));
        }
        if (lane == 0) p.list_cnt[sc * kHalfShell + gr] = cnt;
        if (gr == 0 && lane >= G && lane < kHalfShell) p.list_cnt[sc * kHalfShell + lane] = 0;   // unused parts
    }
}

// Exclusive scans of the SCs' entry counts and chunk counts, each SC's total
// summed over its parts first (stored in sc_tot).  One block's part: SCs
// [lo, hi) from the running totals base[0..1] of the SCs before lo; each warp
// owns a contiguous run of SCs and reads it 32 at a time.  Leaves the block's
// totals in s_tot / s_base (warp 31's base plus total).  WRITE = false: the
// totals (and sc_tot) only.
template <bool WRITE>
__device__ __forceinline__ void scan_scs(const Params& p, int lo, int hi, const int base[2], int (*s_tot)[2],
                                         int (*s_base)[2])
{
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int kWarps = 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int run = ((hi - lo + kWarps - 1) / kWarps + 31) & ~31;
    const int s_lo = min(lo + warp * run, hi), s_hi = min(s_lo + run, hi);
    int te = 0, tc = 0;
    for (int s = s_lo + lane; s < s_hi; s += 32) {
        int t = 0;
        if (!WRITE) {
#pragma unroll
            for (int k = 0; k < kHalfShell; ++k) t += p.list_cnt[s * kHalfShell + k];
            p.sc_tot[s] = t;
        } else {
            t = p.sc_tot[s];
        }
        te += t;
        tc += (t + kChunk - 1) / kChunk;
    }
    for (int o = 16; o; o >>= 1) {
        te += __shfl_xor_sync(kFull, te, o);
        tc += __shfl_xor_sync(kFull, tc, o);
    }
    if (lane == 0) { s_tot[warp][0] = te; s_tot[warp][1] = tc; }
    __syncthreads();
    if (warp == 0) {
        int ie = s_tot[lane][0], ic = s_tot[lane][1];
        for (int o = 1; o < 32; o <<= 1) {
            const int ue = __shfl_up_sync(kFull, ie, o), uc = __shfl_up_sync(kFull, ic, o);
            if (lane >= o) { ie += ue; ic += uc; }
        }
        s_base[lane][0] = base[0] + ie - s_tot[lane][0];
        s_base[lane][1] = base[1] + ic - s_tot[lane][1];
    }
    __syncthreads();
    if (!WRITE) return;
    int be = s_base[warp][0], bc = s_base[warp][1];
    for (int g0 = s_lo; g0 < s_hi; g0 += 32) {
        const int s = g0 + lane;
        const int t = s < s_hi ? p.sc_tot[s] : 0;
        const int ch = (t + kChunk - 1) / kChunk;
        int ie = t, ic = ch;
        for (int o = 1; o < 32; o <<= 1) {
            const int ue = __shfl_up_sync(kFull, ie, o), uc = __shfl_up_sync(kFull, ic, o);
            if (lane >= o) { ie += ue; ic += uc; }
        }
        if (s < s_hi) {
            p.sc_eoff[s] = be + ie - t;
            p.sc_coff[s] = bc + ic - ch;
        }
        be += __shfl_sync(kFull, ie, 31);
        bc += __shfl_sync(kFull, ic, 31);
    }
}

// The list's totals into counters[6] (entries) and counters[7] (chunks),
// ERR_LIST when the list is too small for them.
__device__ __forceinline__ void scan_scs_finish(const Params& p, long long E, long long Cn)
{
    p.counters[6] = (int)min(E, (long long)0x7fffffff);
    p.counters[7] = (int)min(Cn, (long long)0x7fffffff);
    p.counters[2] = 0;   // work counter of the force kernel
    if (E > p.pl_cap || Cn > p.chunk_cap) atomicOr(p.err, ERR_LIST);
}

// Few SCs: one block does both passes.
__global__ void __launch_bounds__(1024) k_list_scan(Params p)
{
    __shared__ int s_tot[32][2], s_base[32][2];
    const int n = (*p.err & ERR_CELL) ? 0 : p.counters[0];
    const int zero[2] = {0, 0};
    scan_scs<false>(p, 0, n, zero, s_tot, s_base);
    scan_scs<true>(p, 0, n, zero, s_tot, s_base);
    if (threadIdx.x == 0)
        scan_scs_finish(p, (long long)s_base[31][0] + s_tot[31][0], (long long)s_base[31][1] + s_tot[31][1]);
}

// Many SCs: each CTA sums its range; one CTA scans the sums (and finishes);
// each CTA scans its range from its base (p.scan_tmp: [CTA][2]).
__device__ __forceinline__ void sc_cta_range(int n, int& lo, int& hi)
{
    const int per = ((n + (int)gridDim.x - 1) / (int)gridDim.x + 31) & ~31;
    lo = min((int)blockIdx.x * per, n);
    hi = min(lo + per, n);
}
__global__ void __launch_bounds__(1024) k_list_scan_sums(Params p)
{
    __shared__ int s_tot[32][2], s_base[32][2];
    const int n = (*p.err & ERR_CELL) ? 0 : p.counters[0];
    int lo, hi;
    sc_cta_range(n, lo, hi);
    const int zero[2] = {0, 0};
    scan_scs<false>(p, lo, hi, zero, s_tot, s_base);
    if (threadIdx.x == 0)
        for (int k = 0; k < 2; ++k) p.scan_tmp[2 * blockIdx.x + k] = s_base[31][k] + s_tot[31][k];
}
__global__ void __launch_bounds__(1024) k_list_scan_top(Params p, int n_ctas)
{
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ long long s_w[32][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long v[2] = {0, 0}, inc[2];
    if ((int)threadIdx.x < n_ctas)
        for (int k = 0; k < 2; ++k) v[k] = p.scan_tmp[2 * threadIdx.x + k];
    for (int k = 0; k < 2; ++k) inc[k] = v[k];
    for (int o = 1; o < 32; o <<= 1)
        for (int k = 0; k < 2; ++k) {
            const long long u = __shfl_up_sync(kFull, inc[k], o);
            if (lane >= o) inc[k] += u;
        }
    if (lane == 31)
        for (int k = 0; k < 2; ++k) s_w[warp][k] = inc[k];
    __syncthreads();
    if (warp == 0) {
        long long w[2], wi[2];
        for (int k = 0; k < 2; ++k) w[k] = wi[k] = s_w[lane][k];
        for (int o = 1; o < 32; o <<= 1)
            for (int k = 0; k < 2; ++k) {
                const long long u = __shfl_up_sync(kFull, wi[k], o);
                if (lane >= o) wi[k] += u;
            }
        for (int k = 0; k < 2; ++k) s_w[lane][k] = wi[k] - w[k];
        if (lane == 31) scan_scs_finish(p, wi[0], wi[1]);
    }
    __syncthreads();
    if ((int)threadIdx.x < n_ctas)
        for (int k = 0; k < 2; ++k) p.scan_tmp[2 * threadIdx.x + k] = (int)min(s_w[warp][k] + inc[k] - v[k], (long long)0x7fffffff);
}
__global__ void __launch_bounds__(1024) k_list_scan_apply(Params p)
{
    __shared__ int s_tot[32][2], s_base[32][2];
    const int n = (*p.err & ERR_CELL) ? 0 : p.counters[0];
    int lo, hi;
    sc_cta_range(n, lo, hi);
    const int base[2] = {p.scan_tmp[2 * blockIdx.x], p.scan_tmp[2 * blockIdx.x + 1]};
    scan_scs<true>(p, lo, hi, base, s_tot, s_base);
}

// Entry of one j-cluster: the i-atoms of the clusters in range that lie within
// r_cut + skin of the j-cluster's box (padding slots are far away), as a
// column-major mask (bit a*8 + k: atom a of i-cluster k), and whether an
// i-cluster in range may share a fragment with it.  The i-atoms are broadcast
// reads of the staged SC.
__device__ __forceinline__ uint4 list_entry(const Params& p, const ListWarp& w, const ListJ& j, unsigned any_m,
                                            float rcb2)
{
    const int2 jfr = j.m ? p.bb_frag[j.jc] : make_int2(0, 0);
    unsigned mlo = 0u, mhi = 0u;
    bool share = false;
#pragma unroll
    for (int k = 0; k < kSuperClusters; ++k) {
        if (!((any_m >> k) & 1u)) continue;   // no lane has i-cluster k in range
        const bool kin = (j.m >> k) & 1u;
        unsigned klo = 0u, khi = 0u;   // column k's bits, kept only if cluster k is in range
#pragma unroll
        for (int a = 0; a < kClusterSize; ++a) {
            const float4 xi = w.ip[k * kClusterSize + a];
            const float gx = max3f(xi.x - j.jh.x, j.jl.x - xi.x, 0.0f);
            const float gy = max3f(xi.y - j.jh.y, j.jl.y - xi.y, 0.0f);
            const float gz = max3f(xi.z - j.jh.z, j.jl.z - xi.z, 0.0f);
            const bool in = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx))) < rcb2;
            if (a < 4) klo |= (in ? 1u : 0u) << (a * 8 + k);
            else khi |= (in ? 1u : 0u) << ((a - 4) * 8 + k);
        }
        if (kin) {
            mlo |= klo;
            mhi |= khi;
        }
        const int2 ifr = w.fr[k];
        share |= kin && !(ifr.y < jfr.x || jfr.y < ifr.x);
    }
    return make_uint4((unsigned)j.jc, (unsigned)j.nb | (share ? kEntryExcl : 0u), mlo, mhi);
}

__global__ void __launch_bounds__(kListWarps * 32, 4) k_list_write(Params p)
{
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ ListWarp s_w[kListWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ListWarp& w = s_w[warp];
    if (*p.err & (ERR_CELL | ERR_LIST)) return;
    const int n_sc = p.counters[0];
    const int G = list_parts(n_sc);
    const float rcb = list_rlist_f(p) + kBBoxMargin;
    const float rcb2 = rcb * rcb;
    for (int item = blockIdx.x * kListWarps + warp; item < n_sc * G; item += gridDim.x * kListWarps) {
        const int sc = item / G, gr = item - sc * G;
        const int tot = p.sc_tot[sc];
        if (tot == 0) continue;
        const ListSC s = list_sc(p, sc);
        const int e0 = p.sc_eoff[sc], c0 = p.sc_coff[sc];
        if (gr == 0)
            for (int t = lane; t * kChunk < tot; t += 32)
                p.pl_chunk[c0 + t] = make_int4(sc, e0 + t * kChunk, min(kChunk, tot - t * kChunk), s.rr);
        // this item's first entry: the SC's offset plus the counts of its earlier parts
        const int cnt_l = lane < G ? p.list_cnt[sc * kHalfShell + lane] : 0;
        int pre = lane < gr ? cnt_l : 0;
        for (int o = 16; o; o >>= 1) pre += __shfl_xor_sync(kFull, pre, o);
        const int mine = __shfl_sync(kFull, cnt_l, gr);
        if (mine == 0) continue;
        int total;
        const ListCell c = list_cells(p, s, lane, &total);
        const int i0 = (int)((long long)total * gr / G), i1 = (int)((long long)total * (gr + 1) / G);
        __syncwarp();
        if (lane < s.ncl) {
            w.lo[lane] = p.bb_lo[s.fc + lane];
            w.hi[lane] = p.bb_hi[s.fc + lane];
            w.fr[lane] = p.bb_frag[s.fc + lane];
        }
        for (int a = lane; a < kSCAtoms; a += 32) {
            // slot order (cluster k, atom a); absent clusters far away
            float4 v = make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.0f);
            if ((a >> 3) < s.ncl) {
                const int slot = s.fc * kClusterSize + a;
                if (p.precision == 0) {
                    v = p.xq[slot];
                } else {
                    const double4_32a t = p.xq64[slot];
                    v = make_float4((float)t.x, (float)t.y, (float)t.z, 0.0f);
                }
            }
            w.ip[a] = v;
        }
        __syncwarp();
        int off = e0 + pre;
        const int end = off + mine;
        for (int base = i0; base < i1; base += 32) {
            const ListJ j = list_j(p, w, s, c, base + lane, i1, rcb2);
            const unsigned bal = __ballot_sync(kFull, j.m != 0u);
            const int at = off + __popc(bal & ((1u << lane) - 1u));
            const uint4 e = list_entry(p, w, j, __reduce_or_sync(kFull, j.m), rcb2);
            if (j.m && at < end) p.pl[at] = e;
            off += __popc(bal);
        }
        // both passes see the same boxes and round identically, so `off` ends at
        // `end`; should it fall short, pad with empty entries (a real cluster, no
        // i-atom in range) rather than leave slots unwritten
        for (int at = off + lane; at < end; at += 32) p.pl[at] = make_uint4((unsigned)s.fc, 0u, 0u, 0u);
    }
}

// Forces over the cluster-pair list.  A warp takes one chunk (up to kChunk
// entries of one SC) at a time from an atomic counter.  Blocks of 4, 8 or 12
// warps (the FP32 bounds keep 85 registers per thread either way: three
// 8-warp or two 12-warp blocks per SM); each block holds its own copy of the
// LJ table, so with many type states the 12-warp shape keeps more warps
// resident than the shared memory allows 8-warp blocks.
template <bool FP64, bool ENERGY, bool HYB>
__global__ void __launch_bounds__(FP64 ? 256 : 384, 2) k_pair(Params p)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    using T4 = typename P::T4;
    using S4 = typename P::S4;
    using C2 = typename P::C2;
    using WS = WarpSmem<FP64, HYB>;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nts = p.n_ts_lj;
    C2* s_lj = reinterpret_cast<C2*>(smem);
    const unsigned char* lj_bytes = smem;
    const size_t tab = ((size_t)nts * nts * sizeof(C2) + 127) / 128 * 128;
    // s_kq[c]: the set bits of the 8-bit column mask c as 4-bit cluster indices,
    // lowest first, the unused nibbles 8 (a column's stand-in row)
    unsigned* s_kq = reinterpret_cast<unsigned*>(smem + tab);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WS& w = reinterpret_cast<WS*>(smem + tab + 256 * sizeof(unsigned))[warp];

    for (int k = threadIdx.x; k < nts * nts; k += blockDim.x) s_lj[k] = P::table(p)[k];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) {
        unsigned q = 0x88888888u;
        int n = 0;
        for (int k = 0; k < 8; ++k)
            if ((c >> k) & 1) {
                q = (q & ~(0xfu << (4 * n))) | ((unsigned)k << (4 * n));
                ++n;
            }
        s_kq[c] = q;
    }
    for (int k = lane; k < 4 * kFiRow; k += 32) w.fi[k] = P::mk(T(0), T(0), T(0), T(0));
    if (lane < kClusterSize) {
        w.ix[kSCAtoms + lane] = P::mk(T(-1.0e6), T(-1.0e6), T(-1.0e6), T(0));
        w.it[kSCAtoms + lane] = make_int2(0, (int)0x80000000);
        if constexpr (HYB) w.hy.ih[kSCAtoms + lane] = P::mk(T(0), T(0), T(0), T(0));
    }
    __syncthreads();
    if (*p.err & (ERR_CELL | ERR_LIST)) return;

    // bonded terms (Sec. II.B, Eqs. 9-10), one per thread over the grid before
    // the chunks: their dependent loads overlap the other warps' pair work, and
    // they add to the same fixed-point sums
    if (p.n_bonds + p.n_angles > 0) {
        const T* bp;
        const T* ap;
        if constexpr (FP64) { bp = p.bond_pd; ap = p.angle_pd; }
        else { bp = p.bond_pf; ap = p.angle_pf; }
        const int nb = p.n_bonds, nt = p.n_bonds + p.n_angles;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
            if (t < nb) bonded::bond_term<T, ENERGY>(p, bp, t);
            else bonded::angle_term<T, ENERGY>(p, ap, t - nb);
        }
    }

    const int tx = lane & 7, ty = lane >> 3;
    const int n_chunks = min(p.counters[7], p.chunk_cap);
    // after the j-force reduction lane (tx, ty) holds component tx & 3 of atom
    // ty (tx < 4) or ty + 4 (tx >= 4) of the entry's j-cluster
    const int comp = tx & 3;
    long long* const jdst = comp == 0 ? p.fx : (comp == 1 ? p.fy : p.fz);
    // In the step of a Verlet-buffered build the positions are the build's:
    // i-atoms with no j-atom within r_cut + skin are dropped from an entry's
    // mask for the list's lifetime (they cannot come within r_cut before the
    // next build), and so is the fragment flag of an entry with no pair in
    // range inside one fragment.  Lane column tx always takes the atoms tx of
    // the entry's i-clusters in cluster order, so the dropped atoms only ever
    // added exact zeros: every sum comes out bit-identical with either mask.
    const bool prune = p.builds != nullptr && list_half_skin2(p) > 0.0f && p.builds[1] != 0;
    const float rlb = list_rlist_f(p) + kBBoxMargin;
    const T rl2 = T(rlb) * T(rlb);
    const T rc2 = FP64 ? T(p.rc2) : T(p.rc2_f);
    const T irc = T(1.0 / p.r_cut);
    const T coulf = T(p.coulomb_f);

    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.counters[2], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_chunks) break;
        const int4 ch = p.pl_chunk[item];          // (sc, first entry, entries, replica)
        const int sc = ch.x, n_ent = ch.z, rr = ch.w;
        __syncwarp();   // the previous chunk's reads of the staged entries are done
        if (lane < n_ent) w.ent[lane] = p.pl[ch.y + lane];
        const int fc = p.sc_first[sc], ncl = p.sc_ncl[sc];
        const Grid& g = p.grid_b[rr];
        const T kap = FP64 ? T(p.rs[rr].kappa_force) : T(p.rs[rr].kappa_f);
        const T kl = kap * T(-1.4426950408889634);   // -kappa log2(e)
        const T erc = ENERGY ? P::expneg(kap * T(p.r_cut)) : T(0);
        HybArg<T> ha{};
        const HybQ* hrows = nullptr;
        if constexpr (HYB) {
            hrows = p.hq + (size_t)rr * kHybQ;
            const HybRep hr = p.hrep[rr];
            ha.kap = kap;
            ha.c2 = FP64 ? T(hr.c2) : T(hr.c2f);
            ha.rpm2 = FP64 ? T(hr.rpm2) : T(hr.rpm2f);
            ha.hf = T(0.5) * coulf;
            ha.rows = hrows;
        }

        // the super-cluster's atoms and the chunk's j-atoms (shifted into the
        // SC's cell frame) into shared memory: one load latency per chunk
        // instead of one per entry
        __syncwarp();
        for (int a = lane; a < kSCAtoms; a += 32) {
            if ((a >> 3) < ncl) {
                const int slot = fc * kClusterSize + a;
                const T4 v = P::pos(p, slot);
                const int2 t = p.tf[slot];
                w.ix[a] = P::mk(v.x, v.y, v.z, coulf * v.w);
                w.it[a] = make_int2(t.x * nts * (int)sizeof(C2), t.y);   // byte offset of the LJ row
                if constexpr (HYB) {
                    const HybQ& hq = hrows[(int)v.w];
                    const T G = FP64 ? T(hq.G) : T(hq.Gf);
                    w.hy.ih[a] = P::mk(T(0.5) * coulf * G, T(0.5) * coulf * v.w, v.w, T(0));
                }
            }
        }
        for (int a0 = 0; a0 < kChunk * kClusterSize; a0 += 32) {
            const int a = a0 + lane, e = a >> 3;                 // entry e, atom a & 7
            if (e < n_ent) {
                const unsigned jc = w.ent[e].x, cd = w.ent[e].y;
                int dx, dy, dz;
                half_shell((int)(cd & 0xffu), dx, dy, dz);
                const int slot = (int)jc * kClusterSize + (a & 7);
                const T4 v = P::pos(p, slot);
                const int2 t = p.tf[slot];
                if (FP64) w.jx[a] = P::mk(v.x + T(dx * g.edge[0]), v.y + T(dy * g.edge[1]), v.z + T(dz * g.edge[2]), v.w);
                else w.jx[a] = P::mk(v.x + T((float)dx * g.edge_f[0]), v.y + T((float)dy * g.edge_f[1]),
                                     v.z + T((float)dz * g.edge_f[2]), v.w);
                w.jt[a] = make_int2(t.x * (int)sizeof(C2), t.y);   // byte offset of the LJ column
                w.jqk[a] = v.w * kap;
                if constexpr (HYB) {
                    const HybQ& hq = hrows[(int)v.w];
                    w.hy.jG[a] = FP64 ? T(hq.G) : T(hq.Gf);
                }
            }
        }
        __syncwarp();
        int npair = 0;

        for (int v = 0; v < n_ent; ++v) {
            const PairEntry e4 = w.ent[v];   // one broadcast read
            const int jcl = (int)e4.x;
            const unsigned code = e4.y;
            const int nb = (int)(code & 0xffu);
            const bool excl = (code & kEntryExcl) != 0u;
            const unsigned mlo = e4.z, mhi = e4.w;
            if ((mlo | mhi) == 0u) continue;   // no i-atom in range (or emptied by pruning)
            const int s0 = jcl * kClusterSize + ty, s1 = s0 + 4;
            const S4 a0 = w.jx[v * kClusterSize + ty], a1 = w.jx[v * kClusterSize + ty + 4];
            const int2 t0 = w.jt[v * kClusterSize + ty], t1 = w.jt[v * kClusterSize + ty + 4];
            const T x0 = a0.x, y0 = a0.y, z0 = a0.z;
            const T x1 = a1.x, y1 = a1.y, z1 = a1.z;
            const T q0k = w.jqk[v * kClusterSize + ty], q1k = w.jqk[v * kClusterSize + ty + 4];
            const int j0off = t0.x, j1off = t1.x;
            HybArg<T> h0 = ha, h1 = ha;   // the j-atom halves of the hybrid arguments
            if constexpr (HYB) {
                h0.Gj = w.hy.jG[v * kClusterSize + ty];
                h1.Gj = w.hy.jG[v * kClusterSize + ty + 4];
                h0.Gjk = h0.Gj * kap;
                h1.Gjk = h1.Gj * kap;
            }
            const int kdiag = nb == 0 ? jcl - fc : -1;   // i-cluster equal to this j-cluster

            // this lane column's i-clusters (byte tx of the column-major mask: bit k
            // when atom tx of i-cluster k is in); a tile takes the next one of every column
            const unsigned col0 = __byte_perm(mlo, mhi, (unsigned)tx) & 0xffu;   // byte tx of (mhi:mlo)
            const int n_t = (int)__reduce_max_sync(kFull, (unsigned)__popc(col0));

            T fj0x = 0, fj0y = 0, fj0z = 0, fj1x = 0, fj1y = 0, fj1z = 0;
            unsigned keep = 0u;   // PRUNE: i-clusters whose atom tx has a j-atom of this lane in range
            bool share = false;   // PRUNE: a pair in range within one fragment
            // DIAG: the self-cluster diagonal (i < j inside the cluster); EXCL:
            // pairs within one fragment are possible; PRUNE: build step
            auto tiles = [&](auto diag, auto ex, auto pr) {
                constexpr bool DIAG = decltype(diag)::value;
                constexpr bool EXCL = DIAG || decltype(ex)::value;
                constexpr bool PRUNE = decltype(pr)::value;
                unsigned kq = s_kq[col0];
                for (int t = 0; t < n_t; ++t) {
                    const int k = (int)(kq & 0xfu);   // 8 once the column is used up
                    kq >>= 4;
                    const int ia = k * kClusterSize + tx;   // k = 8: the stand-in row
                    const S4 xi = w.ix[ia];
                    const int2 ti = w.it[ia];
                    S4 acc = w.fi[ty * kFiRow + ia];
                    bool ok0 = true, ok1 = true;
                    if (DIAG) {
                        const bool dg = k == kdiag;
                        ok0 = !dg || tx < ty;
                        ok1 = !dg || tx < ty + 4;
                    }
                    T r20, r21;
                    if constexpr (HYB) {
                        const S4 hi = w.hy.ih[ia];
                        h0.hGi = h1.hGi = hi.x;
                        h0.hqi = h1.hqi = hi.y;
                        h0.qi = h1.qi = hi.z;
                    }
                    pair<FP64, ENERGY, EXCL, HYB>(xi, ti.x, ti.y, x0, y0, z0, a0.w, q0k, j0off, t0.y, ok0, lj_bytes, kl,
                                                  rc2, acc.x, acc.y, acc.z, fj0x, fj0y, fj0z, acc.w, npair, erc, irc,
                                                  r20, h0);
                    pair<FP64, ENERGY, EXCL, HYB>(xi, ti.x, ti.y, x1, y1, z1, a1.w, q1k, j1off, t1.y, ok1, lj_bytes, kl,
                                                  rc2, acc.x, acc.y, acc.z, fj1x, fj1y, fj1z, acc.w, npair, erc, irc,
                                                  r21, h1);
                    w.fi[ty * kFiRow + ia] = acc;
                    if (PRUNE) {   // this lane's pairs in range: combined over the warp after the entry
                        const bool n0 = ok0 && r20 < rl2, n1 = ok1 && r21 < rl2;
                        if (n0 || n1) keep |= 1u << k;   // never for the far stand-in row
                        if (EXCL) share |= (n0 && ti.y == t0.y) || (n1 && ti.y == t1.y);
                    }
                }
            };
            if (prune) {
                if ((unsigned)kdiag < (unsigned)ncl) tiles(std::true_type{}, std::true_type{}, std::true_type{});
                else if (excl) tiles(std::false_type{}, std::true_type{}, std::true_type{});
                else tiles(std::false_type{}, std::false_type{}, std::true_type{});
                // columns back to the column-major mask (byte tx: the OR over the
                // column's four lane rows), and any pair in range within a fragment
                const unsigned klo = __reduce_or_sync(kFull, tx < 4 ? keep << ((tx & 3) * 8) : 0u);
                const unsigned khi = __reduce_or_sync(kFull, tx >= 4 ? keep << ((tx & 3) * 8) : 0u);
                share = __any_sync(kFull, share);
                if (lane == 0) {
                    if (klo != mlo || khi != mhi)
                        *reinterpret_cast<uint2*>(&p.pl[ch.y + v].z) = make_uint2(klo, khi);
                    if (share != excl) p.pl[ch.y + v].y = (unsigned)nb | (share ? kEntryExcl : 0u);
                }
            } else {
                if ((unsigned)kdiag < (unsigned)ncl) tiles(std::true_type{}, std::true_type{}, std::false_type{});
                else if (excl) tiles(std::false_type{}, std::true_type{}, std::false_type{});
                else tiles(std::false_type{}, std::false_type{}, std::false_type{});
            }
            // j forces: sum over the 8 i-lanes of each ty group.  Lanes tx < 4 keep
            // atom ty (j0), lanes tx >= 4 atom ty + 4 (j1); then each lane holds one
            // component of one atom and issues one RED.
            {
                const bool up = tx >= 4;
                T ax = up ? fj1x : fj0x, ay = up ? fj1y : fj0y, az = up ? fj1z : fj0z;
                ax += __shfl_xor_sync(kFull, up ? fj0x : fj1x, 4);
                ay += __shfl_xor_sync(kFull, up ? fj0y : fj1y, 4);
                az += __shfl_xor_sync(kFull, up ? fj0z : fj1z, 4);
#pragma unroll
                for (int o = 1; o < 4; o <<= 1) {
                    ax += __shfl_xor_sync(kFull, ax, o);
                    ay += __shfl_xor_sync(kFull, ay, o);
                    az += __shfl_xor_sync(kFull, az, o);
                }
                if (comp < 3) {
                    const T v3 = comp == 0 ? ax : (comp == 1 ? ay : az);
                    red_fix<FP64>(jdst + (up ? s1 : s0), v3, p.err);
                }
            }
        }
        __syncwarp();
        // i forces of this chunk: sum the 4 ty partials of each atom, clearing
        // them for the next chunk (tiles touch only the rows of the SC's
        // clusters, which this loop covers, and the stand-in rows, which stay 0)
        for (int a = lane; a < ncl * kClusterSize; a += 32) {
            S4 sum = w.fi[a];
            w.fi[a] = P::mk(T(0), T(0), T(0), T(0));
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                const S4 v = w.fi[q * kFiRow + a];
                w.fi[q * kFiRow + a] = P::mk(T(0), T(0), T(0), T(0));
                sum.x += v.x; sum.y += v.y; sum.z += v.z;
                if (ENERGY) sum.w += v.w;
            }
            const int slot = fc * kClusterSize + a;
            red_fix<FP64>(p.fx + slot, sum.x, p.err);
            red_fix<FP64>(p.fy + slot, sum.y, p.err);
            red_fix<FP64>(p.fz + slot, sum.z, p.err);
            if (ENERGY) red_fix<FP64>(p.epot + slot, sum.w, p.err);
        }
        __syncwarp();
        if (ENERGY) {
#pragma unroll
            for (int o = 16; o; o >>= 1) npair += __shfl_xor_sync(kFull, npair, o);
            if (lane == 0 && npair) atomicAdd((unsigned long long*)p.pair_count, (unsigned long long)npair);
        }
    }
}

// Walks of the cluster-pair list for the analyses: every unordered pair of
// atoms within r_cut once, with the force kernel's traversal (chunks, staged
// atoms, column queues), so the distances are the force evaluation's.  The
// per-pair work is an operation type:
//   RdfOp   pair-distance histogram for the radial distribution functions of
//           Sec. II.C, Eq. 18: every pair within r_max <= r_cut by species
//           pair (a <= b) and bin k = floor(r / dr), counted in a block
//           histogram in shared memory (when it fits, else straight to global
//           memory) and added to the global one as 64-bit integers;
//   FragOp  fragments for the ion yields of Sec. III: every pair closer than
//           r_frag <= r_cut joins the atoms' sets in a lock-free union-find
//           whose parent indices only decrease, so each root is its set's
//           smallest atom index.
template <bool FP64>
struct WalkWarp {
    typename Prec<FP64>::S4 ix[kFiRow];                  // x, y, z, species of the SC atoms (-1: none)
    typename Prec<FP64>::S4 jx[kChunk * kClusterSize];   // the chunk's j-atoms, shifted
    int ia[kFiRow];                                      // their atom indices (-1: none)
    int ja[kChunk * kClusterSize];
};

template <bool FP64>
struct RdfOp {
    using T = typename Prec<FP64>::T;
    using S4 = typename Prec<FP64>::S4;
    int n_bins, nsp, smem_hist;
    T rmax2, inv_dr;
    unsigned long long* hist;
    unsigned* s_h;
    __device__ size_t smem_bytes() const
    {
        return smem_hist ? ((size_t)nsp * nsp * n_bins * sizeof(unsigned) + 15) / 16 * 16 : 0;
    }
    __device__ void init(unsigned char* smem)
    {
        s_h = reinterpret_cast<unsigned*>(smem);
        if (smem_hist)
            for (int k = threadIdx.x; k < nsp * nsp * n_bins; k += blockDim.x) s_h[k] = 0u;
    }
    __device__ void pair(const S4& a, int, const S4& b, int, bool ok)
    {
        const T dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const T r2 = Prec<FP64>::fma(dz, dz, Prec<FP64>::fma(dy, dy, dx * dx));
        if (ok && r2 < rmax2 && a.w >= T(0) && b.w >= T(0)) {
            const int k = min((int)(sqrt(r2) * inv_dr), n_bins - 1);
            const int sa = (int)a.w, sb = (int)b.w;
            const int idx = (min(sa, sb) * nsp + max(sa, sb)) * n_bins + k;
            if (smem_hist) atomicAdd(&s_h[idx], 1u);
            else atomicAdd(&hist[idx], 1ull);
        }
    }
    __device__ void finish()
    {
        if (smem_hist) {
            __syncthreads();
            for (int k = threadIdx.x; k < nsp * nsp * n_bins; k += blockDim.x)
                if (s_h[k]) atomicAdd(&hist[k], (unsigned long long)s_h[k]);
        }
    }
};

// Root of x's set.  Parents only ever point to smaller indices, so the walk
// ends within x steps; each step halves the path (the grandparent written is
// an ancestor whichever thread wrote last).
__device__ __forceinline__ int uf_find(int* parent, int x)
{
    while (true) {
        const int px = __ldcg(parent + x);
        if (px == x) return x;
        const int gp = __ldcg(parent + px);
        if (gp != px) parent[x] = gp;
        x = px;
    }
}

// Joins the sets of a and b: the larger root is hooked under the smaller one
// by a compare-and-swap that succeeds only on a root.  A failed swap means
// another thread hooked that root meanwhile; each retry follows a merge, so
// there are fewer retries than atoms (bounded anyway, with an error flag).
__device__ __forceinline__ void uf_unite(int* parent, int a, int b, int n, unsigned* err)
{
    for (int it = 0; it <= n; ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a > b) { const int t = a; a = b; b = t; }
        if (atomicCAS(parent + b, b, a) == b) return;
    }
    atomicOr(err, ERR_OVERFLOW);
}

template <bool FP64>
struct FragOp {
    using T = typename Prec<FP64>::T;
    using S4 = typename Prec<FP64>::S4;
    T rf2;
    int* parent;
    int n;
    unsigned* err;
    __device__ size_t smem_bytes() const { return 0; }
    __device__ void init(unsigned char*) {}
    __device__ void pair(const S4& a, int ia, const S4& b, int ib, bool ok)
    {
        const T dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const T r2 = Prec<FP64>::fma(dz, dz, Prec<FP64>::fma(dy, dy, dx * dx));
        if (ok && r2 < rf2 && ia >= 0 && ib >= 0) uf_unite(parent, ia, ib, n, err);
    }
    __device__ void finish() {}
};

template <bool FP64, class Op>
__global__ void __launch_bounds__(256) k_walk(Params p, Op op)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    using T4 = typename P::T4;
    using S4 = typename P::S4;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t hb = op.smem_bytes();
    op.init(smem);
    unsigned* s_kq = reinterpret_cast<unsigned*>(smem + hb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkWarp<FP64>& w = reinterpret_cast<WalkWarp<FP64>*>(smem + hb + 256 * sizeof(unsigned))[warp];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) {
        unsigned q = 0x88888888u;
        int n = 0;
        for (int k = 0; k < 8; ++k)
            if ((c >> k) & 1) {
                q = (q & ~(0xfu << (4 * n))) | ((unsigned)k << (4 * n));
                ++n;
            }
        s_kq[c] = q;
    }
    if (lane < kClusterSize) {
        w.ix[kSCAtoms + lane] = P::mk(T(-1.0e6), T(-1.0e6), T(-1.0e6), T(-1));
        w.ia[kSCAtoms + lane] = -1;
    }
    __syncthreads();
    const int tx = lane & 7, ty = lane >> 3;
    const int n_chunks = min(p.counters[7], p.chunk_cap);
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.counters[2], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_chunks) break;
        const int4 ch = p.pl_chunk[item];
        const int sc = ch.x, n_ent = ch.z, rr = ch.w;
        const PairEntry ent = lane < n_ent ? p.pl[ch.y + lane] : make_uint4(0u, 0u, 0u, 0u);
        const int fc = p.sc_first[sc], ncl = p.sc_ncl[sc];
        const Grid& g = p.grid_b[rr];
        __syncwarp();
        for (int a = lane; a < kSCAtoms; a += 32) {
            if ((a >> 3) < ncl) {
                const int slot = fc * kClusterSize + a;
                const T4 v = P::pos(p, slot);
                const int at = p.atom_of[slot];
                w.ix[a] = P::mk(v.x, v.y, v.z, at >= 0 ? T(p.species[at]) : T(-1));
                w.ia[a] = at;
            }
        }
        for (int a0 = 0; a0 < kChunk * kClusterSize; a0 += 32) {
            const int a = a0 + lane, e = a >> 3;
            const unsigned jc = __shfl_sync(kFull, ent.x, e);
            const unsigned cd = __shfl_sync(kFull, ent.y, e);
            if (e < n_ent) {
                int dx, dy, dz;
                half_shell((int)(cd & 0xffu), dx, dy, dz);
                const int slot = (int)jc * kClusterSize + (a & 7);
                const T4 v = P::pos(p, slot);
                const int at = p.atom_of[slot];
                const T sp = at >= 0 ? T(p.species[at]) : T(-1);
                if (FP64) w.jx[a] = P::mk(v.x + T(dx * g.edge[0]), v.y + T(dy * g.edge[1]), v.z + T(dz * g.edge[2]), sp);
                else w.jx[a] = P::mk(v.x + T((float)dx * g.edge_f[0]), v.y + T((float)dy * g.edge_f[1]),
                                     v.z + T((float)dz * g.edge_f[2]), sp);
                w.ja[a] = at;
            }
        }
        __syncwarp();
        for (int v = 0; v < n_ent; ++v) {
            const int jcl = (int)__shfl_sync(kFull, ent.x, v);
            const unsigned code = __shfl_sync(kFull, ent.y, v);
            const unsigned mlo = __shfl_sync(kFull, ent.z, v), mhi = __shfl_sync(kFull, ent.w, v);
            if ((mlo | mhi) == 0u) continue;
            const int kdiag = (code & 0xffu) == 0u ? jcl - fc : -1;
            const int j0 = v * kClusterSize + ty;
            const S4 a0 = w.jx[j0], a1 = w.jx[j0 + 4];
            const int b0 = w.ja[j0], b1 = w.ja[j0 + 4];
            const unsigned col0 = ((tx < 4 ? mlo : mhi) >> ((tx & 3) * 8)) & 0xffu;
            const int n_t = (int)__reduce_max_sync(kFull, (unsigned)__popc(col0));
            unsigned kq = s_kq[col0];
            for (int t = 0; t < n_t; ++t) {
                const int k = (int)(kq & 0xfu);
                kq >>= 4;
                const int si = k * kClusterSize + tx;
                const S4 xi = w.ix[si];
                const int ii = w.ia[si];
                const bool dg = k == kdiag;
                op.pair(xi, ii, a0, b0, !dg || tx < ty);
                op.pair(xi, ii, a1, b1, !dg || tx < ty + 4);
            }
        }
    }
    op.finish();
}

template <bool FP64, class Op>
static void launch_walk(const Params& p, cudaStream_t s, int blocks, Op op, size_t op_smem)
{
    const size_t smem = op_smem + 256 * sizeof(unsigned) + 8 * sizeof(WalkWarp<FP64>);
    cudaFuncSetAttribute(k_walk<FP64, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k_walk<FP64, Op><<<blocks, 256, smem, s>>>(p, op);
}

template <bool FP64>
static void rdf_typed(const Params& p, cudaStream_t s, int blocks, int n_bins, double r_max, unsigned long long* hist)
{
    RdfOp<FP64> op{};
    op.n_bins = n_bins;
    op.nsp = p.n_species;
    op.rmax2 = (typename Prec<FP64>::T)(r_max * r_max);
    op.inv_dr = (typename Prec<FP64>::T)((double)n_bins / r_max);
    op.hist = hist;
    const size_t nh = (size_t)p.n_species * p.n_species * n_bins;
    const size_t base = 256 * sizeof(unsigned) + 8 * sizeof(WalkWarp<FP64>);
    const size_t hb = (nh * sizeof(unsigned) + 15) / 16 * 16;
    op.smem_hist = base + hb <= 160 * 1024 ? 1 : 0;
    launch_walk<FP64>(p, s, blocks, op, op.smem_hist ? hb : 0);
}

void launch_rdf(const Params& p, cudaStream_t s, int blocks, int n_bins, double r_max, unsigned long long* hist)
{
    if (p.precision != 0) rdf_typed<true>(p, s, blocks, n_bins, r_max, hist);
    else rdf_typed<false>(p, s, blocks, n_bins, r_max, hist);
}

void launch_frag_link(const Params& p, cudaStream_t s, int blocks, double r_frag, int* parent)
{
    if (p.precision != 0) {
        FragOp<true> op{r_frag * r_frag, parent, p.n_atoms, p.err};
        launch_walk<true>(p, s, blocks, op, 0);
    } else {
        FragOp<false> op{(float)(r_frag * r_frag), parent, p.n_atoms, p.err};
        launch_walk<false>(p, s, blocks, op, 0);
    }
}

template <bool FP64, bool HYB>
static size_t pair_smem(int n_ts, int warps)
{
    const size_t tab = ((size_t)n_ts * n_ts * sizeof(typename Prec<FP64>::C2) + 127) / 128 * 128;
    return tab + 256 * sizeof(unsigned) + (size_t)warps * sizeof(WarpSmem<FP64, HYB>);
}

template <bool FP64, bool ENERGY, bool HYB>
static void set_smem_attr()
{
    static bool done = false;   // one per instantiation
    if (!done) {
        cudaFuncSetAttribute(k_pair<FP64, ENERGY, HYB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_pair<FP64, ENERGY, HYB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        done = true;
    }
}

template <bool FP64, bool ENERGY, bool HYB>
static void launch_one(const Params& p, cudaStream_t s, int blocks, int warps)
{
    set_smem_attr<FP64, ENERGY, HYB>();
    k_pair<FP64, ENERGY, HYB><<<blocks, warps * 32, pair_smem<FP64, HYB>(p.n_ts_lj, warps), s>>>(p);
}

template <bool FP64, bool ENERGY, bool HYB>
static int max_blocks(int warps, int n_ts)
{
    set_smem_attr<FP64, ENERGY, HYB>();
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<FP64, ENERGY, HYB>, warps * 32,
                                                  pair_smem<FP64, HYB>(n_ts, warps));
    return n;
}

int launch_pair_list(const Params& p, cudaStream_t s, int blocks)
{
    int n = 2;
    k_list_count<<<blocks, kListWarps * 32, 0, s>>>(p);
    if (p.sc_cap >= kScanScsMulti) {
        const int ctas = std::min(kScanCtasMax, (p.sc_cap + 2047) / 2048);
        k_list_scan_sums<<<ctas, 1024, 0, s>>>(p);
        k_list_scan_top<<<1, 1024, 0, s>>>(p, ctas);
        k_list_scan_apply<<<ctas, 1024, 0, s>>>(p);
        n += 3;
    } else {
        k_list_scan<<<1, 1024, 0, s>>>(p);
        n += 1;
    }
    k_list_write<<<blocks, kListWarps * 32, 0, s>>>(p);
    return n;
}

void launch_pair_forces(const Params& p, cudaStream_t s, bool energy, int blocks, int warps)
{
    const bool hyb = p.screening != 0;
    if (p.precision == 0) {
        if (hyb) {
            if (energy) launch_one<false, true, true>(p, s, blocks, warps);
            else launch_one<false, false, true>(p, s, blocks, warps);
        } else {
            if (energy) launch_one<false, true, false>(p, s, blocks, warps);
            else launch_one<false, false, false>(p, s, blocks, warps);
        }
    } else {
        if (hyb) {
            if (energy) launch_one<true, true, true>(p, s, blocks, warps);
            else launch_one<true, false, true>(p, s, blocks, warps);
        } else {
            if (energy) launch_one<true, true, false>(p, s, blocks, warps);
            else launch_one<true, false, false>(p, s, blocks, warps);
        }
    }
}

int pair_max_blocks_per_sm(bool fp64, bool energy, bool hyb, int warps, int n_ts)
{
    int n;
    if (!fp64) {
        if (hyb) n = energy ? max_blocks<false, true, true>(warps, n_ts) : max_blocks<false, false, true>(warps, n_ts);
        else n = energy ? max_blocks<false, true, false>(warps, n_ts) : max_blocks<false, false, false>(warps, n_ts);
    } else {
        if (hyb) n = energy ? max_blocks<true, true, true>(warps, n_ts) : max_blocks<true, false, true>(warps, n_ts);
        else n = energy ? max_blocks<true, true, false>(warps, n_ts) : max_blocks<true, false, false>(warps, n_ts);
    }
    return n > 0 ? n : 1;
}

}  // namespace mdg
