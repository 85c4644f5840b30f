// Short-range non-bonded forces: Debye-screened Coulomb (Sec. II.A, Eq. 2)
// plus screened LJ (Sec. II.B, Eq. 8) with charge-scaled LJ sizes (Eq. 11),
// LJ excluded inside a native fragment (Sec. II.B), cut off at r_cut with the
// energy shifted to zero there.
//
// Work decomposition (Newton's third law, every unordered pair once):
//   * atoms are cell-sorted into clusters of 8; up to 8 consecutive clusters
//     of one cell form a super-cluster (SC);
//   * a work item is (SC, a range of the 14 half-shell cells, each cut in four
//     parts of its j-cluster range); a warp owns one item at a time (dynamic
//     scheduling through an atomic counter);
//   * the SC's atoms and per-lane i-force partials live in shared memory;
//     lane (tx = lane & 7, ty = lane >> 3) takes atom tx of an i-cluster and
//     atoms ty, ty+4 of the current j-cluster;
//   * j-clusters are pre-filtered per i-cluster by bounding-box distance, and
//     only the i-clusters whose boxes are in range are visited (a loop over
//     the set bits of a mask, so the code stays small);
//   * forces are summed in FP32 (or FP64) within one (SC, cell, part) for the
//     i side and one (SC, j-cluster) visit for the j side, then converted
//     once to 64-bit fixed point (2^-32 kJ/mol/nm): the per-atom totals are
//     exact integer sums, identical for every launch shape and schedule.
#include "md_internal.cuh"

namespace mdg {

template <bool FP64>
struct Prec;

template <>
struct Prec<false> {
    using T = float;
    using T4 = float4;         // global packed position + charge
    using S4 = float4;         // shared-memory copy
    using C2 = float2;         // c6, c12
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
    using C2 = double2;        // c6, c12
    static __device__ __forceinline__ T4 pos(const Params& p, int slot) { return p.xq64[slot]; }
    static __device__ __forceinline__ T rsq(T x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ T expneg(T x) { return exp(-x); }
    static __device__ __forceinline__ long long fix(T v) { return __double2ll_rn(v * 4294967296.0); }
    static __device__ __forceinline__ bool fix_ok(T v) { return fabs(v) < 1.073741824e9; }
    static __device__ __forceinline__ const C2* table(const Params& p) { return p.lj_d; }
    static __device__ __forceinline__ S4 mk(T a, T b, T c, T d) { S4 s; s.x = a; s.y = b; s.z = c; s.w = d; return s; }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __fma_rn(a, b, c); }
};

// per-warp shared-memory layout
template <bool FP64>
struct WarpSmem {
    typename Prec<FP64>::S4 ix[kSuperClusters * kClusterSize];   // x, y, z, f*q of the SC atoms
    int2 it[kSuperClusters * kClusterSize];                      // LJ row byte offset, fragment
    typename Prec<FP64>::S4 fi[kSuperClusters * 32];             // per (i-cluster, lane) force (+energy)
    float4 lo[kSuperClusters], hi[kSuperClusters];               // i-cluster boxes (cell frame)
    int2 fr[kSuperClusters];                                     // i-cluster fragment ranges
};

template <bool FP64>
__device__ __forceinline__ void red_fix(long long* dst, typename Prec<FP64>::T v, unsigned* err)
{
    if (!Prec<FP64>::fix_ok(v)) {
        atomicOr(err, ERR_OVERFLOW);
        return;
    }
    const long long q = Prec<FP64>::fix(v);
    if (q != 0) atomicAdd((unsigned long long*)dst, (unsigned long long)q);
}

// One pair, d = x_i - x_j.  `ok` drops the duplicates of the self-cluster
// diagonal; equal fragments drop the LJ part.  qjk = q_j * kappa.  The force
// on i is accumulated into (fx, fy, fz), the force on j into (fjx, fjy, fjz);
// with ENERGY the cutoff-shifted pair energy into u.  Multiply-adds are
// written out so that each accumulation is one fused operation.
template <bool FP64, bool ENERGY>
__device__ __forceinline__ void pair(const typename Prec<FP64>::S4& xi, int row_off, int fri,
                                     typename Prec<FP64>::T xj, typename Prec<FP64>::T yj,
                                     typename Prec<FP64>::T zj, typename Prec<FP64>::T qj,
                                     typename Prec<FP64>::T qjk, int tsj_off, int frj, bool ok,
                                     const unsigned char* __restrict__ lj_bytes,
                                     typename Prec<FP64>::T kap, typename Prec<FP64>::T rc2,
                                     typename Prec<FP64>::T& fx, typename Prec<FP64>::T& fy,
                                     typename Prec<FP64>::T& fz, typename Prec<FP64>::T& fjx,
                                     typename Prec<FP64>::T& fjy, typename Prec<FP64>::T& fjz,
                                     typename Prec<FP64>::T& u, int& npair, typename Prec<FP64>::T erc,
                                     typename Prec<FP64>::T irc)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    const T dx = xi.x - xj, dy = xi.y - yj, dz = xi.z - zj;
    const T r2 = P::fma(dz, dz, P::fma(dy, dy, dx * dx));
    const bool in = (r2 < rc2) && ok;
    const T rinv = in ? P::rsq(r2) : T(0);
    const typename P::C2 c = *reinterpret_cast<const typename P::C2*>(lj_bytes + row_off + tsj_off);
    const T rinv2 = rinv * rinv;
    const T rinv6 = rinv2 * rinv2 * rinv2;
    const T lj6 = fri == frj ? T(0) : rinv6;    // bonded in the native structure: no LJ
    const T r = r2 * rinv;
    const T kr = kap * r;
    const T e = P::expneg(kr);
    const T A = c.y * rinv6;                    // c12 / r^12
    const T B = A - c.x;                        // c12/r^12 - c6/r^6
    const T D6 = T(6) * (A + B);                // 12 c12/r^12 - 6 c6/r^6
    const T E1 = P::fma(kr, B, D6);
    const T Cc = xi.w * P::fma(qj, rinv, qjk);  // f q_i q_j (1/r + kappa)
    const T S = P::fma(lj6, E1, Cc);
    const T fs = S * (rinv2 * e);               // F(r)/r
    const T nfs = -fs;
    fx = P::fma(fs, dx, fx); fy = P::fma(fs, dy, fy); fz = P::fma(fs, dz, fz);
    fjx = P::fma(nfs, dx, fjx); fjy = P::fma(nfs, dy, fjy); fjz = P::fma(nfs, dz, fjz);
    if (ENERGY) {
        if (in) {
            const T qq = xi.w * qj;
            const T irc6 = irc * irc * irc * irc * irc * irc;
            const T lj_on = fri == frj ? T(0) : T(1);
            const T ush = erc * (qq * irc + lj_on * (c.y * irc6 - c.x) * irc6);
            u += e * (qq * rinv + lj6 * B) - ush;
            npair += 1;
        }
    }
}

template <bool FP64, bool ENERGY>
__global__ void __launch_bounds__(256, FP64 ? 2 : 3) k_pair(Params p, int nsplit)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    using T4 = typename P::T4;
    using S4 = typename P::S4;
    using C2 = typename P::C2;
    using WS = WarpSmem<FP64>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nts = p.n_ts;
    C2* s_lj = reinterpret_cast<C2*>(smem);
    const unsigned char* lj_bytes = smem;
    const size_t tab = ((size_t)nts * nts * sizeof(C2) + 127) / 128 * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WS& w = reinterpret_cast<WS*>(smem + tab)[warp];

    for (int k = threadIdx.x; k < nts * nts; k += blockDim.x) s_lj[k] = P::table(p)[k];
    __syncthreads();
    if (*p.err & ERR_CELL) return;

    const int tx = lane & 7, ty = lane >> 3;
    const bool gt0 = ty > tx, gt1 = ty + 4 > tx;   // j index above i index (diagonal blocks)
    const int n_items = p.counters[0] * nsplit;
    const float rcb = p.rc_f + kBBoxMargin;
    const float rcb2 = rcb * rcb;
    const T rc2 = FP64 ? T(p.rc2) : T(p.rc2_f);
    const T irc = T(1.0 / p.r_cut);
    const T coulf = T(p.coulomb_f);

    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.counters[2], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        // sub-items of a super-cluster: (half-shell cell, part of its j range),
        // kSubItems of them, grouped nsplit ways into work items
        const int sc = item / nsplit, part = item - sc * nsplit;
        const int sub0 = part * kSubItems / nsplit, sub1 = (part + 1) * kSubItems / nsplit;
        const int c = p.sc_cell[sc], fc = p.sc_first[sc], ncl = p.sc_ncl[sc];
        int rr;
        {
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
        const T kap = FP64 ? T(p.rs[rr].kappa_force) : T(p.rs[rr].kappa_f);
        const T erc = ENERGY ? P::expneg(kap * T(p.r_cut)) : T(0);

        // the super-cluster's atoms and boxes into shared memory
        __syncwarp();
        for (int a = lane; a < kSuperClusters * kClusterSize; a += 32) {
            if ((a >> 3) < ncl) {
                const int slot = fc * kClusterSize + a;
                const T4 v = P::pos(p, slot);
                const int2 t = p.tf[slot];
                w.ix[a] = P::mk(v.x, v.y, v.z, coulf * v.w);
                w.it[a] = make_int2(t.x * nts * (int)sizeof(C2), t.y);   // byte offset of the LJ row
            }
        }
        if (lane < ncl) {
            w.lo[lane] = p.bb_lo[fc + lane];
            w.hi[lane] = p.bb_hi[fc + lane];
            w.fr[lane] = p.bb_frag[fc + lane];
        }
        __syncwarp();

        for (int sub = sub0; sub < sub1; ++sub) {
            const int nb = sub / kJParts, part_j = sub - nb * kJParts;
            int dx, dy, dz;
            half_shell(nb, dx, dy, dz);
            int ncx = cx + dx, ncy = cy + dy, ncz = cz + dz;
            if (g.periodic) {
                ncx = ncx < 0 ? ncx + g.dims[0] : (ncx >= g.dims[0] ? ncx - g.dims[0] : ncx);
                ncy = ncy < 0 ? ncy + g.dims[1] : (ncy >= g.dims[1] ? ncy - g.dims[1] : ncy);
                ncz = ncz < 0 ? ncz + g.dims[2] : (ncz >= g.dims[2] ? ncz - g.dims[2] : ncz);
            } else if (ncx < 0 || ncy < 0 || ncz < 0 || ncx >= g.dims[0] || ncy >= g.dims[1] ||
                       ncz >= g.dims[2]) {
                continue;
            }
            const int c2 = g.cell_off + ncx + g.dims[0] * (ncy + g.dims[1] * ncz);
            const bool self = nb == 0;
            const int jr0 = self ? fc : p.cell_pstart[c2] / kClusterSize;
            const int jr1 = p.cell_pstart[c2 + 1] / kClusterSize;
            const int jn = jr1 - jr0;
            const int j_beg = jr0 + (jn * part_j) / kJParts, j_end = jr0 + (jn * (part_j + 1)) / kJParts;
            if (j_beg >= j_end) continue;
            const float Dfx = (float)dx * g.edge_f[0], Dfy = (float)dy * g.edge_f[1],
                        Dfz = (float)dz * g.edge_f[2];
            const T Dx = FP64 ? T(dx * g.edge[0]) : T(Dfx);
            const T Dy = FP64 ? T(dy * g.edge[1]) : T(Dfy);
            const T Dz = FP64 ? T(dz * g.edge[2]) : T(Dfz);

            for (int k = 0; k < ncl; ++k) w.fi[k * 32 + lane] = P::mk(T(0), T(0), T(0), T(0));
            int npair = 0;
            bool any = false;

            for (int base = j_beg; base < j_end; base += 32) {
                const int jc = base + lane;
                unsigned m = 0;
                if (jc < j_end) {
                    const float4 lo = p.bb_lo[jc], hi = p.bb_hi[jc];
                    const float jlx = lo.x + Dfx, jly = lo.y + Dfy, jlz = lo.z + Dfz;
                    const float jhx = hi.x + Dfx, jhy = hi.y + Dfy, jhz = hi.z + Dfz;
                    const int kmax = self ? min(ncl, jc - fc + 1) : ncl;
#pragma unroll 2
                    for (int k = 0; k < kmax; ++k) {
                        const float4 il = w.lo[k], ih = w.hi[k];
                        const float gx = fmaxf(0.0f, fmaxf(il.x - jhx, jlx - ih.x));
                        const float gy = fmaxf(0.0f, fmaxf(il.y - jhy, jly - ih.y));
                        const float gz = fmaxf(0.0f, fmaxf(il.z - jhz, jlz - ih.z));
                        if (gx * gx + gy * gy + gz * gz < rcb2) m |= 1u << k;
                    }
                }
                unsigned todo = __ballot_sync(0xffffffffu, m != 0);
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    unsigned mk = __shfl_sync(0xffffffffu, m, src);
                    const int jcl = base + src;
                    any = true;
                    const int s0 = jcl * kClusterSize + ty, s1 = s0 + 4;
                    const T4 a0 = P::pos(p, s0), a1 = P::pos(p, s1);
                    const int2 t0 = p.tf[s0], t1 = p.tf[s1];
                    const T x0 = a0.x + Dx, y0 = a0.y + Dy, z0 = a0.z + Dz;
                    const T x1 = a1.x + Dx, y1 = a1.y + Dy, z1 = a1.z + Dz;
                    const T q0k = a0.w * kap, q1k = a1.w * kap;
                    const int j0off = t0.x * (int)sizeof(C2), j1off = t1.x * (int)sizeof(C2);
                    const int kdiag = self ? jcl - fc : -1;   // i-cluster equal to this j-cluster
                    T fj0x = 0, fj0y = 0, fj0z = 0, fj1x = 0, fj1y = 0, fj1z = 0;
                    while (mk) {
                        const int k = __ffs(mk) - 1;
                        mk &= mk - 1;
                        const S4 xi = w.ix[k * kClusterSize + tx];
                        const int2 ti = w.it[k * kClusterSize + tx];
                        const bool dg = k == kdiag;
                        S4 acc = w.fi[k * 32 + lane];
                        pair<FP64, ENERGY>(xi, ti.x, ti.y, x0, y0, z0, a0.w, q0k, j0off, t0.y, !dg || gt0, lj_bytes,
                                           kap, rc2, acc.x, acc.y, acc.z, fj0x, fj0y, fj0z, acc.w, npair, erc, irc);
                        pair<FP64, ENERGY>(xi, ti.x, ti.y, x1, y1, z1, a1.w, q1k, j1off, t1.y, !dg || gt1, lj_bytes,
                                           kap, rc2, acc.x, acc.y, acc.z, fj1x, fj1y, fj1z, acc.w, npair, erc, irc);
                        w.fi[k * 32 + lane] = acc;
                    }
                    // j forces: sum over the 8 i-lanes of each ty group.  Lanes tx < 4 keep
                    // atom ty (j0), lanes tx >= 4 atom ty + 4 (j1); then each lane holds one
                    // component of one atom and issues one RED.
                    {
                        const bool up = tx >= 4;
                        T ax = up ? fj1x : fj0x, ay = up ? fj1y : fj0y, az = up ? fj1z : fj0z;
                        ax += __shfl_xor_sync(0xffffffffu, up ? fj0x : fj1x, 4);
                        ay += __shfl_xor_sync(0xffffffffu, up ? fj0y : fj1y, 4);
                        az += __shfl_xor_sync(0xffffffffu, up ? fj0z : fj1z, 4);
#pragma unroll
                        for (int o = 1; o < 4; o <<= 1) {
                            ax += __shfl_xor_sync(0xffffffffu, ax, o);
                            ay += __shfl_xor_sync(0xffffffffu, ay, o);
                            az += __shfl_xor_sync(0xffffffffu, az, o);
                        }
                        const int comp = tx & 3;
                        if (comp < 3) {
                            const T v = comp == 0 ? ax : (comp == 1 ? ay : az);
                            long long* dst = (comp == 0 ? p.fx : comp == 1 ? p.fy : p.fz) + (up ? s1 : s0);
                            red_fix<FP64>(dst, v, p.err);
                        }
                    }
                }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            __syncwarp();
            // i forces of this (SC, cell): sum the 4 ty partials of each atom
            for (int a = lane; a < ncl * kClusterSize; a += 32) {
                const int k = a >> 3, t = a & 7;
                S4 sum = w.fi[k * 32 + t];
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    const S4 v = w.fi[k * 32 + q * 8 + t];
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
                for (int o = 16; o; o >>= 1) npair += __shfl_xor_sync(0xffffffffu, npair, o);
                if (lane == 0 && npair) atomicAdd((unsigned long long*)p.pair_count, (unsigned long long)npair);
            }
        }
    }
}

template <bool FP64>
static size_t pair_smem(int n_ts, int warps)
{
    const size_t tab = ((size_t)n_ts * n_ts * sizeof(typename Prec<FP64>::C2) + 127) / 128 * 128;
    return tab + (size_t)warps * sizeof(WarpSmem<FP64>);
}

template <bool FP64, bool ENERGY>
static void set_smem_attr()
{
    static bool done = false;   // one per instantiation
    if (!done) {
        cudaFuncSetAttribute(k_pair<FP64, ENERGY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        done = true;
    }
}

template <bool FP64, bool ENERGY>
static void launch_one(const Params& p, cudaStream_t s, int blocks, int warps, int nsplit)
{
    set_smem_attr<FP64, ENERGY>();
    k_pair<FP64, ENERGY><<<blocks, warps * 32, pair_smem<FP64>(p.n_ts, warps), s>>>(p, nsplit);
}

void launch_pair(const Params& p, cudaStream_t s, bool energy, int blocks, int warps, int nsplit)
{
    if (p.precision == 0) {
        if (energy) launch_one<false, true>(p, s, blocks, warps, nsplit);
        else launch_one<false, false>(p, s, blocks, warps, nsplit);
    } else {
        if (energy) launch_one<true, true>(p, s, blocks, warps, nsplit);
        else launch_one<true, false>(p, s, blocks, warps, nsplit);
    }
}

int pair_max_blocks_per_sm(bool fp64, bool energy, int warps, int n_ts)
{
    int n = 0;
    if (!fp64) {
        set_smem_attr<false, false>();
        set_smem_attr<false, true>();
        const size_t smem = pair_smem<false>(n_ts, warps);
        if (energy) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<false, true>, warps * 32, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<false, false>, warps * 32, smem);
    } else {
        set_smem_attr<true, false>();
        set_smem_attr<true, true>();
        const size_t smem = pair_smem<true>(n_ts, warps);
        if (energy) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<true, true>, warps * 32, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<true, false>, warps * 32, smem);
    }
    return n > 0 ? n : 1;
}

}  // namespace mdg
