// Short-range non-bonded forces: Debye-screened Coulomb (Sec. II.A, Eq. 2)
// plus screened LJ (Sec. II.B, Eq. 8) with charge-scaled LJ sizes (Eq. 11),
// LJ excluded inside a native fragment (Sec. II.B), cut off at r_cut with the
// energy shifted to zero there.
//
// Work decomposition (Newton's third law, every unordered pair once):
//   * atoms are cell-sorted into clusters of 8; up to 8 consecutive clusters
//     of one cell form a super-cluster (SC);
//   * a work item is (SC, range of the 14 half-shell cells); a warp owns one
//     item at a time (dynamic scheduling through an atomic counter);
//   * lane (tx = lane & 7, ty = lane >> 3) holds atom tx of each i-cluster in
//     registers and atoms ty, ty+4 of the current j-cluster;
//   * j-clusters are pre-filtered per i-cluster by bounding-box distance;
//   * forces are summed in FP32 (or FP64) inside one (SC, cell, j-cluster)
//     block and converted once to 64-bit fixed point (2^-32 kJ/mol/nm), so the
//     final per-atom sums are exact integer additions -- identical for every
//     launch shape and scheduling order.
#include <cfloat>

#include "md_internal.cuh"

namespace mdg {

template <bool FP64>
struct Prec;

template <>
struct Prec<false> {
    using T = float;
    using T4 = float4;
    using C2 = float2;
    static __device__ __forceinline__ T4 pos(const Params& p, int slot) { return p.xq[slot]; }
    static __device__ __forceinline__ C2 lj(const C2* tab, int idx) { return tab[idx]; }
    static __device__ __forceinline__ T rsq(T x) { return rsqrtf(x); }
    static __device__ __forceinline__ T expneg(T x) { return exp2f(x * -1.4426950408889634f); }
    static __device__ __forceinline__ long long fix(T v) { return __float2ll_rn(v * 4294967296.0f); }
    static __device__ __forceinline__ bool fix_ok(T v) { return fabsf(v) < 1.0737418e9f; }
    static __device__ __forceinline__ const C2* table(const Params& p) { return p.lj_f; }
};

template <>
struct Prec<true> {
    using T = double;
    using T4 = double4_32a;
    using C2 = double2;
    static __device__ __forceinline__ T4 pos(const Params& p, int slot) { return p.xq64[slot]; }
    static __device__ __forceinline__ C2 lj(const C2* tab, int idx) { return tab[idx]; }
    static __device__ __forceinline__ T rsq(T x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ T expneg(T x) { return exp(-x); }
    static __device__ __forceinline__ long long fix(T v) { return __double2ll_rn(v * 4294967296.0); }
    static __device__ __forceinline__ bool fix_ok(T v) { return fabs(v) < 1.073741824e9; }
    static __device__ __forceinline__ const C2* table(const Params& p) { return p.lj_d; }
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

// One pair.  d = x_i - x_j.  Accumulates the force on i (fi) and on j (fj)
// and, with ENERGY, the cutoff-shifted pair energy into u.
template <bool FP64, bool ENERGY, bool SLOW>
__device__ __forceinline__ void pair(typename Prec<FP64>::T xi, typename Prec<FP64>::T yi,
                                     typename Prec<FP64>::T zi, typename Prec<FP64>::T qfi, int rowi,
                                     int fri, typename Prec<FP64>::T xj, typename Prec<FP64>::T yj,
                                     typename Prec<FP64>::T zj, typename Prec<FP64>::T qj, int tsj,
                                     int frj, bool self_ok, const typename Prec<FP64>::C2* lj,
                                     typename Prec<FP64>::T kap, typename Prec<FP64>::T rc2,
                                     typename Prec<FP64>::T& fix_, typename Prec<FP64>::T& fiy,
                                     typename Prec<FP64>::T& fiz, typename Prec<FP64>::T& fjx,
                                     typename Prec<FP64>::T& fjy, typename Prec<FP64>::T& fjz,
                                     typename Prec<FP64>::T& u, int& npair,
                                     typename Prec<FP64>::T erc, typename Prec<FP64>::T irc)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    const T dx = xi - xj, dy = yi - yj, dz = zi - zj;
    const T r2 = dx * dx + dy * dy + dz * dz;
    bool in = r2 < rc2;
    if (SLOW) in = in && self_ok;
    const T rinv = in ? P::rsq(r2) : T(0);
    typename P::C2 c = P::lj(lj, rowi + tsj);
    if (SLOW && fri == frj) { c.x = T(0); c.y = T(0); }
    const T rinv2 = rinv * rinv;
    const T rinv6 = rinv2 * rinv2 * rinv2;
    const T r = r2 * rinv;
    const T kr = kap * r;
    const T e = P::expneg(kr);
    const T A = c.y * rinv6;            // c12 / r^12
    const T B = A - c.x;                // c12/r^12 - c6/r^6
    const T D6 = T(6) * (A + B);        // 12 c12/r^12 - 6 c6/r^6
    const T E1 = kr * B + D6;
    const T qq = qfi * qj;              // f q_i q_j
    const T Cc = qq * (rinv + kap);
    const T S = rinv6 * E1 + Cc;
    const T fs = S * rinv2 * e;         // F(r)/r
    fix_ += fs * dx; fiy += fs * dy; fiz += fs * dz;
    fjx -= fs * dx; fjy -= fs * dy; fjz -= fs * dz;
    if (ENERGY) {
        if (in) {
            const T irc6 = irc * irc * irc * irc * irc * irc;
            const T ush = erc * (qq * irc + (c.y * irc6 - c.x) * irc6);
            u += e * (qq * rinv + rinv6 * B) - ush;
            npair += 1;
        }
    }
}

template <bool FP64, bool ENERGY, int KC>
__global__ void __launch_bounds__(256) k_pair(Params p, int nsplit)
{
    using P = Prec<FP64>;
    using T = typename P::T;
    using T4 = typename P::T4;
    using C2 = typename P::C2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nts = p.n_ts;
    C2* s_lj = reinterpret_cast<C2*>(smem);
    float4* s_bb = reinterpret_cast<float4*>(smem + ((nts * nts * sizeof(C2) + 15) / 16) * 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* w_lo = s_bb + warp * (3 * kSuperClusters);
    float4* w_hi = w_lo + kSuperClusters;
    int2* w_fr = reinterpret_cast<int2*>(w_hi + kSuperClusters);

    for (int k = threadIdx.x; k < nts * nts; k += blockDim.x) s_lj[k] = P::table(p)[k];
    __syncthreads();
    if (*p.err & ERR_CELL) return;

    const int tx = lane & 7, ty = lane >> 3;
    const int n_items = p.counters[0] * nsplit;
    const float rcb = p.rc_f + kBBoxMargin;
    const float rcb2 = rcb * rcb;
    const T rc2 = FP64 ? T(p.rc2) : T(p.rc2_f);
    const T irc = T(1.0 / p.r_cut);

    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.counters[2], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int sc = item / nsplit, part = item - sc * nsplit;
        const int nb0 = part * kHalfShell / nsplit, nb1 = (part + 1) * kHalfShell / nsplit;
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

        // i-cluster bounding boxes into shared memory
        __syncwarp();
        if (lane < ncl) {
            w_lo[lane] = p.bb_lo[fc + lane];
            w_hi[lane] = p.bb_hi[fc + lane];
            w_fr[lane] = p.bb_frag[fc + lane];
        }
        __syncwarp();

        for (int pass = 0; pass * KC < ncl; ++pass) {
            const int kbase = pass * KC;
            // i atoms in registers
            T xi[KC], yi[KC], zi[KC], qfi[KC];
            int rowi[KC], fri[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                const int slot = (fc + kbase + k) * kClusterSize + tx;
                if (kbase + k < ncl) {
                    const T4 a = P::pos(p, slot);
                    const int2 t = p.tf[slot];
                    xi[k] = a.x; yi[k] = a.y; zi[k] = a.z;
                    qfi[k] = T(p.coulomb_f) * a.w;
                    rowi[k] = t.x * nts;
                    fri[k] = t.y;
                } else {
                    xi[k] = yi[k] = zi[k] = T(1.0e30); qfi[k] = T(0); rowi[k] = 0; fri[k] = -1;
                }
            }
            for (int nb = nb0; nb < nb1; ++nb) {
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
                const int j_end = p.cell_pstart[c2 + 1] / kClusterSize;
                int j_beg = p.cell_pstart[c2] / kClusterSize;
                const bool self = nb == 0;
                if (self) j_beg = fc;
                const float Dfx = (float)dx * g.edge_f[0], Dfy = (float)dy * g.edge_f[1],
                            Dfz = (float)dz * g.edge_f[2];
                const T Dx = FP64 ? T(dx * g.edge[0]) : T(Dfx);
                const T Dy = FP64 ? T(dy * g.edge[1]) : T(Dfy);
                const T Dz = FP64 ? T(dz * g.edge[2]) : T(Dfz);

                T fi[KC][3];
                T ui[KC];
#pragma unroll
                for (int k = 0; k < KC; ++k) { fi[k][0] = fi[k][1] = fi[k][2] = T(0); ui[k] = T(0); }
                int npair = 0;
                bool any = false;

                for (int base = j_beg; base < j_end; base += 32) {
                    const int jc = base + lane;
                    unsigned m = 0, xm = 0;
                    if (jc < j_end) {
                        const float4 lo = p.bb_lo[jc], hi = p.bb_hi[jc];
                        const int2 fr = p.bb_frag[jc];
                        const float jlx = lo.x + Dfx, jly = lo.y + Dfy, jlz = lo.z + Dfz;
                        const float jhx = hi.x + Dfx, jhy = hi.y + Dfy, jhz = hi.z + Dfz;
#pragma unroll
                        for (int k = 0; k < KC; ++k) {
                            const int kk = kbase + k;
                            if (kk < ncl && (!self || jc >= fc + kk)) {
                                const float4 il = w_lo[kk], ih = w_hi[kk];
                                const float gx = fmaxf(0.0f, fmaxf(il.x - jhx, jlx - ih.x));
                                const float gy = fmaxf(0.0f, fmaxf(il.y - jhy, jly - ih.y));
                                const float gz = fmaxf(0.0f, fmaxf(il.z - jhz, jlz - ih.z));
                                if (gx * gx + gy * gy + gz * gz < rcb2) {
                                    m |= 1u << k;
                                    const int2 ifr = w_fr[kk];
                                    if ((self && jc == fc + kk) || (fr.x <= ifr.y && ifr.x <= fr.y))
                                        xm |= 1u << k;
                                }
                            }
                        }
                    }
                    unsigned todo = __ballot_sync(0xffffffffu, m != 0);
                    while (todo) {
                        const int src = __ffs(todo) - 1;
                        todo &= todo - 1;
                        const unsigned jm = __shfl_sync(0xffffffffu, m, src);
                        const unsigned jx = __shfl_sync(0xffffffffu, xm, src);
                        const int jcl = base + src;
                        any = true;
                        const int s0 = jcl * kClusterSize + ty, s1 = s0 + 4;
                        const T4 a0 = P::pos(p, s0), a1 = P::pos(p, s1);
                        const int2 t0 = p.tf[s0], t1 = p.tf[s1];
                        const T x0 = a0.x + Dx, y0 = a0.y + Dy, z0 = a0.z + Dz;
                        const T x1 = a1.x + Dx, y1 = a1.y + Dy, z1 = a1.z + Dz;
                        T fj0x = 0, fj0y = 0, fj0z = 0, fj1x = 0, fj1y = 0, fj1z = 0;
#pragma unroll
                        for (int k = 0; k < KC; ++k) {
                            if (jm & (1u << k)) {
                                if (jx & (1u << k)) {
                                    const bool diag = self && jcl == fc + kbase + k;
                                    pair<FP64, ENERGY, true>(xi[k], yi[k], zi[k], qfi[k], rowi[k], fri[k], x0, y0, z0,
                                                             a0.w, t0.x, t0.y, !diag || ty > tx, s_lj, kap, rc2,
                                                             fi[k][0], fi[k][1], fi[k][2], fj0x, fj0y, fj0z, ui[k],
                                                             npair, erc, irc);
                                    pair<FP64, ENERGY, true>(xi[k], yi[k], zi[k], qfi[k], rowi[k], fri[k], x1, y1, z1,
                                                             a1.w, t1.x, t1.y, !diag || ty + 4 > tx, s_lj, kap, rc2,
                                                             fi[k][0], fi[k][1], fi[k][2], fj1x, fj1y, fj1z, ui[k],
                                                             npair, erc, irc);
                                } else {
                                    pair<FP64, ENERGY, false>(xi[k], yi[k], zi[k], qfi[k], rowi[k], 0, x0, y0, z0,
                                                              a0.w, t0.x, 0, true, s_lj, kap, rc2, fi[k][0], fi[k][1],
                                                              fi[k][2], fj0x, fj0y, fj0z, ui[k], npair, erc, irc);
                                    pair<FP64, ENERGY, false>(xi[k], yi[k], zi[k], qfi[k], rowi[k], 0, x1, y1, z1,
                                                              a1.w, t1.x, 0, true, s_lj, kap, rc2, fi[k][0], fi[k][1],
                                                              fi[k][2], fj1x, fj1y, fj1z, ui[k], npair, erc, irc);
                                }
                            }
                        }
                        // j forces: sum over the 8 i-lanes of each ty group
#pragma unroll
                        for (int o = 1; o < 8; o <<= 1) {
                            fj0x += __shfl_xor_sync(0xffffffffu, fj0x, o);
                            fj0y += __shfl_xor_sync(0xffffffffu, fj0y, o);
                            fj0z += __shfl_xor_sync(0xffffffffu, fj0z, o);
                            fj1x += __shfl_xor_sync(0xffffffffu, fj1x, o);
                            fj1y += __shfl_xor_sync(0xffffffffu, fj1y, o);
                            fj1z += __shfl_xor_sync(0xffffffffu, fj1z, o);
                        }
                        if (tx < 6) {
                            const T v = tx == 0 ? fj0x : tx == 1 ? fj0y : tx == 2 ? fj0z
                                      : tx == 3 ? fj1x : tx == 4 ? fj1y : fj1z;
                            const int slot = tx < 3 ? s0 : s1;
                            long long* dst = (tx % 3 == 0 ? p.fx : tx % 3 == 1 ? p.fy : p.fz) + slot;
                            red_fix<FP64>(dst, v, p.err);
                        }
                    }
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                // i forces of this (SC, cell): sum over the 4 ty lanes, one RED per atom component
#pragma unroll
                for (int k = 0; k < KC; ++k) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        fi[k][d] += __shfl_xor_sync(0xffffffffu, fi[k][d], 8);
                        fi[k][d] += __shfl_xor_sync(0xffffffffu, fi[k][d], 16);
                    }
                    if (ENERGY) {
                        ui[k] += __shfl_xor_sync(0xffffffffu, ui[k], 8);
                        ui[k] += __shfl_xor_sync(0xffffffffu, ui[k], 16);
                    }
                }
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    if (kbase + k < ncl && (k % 4) == ty) {
                        const int slot = (fc + kbase + k) * kClusterSize + tx;
                        red_fix<FP64>(p.fx + slot, fi[k][0], p.err);
                        red_fix<FP64>(p.fy + slot, fi[k][1], p.err);
                        red_fix<FP64>(p.fz + slot, fi[k][2], p.err);
                        if (ENERGY) red_fix<FP64>(p.epot + slot, ui[k], p.err);
                    }
                }
                if (ENERGY) {
#pragma unroll
                    for (int o = 16; o; o >>= 1) npair += __shfl_xor_sync(0xffffffffu, npair, o);
                    if (lane == 0 && npair) atomicAdd((unsigned long long*)p.pair_count, (unsigned long long)npair);
                }
            }
        }
    }
}

template <bool FP64, bool ENERGY, int KC>
static void launch_one(const Params& p, cudaStream_t s, int blocks, int warps, int nsplit)
{
    const size_t tab = ((size_t)p.n_ts * p.n_ts * sizeof(typename Prec<FP64>::C2) + 15) / 16 * 16;
    const size_t smem = tab + (size_t)warps * 3 * kSuperClusters * sizeof(float4);
    k_pair<FP64, ENERGY, KC><<<blocks, warps * 32, smem, s>>>(p, nsplit);
}

void launch_pair(const Params& p, cudaStream_t s, bool energy, int blocks, int warps, int nsplit)
{
    if (p.precision == 0) {
        if (energy) launch_one<false, true, 8>(p, s, blocks, warps, nsplit);
        else launch_one<false, false, 8>(p, s, blocks, warps, nsplit);
    } else {
        if (energy) launch_one<true, true, 4>(p, s, blocks, warps, nsplit);
        else launch_one<true, false, 4>(p, s, blocks, warps, nsplit);
    }
}

int pair_max_blocks_per_sm(bool fp64, bool energy, int warps, int n_ts)
{
    int n = 0;
    const size_t tab = ((size_t)n_ts * n_ts * (fp64 ? sizeof(double2) : sizeof(float2)) + 15) / 16 * 16;
    const size_t smem = tab + (size_t)warps * 3 * kSuperClusters * sizeof(float4);
    if (!fp64) {
        if (energy) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<false, true, 8>, warps * 32, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<false, false, 8>, warps * 32, smem);
    } else {
        if (energy) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<true, true, 4>, warps * 32, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair<true, false, 4>, warps * 32, smem);
    }
    return n > 0 ? n : 1;
}

}  // namespace mdg
