// Per-atom part of one timestep: velocity kick + drift (Sec. II.B, Eq. 12,
// velocity Verlet), the stochastic collisional-radiative charge update
// (Sec. II.A), and the free-electron-gas reduction that sets the Debye length
// (Sec. II.A, Eq. 3) together with the next cell grid.
//
// The charge update must reproduce the CPU oracle bit for bit, so its
// floating-point work uses only IEEE double basic operations written with
// explicit round-to-nearest intrinsics (no fused multiply-add), and this file
// is compiled with -fmad=false as a second guard.
#include "md_internal.cuh"

namespace mdg {

constexpr int kAccCopies = 16;   // accumulator copies per replica (spread contention)
// atoms per block of the step kernel: one warp of each role.  Blocks this
// small wait at their barriers for two warps only, so the SM keeps issuing
// from the other blocks (water box: 1.8 us less per step than 128 atoms per
// block; 2 M-atom droplet: 87 us less)
constexpr int kStepAtoms = 32;
constexpr int kStepThreads = 2 * kStepAtoms;   // two threads per atom: kick/drift and charge update

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers M0, M1 on
// words 0 and 2, Weyl key schedule W0, W1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The 53-bit uniform ((a >> 5) 2^26 + (b >> 6)) 2^-53.  Its value is the
// integer m times a power of two, exactly, so the double is assembled from m
// in the integer pipe (GB300 issues FP64 at 2 lanes per SM per clock): the
// exponent from the leading one of m, the 52 bits below it as the mantissa.
__device__ __forceinline__ double u53(unsigned a, unsigned b)
{
    const unsigned long long m = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
    if (m == 0ull) return 0.0;
    const int lz = __clzll((long long)m);                           // 11 .. 63
    const unsigned long long mant = ((m << lz) << 1) >> 12;         // the bits below the leading one
    const unsigned long long ex = (unsigned long long)(1033 - lz);  // 1023 + (63 - lz) - 53
    return __longlong_as_double((long long)((ex << 52) | mant));
}

// 1 - e^{-x}: x = k/16 + r, (1 - E_k) + E_k (1 - e^{-r}), degree-12 Taylor
// polynomial of 1 - e^{-r} in nested form; E_k and 1/m come from host tables.
__device__ __forceinline__ double one_minus_exp_neg(double x, const double* etab,
                                                    const double* inv)
{
    if (!(x > 0.0)) return 0.0;
    double xs = __dmul_rn(x, 16.0);
    if (xs >= (double)kNEtab) return 1.0;
    int k = (int)xs;
    double r = __dsub_rn(x, __dmul_rn((double)k, 0.0625));
    double t = 1.0;
#pragma unroll
    for (int m = 12; m >= 2; --m) t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(r, inv[m]), t));
    double g = __dmul_rn(r, t);
    if (k == 0) return g;
    double ek = etab[k];
    return __dadd_rn(__dsub_rn(1.0, ek), __dmul_rn(ek, g));
}

__device__ __forceinline__ double interp(const double* K, int i0, double w)
{
    return __dadd_rn(K[i0], __dmul_rn(w, __dsub_rn(K[i0 + 1], K[i0])));
}

// ---------------------------------------------------------------------------
// Per-replica scalars for the step `step` (Eq. 3 and the CR helpers) and
// the cell grid for the positions just reduced into the bounding box.
// Executed by one thread per replica.
// ---------------------------------------------------------------------------
__device__ void plasma_scalars(const Params& p, int r, long long step, RepState& st)
{
    double te, ne;
    if (p.plasma_mode == 1) {
        long long idx = (long long)r * (p.max_steps + 1) + (step <= p.max_steps ? step : p.max_steps);
        ne = p.pres_ne[idx];
        te = p.pres_te[idx];
    } else if (st.n_e > 0) {
        te = __ddiv_rn((double)st.e_gas, __dmul_rn(1500.0, (double)st.n_e));
        ne = __ddiv_rn((double)st.n_e, p.volume[r]);
    } else {
        te = 0.0;
        ne = 0.0;
    }
    double kap = 0.0;
    if (ne > 0.0) {
        double tc = te > p.te_floor ? te : p.te_floor;
        double k2 = __ddiv_rn(__dmul_rn(p.four_pi_f, ne), __dmul_rn(tc, kEvKJmol));
        kap = __dsqrt_rn(k2);
    }
    st.te_ev = te;
    st.n_dens = ne;
    st.kappa = kap;
    st.ne_dt = __dmul_rn(ne, p.dt);
    double x = __dmul_rn(te, p.inv_dte);
    if (x > (double)(p.n_te - 1)) x = (double)(p.n_te - 1);
    if (x < 0.0) x = 0.0;
    int i0 = (int)x;
    if (i0 > p.n_te - 2) i0 = p.n_te - 2;
    st.it0 = i0;
    st.wt = __dsub_rn(x, (double)i0);
    double kf = p.kappa_fixed >= 0.0 ? p.kappa_fixed : kap;
    st.kappa_force = kf;
    st.kappa_f = (float)kf;
}

// Adaptive skin: whether this step rebuilds (x) and whether the list it builds
// carries the skin (y), from the step's largest displacement and the current
// list.  A pure function, so that the warps sizing the grids and the thread
// that records the decision agree.
__device__ __forceinline__ int2 adapt_decision(const Params& p, unsigned maxd2)
{
    const ListCtl& c = *p.lc;
    if (c.buffered) {
        const int rebuild = maxd2 > __float_as_uint(c.half_skin2) ? 1 : 0;
        return make_int2(rebuild, rebuild && c.since_build + 1 < kAdaptOffLife ? 0 : 1);
    }
    // one step since the last build: maxd2 is the largest one-step
    // displacement d, and a buffered list would last (skin/2) / d steps
    return make_int2(1, __uint_as_float(maxd2) * (float)(kAdaptOnLife * kAdaptOnLife) <= p.half_skin2 ? 1 : 0);
}

// Radius of the list this step builds: the cells' smallest edge.
template <bool SETCOND>
__device__ __forceinline__ double next_rlist(const Params& p, unsigned maxd2)
{
    if (SETCOND && p.lc) return adapt_decision(p, maxd2).y ? p.r_list : p.r_cut;
    return list_rlist(p);
}

__device__ void make_grid(const Params& p, int r, const unsigned long long* mn,
                          const unsigned long long* mx, double rl)
{
    Grid& g = p.grid[r];
    if (g.periodic) return;   // periodic grids are fixed at init
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = mn[d] == ~0ull ? 0.0 : from_ordered(mn[d]);
        hi[d] = mx[d] == 0ull ? 0.0 : from_ordered(mx[d]);
        if (!(hi[d] >= lo[d])) { lo[d] = 0.0; hi[d] = 0.0; }
    }
    double f = 1.0;   // cell edges >= rl, the radius of the list built on the grid
    int n[3];
    for (int it = 0; it < 400; ++it) {
        long long prod = 1;
        for (int d = 0; d < 3; ++d) {
            double m = floor((hi[d] - lo[d]) / (rl * f));
            n[d] = m < 1.0 ? 1 : (m > 1.0e6 ? 1000000 : (int)m);
            prod *= n[d];
        }
        if (prod <= g.cell_cap) break;
        f *= 1.125;
    }
    for (int d = 0; d < 3; ++d) {
        double ext = hi[d] - lo[d];
        double e = n[d] == 1 ? (ext > rl ? ext : rl) : ext / n[d];
        g.origin[d] = lo[d];
        g.edge[d] = e;
        g.inv_edge[d] = 1.0 / e;
        g.edge_f[d] = (float)e;
        g.dims[d] = n[d];
    }
}

// Velocity increment of a half kick, (dt/2m) F.  The mixed path forms it in
// FP32 (it is ~1e-4 of v, so its rounding is far below the FP32 force error);
// the FP64 path in FP64.  Every kernel that applies or reports a half kick
// uses this function, so stepping and state read-out round identically.
__device__ __forceinline__ void half_kick(const Params& p, int s, int slot, double& ax, double& ay,
                                          double& az)
{
    const double c = p.hdtm[s];
    if (p.precision == 0) {
        const float cf = p.hdtm_f[s];   // (float)(c 2^-32), formed on the host
        ax = (double)(cf * (float)p.fx[slot]);
        ay = (double)(cf * (float)p.fy[slot]);
        az = (double)(cf * (float)p.fz[slot]);
    } else {
        ax = c * ((double)p.fx[slot] * kFixInv);
        ay = c * ((double)p.fy[slot] * kFixInv);
        az = c * ((double)p.fz[slot] * kFixInv);
    }
}

// ---------------------------------------------------------------------------
// k_step_a: one thread per atom (original order).
// ---------------------------------------------------------------------------
constexpr int kInlineReps = 4;   // up to this many replicas the step kernel's last block reduces them

// Three standard normal numbers for the Langevin force (Sec. II.B, Eq. 14)
// from four Philox words: Box-Muller on u = (w + 1/2) 2^-32 for the pairs
// (w0, w1) and (w2, w3), of which the first three results are used.  The
// mixed path works in FP32 (u rounded to 24 bits, relative error 6e-8 down to
// the smallest u, which rounds up to 1 at most), the FP64 path in FP64.
__device__ __forceinline__ void gauss3(uint4 w, bool fp32, double& g0, double& g1, double& g2)
{
    if (fp32) {
        const float ua = __fmul_rn(__fadd_rn((float)w.x, 0.5f), 2.3283064e-10f);
        const float ub = __fmul_rn(__fadd_rn((float)w.y, 0.5f), 2.3283064e-10f);
        const float uc = __fmul_rn(__fadd_rn((float)w.z, 0.5f), 2.3283064e-10f);
        const float ud = __fmul_rn(__fadd_rn((float)w.w, 0.5f), 2.3283064e-10f);
        const float ra = sqrtf(-2.0f * logf(ua)), rb = sqrtf(-2.0f * logf(uc));
        float sb, cb;
        sincospif(2.0f * ub, &sb, &cb);
        g0 = (double)(ra * cb);
        g1 = (double)(ra * sb);
        g2 = (double)(rb * cospif(2.0f * ud));
    } else {
        const double s = 2.3283064365386963e-10;   // 2^-32
        const double ua = ((double)w.x + 0.5) * s, ub = ((double)w.y + 0.5) * s;
        const double uc = ((double)w.z + 0.5) * s, ud = ((double)w.w + 0.5) * s;
        const double ra = sqrt(-2.0 * log(ua)), rb = sqrt(-2.0 * log(uc));
        double sb, cb;
        sincospi(2.0 * ub, &sb, &cb);
        g0 = ra * cb;
        g1 = ra * sb;
        g2 = rb * cospi(2.0 * ud);
    }
}

// Hybrid ion-sphere / Debye electrostatics of every charge state at the
// plasma state just computed (Sec. II.A, Eqs. 4-7), by the warp that reduced
// replica rr.  An ion of charge Q has R = (3Q / (4 pi n_e))^{1/3} (Eq. 4) and
// the transition radius r' of Eq. 7, evaluated as s^3 / (kappa (t^2 + t + 1))
// with s = kappa R and t = (1 + s^3)^{1/3} (no cancellation).  Its potential
// is Q/r + c1 - c2 r^2 inside r' and G e^{-kappa r}/r outside; the continuity
// of the potential and its first two derivatives at r' gives, with
// x = kappa r' and D = 3 + 3x + x^2, G = 3 Q e^x / D,
// c1 = -Q kappa (3 + 3x/2) / D and c2 = -2 pi n_e / 3 for every Q.
// Without an ion sphere (Q = 0, n_e = 0 or kappa = 0): r' = 0, G = Q.
__device__ void hyb_table(const Params& p, int rr, int lane, double kap, double ne)
{
    HybQ* rows = p.hq + (size_t)rr * kHybQ;
    const double c2 = -2.0 * kPi * ne / 3.0;
    const double rc = p.r_cut;
    double rpm = 0.0;
    for (int q = lane; q <= p.z_max; q += 32) {   // the charge states the species can reach
        const double Q = (double)q;
        double G = Q, rp = 0.0, c1 = 0.0;
        if (q > 0 && ne > 0.0 && kap > 0.0) {
            const double R = cbrt(3.0 * Q / (4.0 * kPi * ne));
            const double s = R * kap, s3 = s * s * s;
            const double t = cbrt(1.0 + s3);
            rp = s3 / (kap * (t * t + t + 1.0));
            const double x = kap * rp;
            const double D = 3.0 + 3.0 * x + x * x;
            c1 = -Q * kap * (3.0 + 1.5 * x) / D;
            G = 3.0 * Q * exp(x) / D;
        }
        const double phirc = rc < rp ? Q / rc + c1 - c2 * rc * rc : G * exp(-kap * rc) / rc;
        HybQ h;
        h.G = G; h.rp = rp; h.c1 = c1; h.phirc = phirc;
        h.Gf = (float)fmin(G, 1.0e30); h.rpf = (float)rp; h.c1f = (float)c1; h.phircf = (float)phirc;
        rows[q] = h;
        rpm = fmax(rpm, rp);
    }
    for (int o = 16; o; o >>= 1) rpm = fmax(rpm, __shfl_xor_sync(0xffffffffu, rpm, o));
    if (lane == 0) {
        HybRep r;
        r.c2 = c2; r.rpm2 = rpm * rpm; r.c2f = (float)c2; r.rpm2f = (float)(rpm * rpm);
        p.hrep[rr] = r;
    }
}

// Replica rr's per-step reduction by one warp: lane c reads accumulator copy
// c and clears it, the warp reduces, lane 0 updates the plasma scalars (Eq. 3)
// and the next grid.
__device__ void finalize_replica(const Params& p, int rr, int lane, long long next, double rl)
{
    RepAccum* a = p.acc + (size_t)rr * kAccCopies;
    RepState st;
    if (lane == 0) st = p.rs[rr];   // issued before the accumulators are read and cleared
    long long v[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    if (lane < kAccCopies) {
        v[0] = __ldcg(&a[lane].dNe);
        v[1] = __ldcg(&a[lane].dE);
        for (int k = 0; k < 4; ++k) v[2 + k] = __ldcg(&a[lane].counts[k]);
        for (int d = 0; d < 3; ++d) {
            mn[d] = __ldcg(&a[lane].bmin[d]);
            mx[d] = __ldcg(&a[lane].bmax[d]);
        }
        a[lane].dNe = 0;
        a[lane].dE = 0;
        for (int k = 0; k < 4; ++k) a[lane].counts[k] = 0;
        for (int d = 0; d < 3; ++d) {
            a[lane].bmin[d] = ~0ull;
            a[lane].bmax[d] = 0ull;
        }
    }
    for (int o = kAccCopies / 2; o; o >>= 1) {   // lanes 0..kAccCopies-1 hold the copies
        for (int k = 0; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        for (int d = 0; d < 3; ++d) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, mn[d], o);
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx[d], o);
            mn[d] = x < mn[d] ? x : mn[d];
            mx[d] = y > mx[d] ? y : mx[d];
        }
    }
    if (lane == 0) {
        st.n_e += v[0];
        st.e_gas += v[1];
        if (st.e_gas < 0) st.e_gas = 0;
        for (int k = 0; k < 4; ++k) st.counts[k] += v[2 + k];
        plasma_scalars(p, rr, next, st);
        p.rs[rr] = st;
        make_grid(p, rr, mn, mx, rl);
    }
    if (p.screening) {
        const double kap = __shfl_sync(0xffffffffu, st.kappa_force, 0);
        const double ne = __shfl_sync(0xffffffffu, st.n_dens, 0);
        hyb_table(p, rr, lane, kap, ne);
    }
    if (p.langevin) {
        // Langevin update of the next step per species (Eqs. 13-14): gamma =
        // n_e g_s, c = e^{-gamma dt}, sigma = sqrt((1 - c^2) k_B T_e / m_s)
        const double ne = __shfl_sync(0xffffffffu, st.n_dens, 0);
        const double te = __shfl_sync(0xffffffffu, st.te_ev, 0);
        if (lane < p.n_species) {
            const double gam = ne * p.lgv_g[lane];
            const double c = exp(-gam * p.dt);
            const double kT = te * kEvKJmol;
            p.lgv[(size_t)rr * kMaxSpecies + lane] = make_double2(c, sqrt((1.0 - c * c) * kT / p.mass[lane]));
        }
    }
}

// Once per step, after every replica: counters, step number and, with the
// Verlet buffer, the rebuild decision and the graph condition.
template <bool SETCOND>
__device__ void finalize_step(const Params& p, int mode, long long next, unsigned maxd2)
{
    p.counters[3] = 0;
    if (mode & STEP_ADVANCE) *p.step = next;
    if (mode & STEP_KICK_DRIFT) *p.kick_full = 1;
    if constexpr (SETCOND) {
        p.counters[2] = 0;   // work counter of the force kernel (also reset by a build)
        // rebuild once some atom may have closed half of the skin: pairs
        // within r_cut now were within r_cut + skin at the build
        *p.maxd2 = 0u;
        int rebuild;
        if (p.lc) {
            // adaptive skin: the buffer stays only while lists live long enough to pay
            ListCtl& c = *p.lc;
            const int2 d = adapt_decision(p, maxd2);
            rebuild = d.x;
            if (d.y != c.buffered) {
                c.buffered = d.y;
                c.rlist_f = d.y ? p.rlist_f : p.rc_f;
                c.r_list = d.y ? p.r_list : p.r_cut;
                c.half_skin2 = d.y ? p.half_skin2 : 0.0f;
            }
            if (rebuild && !d.y) c.unbuffered_builds += 1;
            c.since_build = rebuild ? 0 : c.since_build + 1;
        } else {
            rebuild = maxd2 > __float_as_uint(p.half_skin2) ? 1 : 0;
        }
        p.builds[0] += rebuild;
        p.builds[1] = rebuild;
        cudaGraphSetConditional(p.cond, (unsigned)rebuild);
    }
}

// SETCOND: the Verlet-buffered variant that decides the rebuild and sets the
// graph condition (ncu does not profile kernels that can set one, so the
// every-step variant is a separate instantiation).  MINB: resident blocks per
// SM the registers are sized for; 16 (64 registers) for grids of many blocks
// per SM, where the FP64 pipe binds and more resident warps pay (2 M-atom
// droplet: 3.80 -> 3.71 ms per step); 10 (96 registers) for small grids, which
// are latency-bound (water box: 108.4 against 110.9 us per step with 16)
template <bool SETCOND, int MINB>
__global__ void __launch_bounds__(kStepThreads, MINB) k_step_a(Params p, int mode)
{
    __shared__ long long s_acc[kRepWindow][6];
    __shared__ unsigned long long s_bmin[kRepWindow][3], s_bmax[kRepWindow][3];
    __shared__ int s_last;
    __shared__ unsigned s_maxd2;
    __shared__ double s_rl;
    __shared__ uint8_t s_q[kStepAtoms];   // charges after this step's update (charge-update warps)
    // a cluster-pair list overflow freezes the state at the step whose forces
    // are missing; the host grows the list, recomputes them and resumes
    if (*p.err & ERR_LIST) return;
    const int tid = threadIdx.x;
    for (int k = tid; k < kRepWindow * 6; k += blockDim.x) (&s_acc[0][0])[k] = 0;
    for (int k = tid; k < kRepWindow * 3; k += blockDim.x) {
        (&s_bmin[0][0])[k] = ~0ull;
        (&s_bmax[0][0])[k] = 0ull;
    }
    if (tid == 0) s_maxd2 = 0u;
    __syncthreads();

    const long long step = *p.step;
    const int kick_full = *p.kick_full;
    // the first kStepAtoms threads kick, drift and re-pack atoms first ..
    // first + kStepAtoms - 1; the others run the charge update of the same
    // atoms (independent until the re-pack)
    const bool cr_role = tid >= kStepAtoms;
    const int first = blockIdx.x * kStepAtoms;
    const int r0 = p.rep[first < p.n_atoms ? first : p.n_atoms - 1];
    const int i = first + (tid & (kStepAtoms - 1));
    const bool live = i < p.n_atoms;
    const int lane = tid & 31;
    int r = live ? p.rep[i] : -1;
    double pos[3] = {0.0, 0.0, 0.0};
    bool vac = false;
    // inputs of this atom's re-pack (Verlet-buffered list), loaded before the
    // charge update is waited for
    const bool repack = live && !cr_role && p.xr && (mode & STEP_KICK_DRIFT);
    int pk_slot = 0, pk_sp = 0, pk_fr = 0, pk_q = 0, pk_per = 0;
    double pk_cen[3] = {0.0, 0.0, 0.0}, pk_box[3] = {0.0, 0.0, 0.0};

    if (live && !cr_role) {
        const int s = p.species[i];
        double x = p.x[i], y = p.y[i], z = p.z[i];
        if (repack) {
            pk_slot = p.slot_of[i];
            const double4_32a c = p.cl_cen[pk_slot / kClusterSize];
            pk_cen[0] = c.x; pk_cen[1] = c.y; pk_cen[2] = c.z;
            const Grid& gb = p.grid_b[r];
            pk_per = gb.periodic;
            pk_box[0] = gb.box[0]; pk_box[1] = gb.box[1]; pk_box[2] = gb.box[2];
            pk_sp = s;
            pk_fr = p.frag[i];
            pk_q = p.q[i];
        }
        if (mode & STEP_KICK_DRIFT) {
            // the state holds v_{n-1/2} once stepping has started: finish the
            // previous step's half kick, then this step's (two separate adds,
            // exactly as velocity Verlet rounds them)
            double ax, ay, az;
            half_kick(p, s, p.slot_of[i], ax, ay, az);
            double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
            if (kick_full) { vx = vx + ax; vy = vy + ay; vz = vz + az; }
            vx = vx + ax; vy = vy + ay; vz = vz + az;
            if (p.langevin) {
                // electron-ion coupling (Eqs. 13-14): exact Ornstein-Uhlenbeck
                // update with Philox stream 1 of (seed, atom, step)
                const double2 cs = p.lgv[(size_t)r * kMaxSpecies + s];
                const unsigned long long sd = p.seed[r];
                const uint4 w4 = philox4x32_10(make_uint4((unsigned)p.local_id[i], (unsigned)step, 1u, 0u),
                                               make_uint2((unsigned)sd, (unsigned)(sd >> 32)));
                double gx, gy, gz;
                gauss3(w4, p.precision == 0, gx, gy, gz);
                vx = cs.x * vx + cs.y * gx;
                vy = cs.x * vy + cs.y * gy;
                vz = cs.x * vz + cs.y * gz;
            }
            // x + dt v with one rounding (GB300 issues FP64 at 2 lanes per SM per clock)
            x = __fma_rn(p.dt, vx, x);
            y = __fma_rn(p.dt, vy, y);
            z = __fma_rn(p.dt, vz, z);
            const Grid& g = p.grid[r];
            if (g.periodic) {
                // wrap only atoms that left the box (FP64 division is slow); the
                // tests run on the bit patterns
                const double L0 = g.box[0], L1 = g.box[1], L2 = g.box[2];
                if (below_zero(x) || at_or_above(x, L0)) { x -= L0 * floor(x / L0); if (x >= L0) x -= L0; }
                if (below_zero(y) || at_or_above(y, L1)) { y -= L1 * floor(y / L1); if (y >= L1) y -= L1; }
                if (below_zero(z) || at_or_above(z, L2)) { z -= L2 * floor(z / L2); if (z >= L2) z -= L2; }
            }
            // finite check on the exponent bits (integer ops; FP64 compares are slow here)
            if (((__double2hiint(x) & 0x7ff00000) == 0x7ff00000) || ((__double2hiint(y) & 0x7ff00000) == 0x7ff00000) ||
                ((__double2hiint(z) & 0x7ff00000) == 0x7ff00000) || ((__double2hiint(vx) & 0x7ff00000) == 0x7ff00000) ||
                ((__double2hiint(vy) & 0x7ff00000) == 0x7ff00000) || ((__double2hiint(vz) & 0x7ff00000) == 0x7ff00000))
                atomicOr(p.err, ERR_NONFINITE);
            p.vx[i] = vx; p.vy[i] = vy; p.vz[i] = vz;
            p.x[i] = x; p.y[i] = y; p.z[i] = z;
            if (p.xr) {
                // displacement since the last list build (minimum image), squared
                // in FP32: it only decides the rebuild, against half the skin
                double d[3] = {x - p.xr[i], y - p.yr[i], z - p.zr[i]};
                if (g.periodic)
                    for (int k = 0; k < 3; ++k) {
                        const int o = beyond_half(d[k], g.box[k]);
                        if (o > 0) d[k] -= g.box[k];
                        else if (o < 0) d[k] += g.box[k];
                    }
                const float e0 = (float)d[0], e1 = (float)d[1], e2 = (float)d[2];
                const float d2 = e0 * e0 + e1 * e1 + e2 * e2;
                // non-negative floats order like their bit patterns (NaN sorts high)
                atomicMax(&s_maxd2, __float_as_uint(d2));
            }
        }
        pos[0] = x; pos[1] = y; pos[2] = z;
        vac = !p.grid[r].periodic;
    }

    // ---- bounding box of vacuum replicas (warp-reduced when uniform) ----
    {
        const unsigned full = 0xffffffffu;
        const int rl0 = __shfl_sync(full, r, 0);
        const bool uniform = __all_sync(full, r == rl0) && rl0 >= 0;
        const bool any_vac = __any_sync(full, vac);
        if (any_vac) {
            if (uniform) {
                if (__shfl_sync(full, (int)vac, 0)) {
                    for (int d = 0; d < 3; ++d) {
                        unsigned long long mn = ordered_bits(pos[d]), mx = mn;
                        for (int o = 16; o; o >>= 1) {
                            unsigned long long a = __shfl_xor_sync(full, mn, o);
                            unsigned long long b = __shfl_xor_sync(full, mx, o);
                            mn = a < mn ? a : mn;
                            mx = b > mx ? b : mx;
                        }
                        if (lane == 0) {
                            const int w = rl0 - r0;
                            if (w < kRepWindow) {
                                atomicMin(&s_bmin[w][d], mn);
                                atomicMax(&s_bmax[w][d], mx);
                            } else {
                                RepAccum* a = p.acc + (size_t)rl0 * kAccCopies + (blockIdx.x & (kAccCopies - 1));
                                atomicMin(&a->bmin[d], mn);
                                atomicMax(&a->bmax[d], mx);
                            }
                        }
                    }
                }
            } else if (vac) {
                const int w = r - r0;
                for (int d = 0; d < 3; ++d) {
                    unsigned long long o = ordered_bits(pos[d]);
                    if (w < kRepWindow) {
                        atomicMin(&s_bmin[w][d], o);
                        atomicMax(&s_bmax[w][d], o);
                    } else {
                        RepAccum* a = p.acc + (size_t)r * kAccCopies + (blockIdx.x & (kAccCopies - 1));
                        atomicMin(&a->bmin[d], o);
                        atomicMax(&a->bmax[d], o);
                    }
                }
            }
        }
    }

    // ---- collisional-radiative update (reading of Sec. II.A) ----
    if (live && cr_role && (mode & STEP_CR) && p.charge_mode == kChargeTable) {
        // charges from the CR charge-state fractions (reading of Sec. II.A): the
        // atom's fixed quantile u (Philox stream 2) against the running sums of
        // its species at the end of this step (table row step + 1)
        const int s = p.species[i];
        const int Z = p.zs[s];
        const int qi = p.q[i];
        int qn = qi;
        if (step < p.max_steps) {
            const double* cum = p.qcum + ((size_t)r * (p.max_steps + 1) + (size_t)(step + 1)) * p.n_ts + p.ts_off[s];
            const unsigned long long sd = p.seed[r];
            const uint4 w4 = philox4x32_10(make_uint4((unsigned)p.local_id[i], 0u, 2u, 0u),
                                           make_uint2((unsigned)sd, (unsigned)(sd >> 32)));
            const double u = u53(w4.x, w4.y);
            qn = Z;
            for (int k = 0; k <= Z; ++k)
                if (u < cum[k]) { qn = k; break; }
        } else {
            atomicOr(p.err, ERR_TABLE_END);
        }
        s_q[i - first] = (uint8_t)qn;
        if (qn != qi || p.h[i]) {
            p.q[i] = (uint8_t)qn;
            p.h[i] = 0;
        }
        const int dq = qn - qi;
        if (dq != 0) {
            const int w = r - r0;
            const unsigned long long up = (unsigned long long)(dq > 0 ? dq : -dq);
            if (w < kRepWindow) {
                atomicAdd((unsigned long long*)&s_acc[w][0], (unsigned long long)(long long)dq);
                atomicAdd((unsigned long long*)&s_acc[w][dq > 0 ? 2 : 5], up);
            } else {
                RepAccum* a = p.acc + (size_t)r * kAccCopies + (blockIdx.x & (kAccCopies - 1));
                atomicAdd((unsigned long long*)&a->dNe, (unsigned long long)(long long)dq);
                atomicAdd((unsigned long long*)&a->counts[dq > 0 ? 0 : 3], up);
            }
        }
    }
    if (live && cr_role && (mode & STEP_CR) && p.charge_mode != kChargeTable) {
        const int s = p.species[i];
        const int Z = p.zs[s];
        const int qi = p.q[i], hi = p.h[i];
        s_q[i - first] = (uint8_t)qi;   // replaced below if an event changes it
        const int ts = p.ts_off[s] + qi;
        const RepState st = p.rs[r];
        double dF = 0.0;
        if (step < p.max_steps) dF = p.dF[(long long)r * p.max_steps + step];
        else atomicOr(p.err, ERR_TABLE_END);
        const double a_pi = __dmul_rn(p.sigma_pi[2 * ts + hi], dF);
        const double a_a = hi ? p.auger_dt[s] : 0.0;
        double a_ci = 0.0, a_rec = 0.0;
        if (qi < Z) a_ci = __dmul_rn(st.ne_dt, interp(p.k_ci + (long long)ts * p.n_te, st.it0, st.wt));
        if (qi > 0 && hi == 0)
            a_rec = __dmul_rn(st.ne_dt, interp(p.k_rec + (long long)ts * p.n_te, st.it0, st.wt));
        const double c1 = __dadd_rn(a_pi, a_a);
        const double c2 = __dadd_rn(c1, a_ci);
        const double lam = __dadd_rn(c2, a_rec);
        int ch = -1;
        // lam and u0 are non-negative doubles, whose order is that of their
        // bit patterns: the tests run in the integer pipe
        if (__double_as_longlong(lam) > 0ll) {
            const unsigned long long sd = p.seed[r];
            const uint4 w4 = philox4x32_10(make_uint4((unsigned)p.local_id[i], (unsigned)step, 0u, 0u),
                                           make_uint2((unsigned)sd, (unsigned)(sd >> 32)));
            const double u0 = u53(w4.x, w4.y);
            // 1 - e^{-lam} <= lam, so u0 >= lam decides "no event" exactly
            if ((unsigned long long)__double_as_longlong(u0) < (unsigned long long)__double_as_longlong(lam) &&
                u0 < one_minus_exp_neg(lam, p.etab, p.inv12)) {
                const double t = __dmul_rn(u53(w4.z, w4.w), lam);
                if (t < a_pi) ch = 0;
                else if (t < c1) ch = 1;
                else if (t < c2) ch = 2;
                else if (t < lam) ch = 3;
                else ch = a_rec > 0.0 ? 3 : (a_ci > 0.0 ? 2 : (a_a > 0.0 ? 1 : 0));
            }
        }
        if (ch >= 0) {
            int qn = qi, hn = hi;
            long long de;
            if (ch == 0) {
                qn = qi + 1;
                de = p.e_pi_mev[2 * ts + hi];
                if (qn == Z) hn = 0;
                else if (Z >= 3 && hi == 0 && Z - qn >= 2) hn = 1;
            } else if (ch == 1) {
                qn = qi + 1;
                hn = 0;
                de = p.e_auger_mev[s];
            } else if (ch == 2) {
                qn = qi + 1;
                if (qn == Z) hn = 0;
                de = -p.ip_mev[ts];
            } else {
                qn = qi - 1;
                de = p.ip_mev[ts - 1];
            }
            p.q[i] = (uint8_t)qn;
            p.h[i] = (uint8_t)hn;
            s_q[i - first] = (uint8_t)qn;
            const int w = r - r0;
            if (w < kRepWindow) {
                atomicAdd((unsigned long long*)&s_acc[w][0], (unsigned long long)(ch == 3 ? -1ll : 1ll));
                atomicAdd((unsigned long long*)&s_acc[w][1], (unsigned long long)de);
                atomicAdd((unsigned long long*)&s_acc[w][2 + ch], 1ull);
            } else {
                RepAccum* a = p.acc + (size_t)r * kAccCopies + (blockIdx.x & (kAccCopies - 1));
                atomicAdd((unsigned long long*)&a->dNe, (unsigned long long)(ch == 3 ? -1ll : 1ll));
                atomicAdd((unsigned long long*)&a->dE, (unsigned long long)de);
                atomicAdd((unsigned long long*)&a->counts[ch], 1ull);
            }
        }
    }
    // ---- Verlet-buffered list: the packed record of this atom for the forces
    // of this step, in the slot of the last build (a build, if one follows,
    // rewrites all records); the force sums are cleared after the kick read them
    __syncthreads();   // the charges of this step are written
    if (repack) {
        const int qi = (mode & STEP_CR) ? (int)s_q[i - first] : pk_q;
        pack_record(p, pk_slot, pos, pk_cen, pk_per, pk_box, pk_sp, qi, pk_fr);
    }
    __syncthreads();

    // ---- flush block partials ----
    {
        const int last_atom = min(first + kStepAtoms, p.n_atoms) - 1;
        const int r_last = p.rep[last_atom];
        const int nw = min(r_last - r0 + 1, kRepWindow);
        for (int k = tid; k < nw * 12; k += blockDim.x) {
            const int w = k / 12, f = k % 12;
            RepAccum* a = p.acc + (size_t)(r0 + w) * kAccCopies + (blockIdx.x & (kAccCopies - 1));
            if (f < 6) {
                const long long v = s_acc[w][f];
                if (v != 0) {
                    unsigned long long* dst = f == 0 ? (unsigned long long*)&a->dNe
                                            : f == 1 ? (unsigned long long*)&a->dE
                                                     : (unsigned long long*)&a->counts[f - 2];
                    atomicAdd(dst, (unsigned long long)v);
                }
            } else if (f < 9) {
                if (s_bmin[w][f - 6] != ~0ull) atomicMin(&a->bmin[f - 6], s_bmin[w][f - 6]);
            } else {
                if (s_bmax[w][f - 9] != 0ull) atomicMax(&a->bmax[f - 9], s_bmax[w][f - 9]);
            }
        }
    }

    if (tid == 0 && s_maxd2) atomicMax(p.maxd2, s_maxd2);

    // ---- per-replica reduction (Eq. 3) and next grid: by this kernel's last
    // block for a few replicas, by k_step_fin (a warp per replica) for more ----
    if (p.n_rep > kInlineReps) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.counters[3], 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned m2 = 0u;
    if (tid == 0) {   // the list radius of this step's build, before finalize_step records it
        m2 = SETCOND ? __ldcg(p.maxd2) : 0u;
        s_rl = next_rlist<SETCOND>(p, m2);
    }
    __syncthreads();
    const double rl = s_rl;
    const long long next = (mode & STEP_ADVANCE) ? step + 1 : step;
    const int warp = tid >> 5, n_warps = blockDim.x >> 5;
    for (int rr = warp; rr < p.n_rep; rr += n_warps) finalize_replica(p, rr, lane, next, rl);
    if (tid == 0) finalize_step<SETCOND>(p, mode, next, m2);
}

// Per-replica reduction when there are many replicas: one warp each, then the
// last block finishes the step.
template <bool SETCOND>
__global__ void __launch_bounds__(256) k_step_fin(Params p, int mode)
{
    __shared__ int s_last;
    if (*p.err & ERR_LIST) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const long long step = *p.step;
    const long long next = (mode & STEP_ADVANCE) ? step + 1 : step;
    const int rr = (blockIdx.x * blockDim.x + tid) >> 5;
    // every block reads maxd2 and the list state before the last one records the decision
    const double rl = next_rlist<SETCOND>(p, SETCOND ? __ldcg(p.maxd2) : 0u);
    if (rr < p.n_rep) finalize_replica(p, rr, lane, next, rl);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.counters[3], 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid == 0) finalize_step<SETCOND>(p, mode, next, SETCOND ? __ldcg(p.maxd2) : 0u);
}

static int sm_count()
{
    int d = 0, n = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

void launch_step_a(const Params& p, int mode, cudaStream_t s, int grid_atoms)
{
    (void)grid_atoms;
    static const int n_sm = sm_count();
    constexpr int kWide = 16;   // MINB of the variant for grids of many blocks per SM
    const int blocks = (p.n_atoms + kStepAtoms - 1) / kStepAtoms;
    const int fin_blocks = (p.n_rep * 32 + 255) / 256;
    const bool wide = blocks >= kWide * n_sm;
    if (mode & STEP_SETCOND) {
        if (wide) k_step_a<true, kWide><<<blocks, kStepThreads, 0, s>>>(p, mode);
        else k_step_a<true, 10><<<blocks, kStepThreads, 0, s>>>(p, mode);
        if (p.n_rep > kInlineReps) k_step_fin<true><<<fin_blocks, 256, 0, s>>>(p, mode);
    } else {
        if (wide) k_step_a<false, kWide><<<blocks, kStepThreads, 0, s>>>(p, mode);
        else k_step_a<false, 10><<<blocks, kStepThreads, 0, s>>>(p, mode);
        if (p.n_rep > kInlineReps) k_step_fin<false><<<fin_blocks, 256, 0, s>>>(p, mode);
    }
}

// ---------------------------------------------------------------------------
// Velocities at the integer step (state stores v_{n+1/2} once stepping has
// started), forces in kJ/mol/nm, kinetic energy, Philox diagnostic.
// ---------------------------------------------------------------------------
__global__ void k_velocity_out(Params p, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_atoms) return;
    const int full = *p.kick_full;
    double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
    if (full) {
        double ax, ay, az;
        half_kick(p, p.species[i], p.slot_of[i], ax, ay, az);
        vx = vx + ax; vy = vy + ay; vz = vz + az;
    }
    out[3 * i + 0] = vx;
    out[3 * i + 1] = vy;
    out[3 * i + 2] = vz;
}

__global__ void k_force_out(Params p, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_atoms) return;
    const int slot = p.slot_of[i];
    out[3 * i + 0] = (double)p.fx[slot] * kFixInv;
    out[3 * i + 1] = (double)p.fy[slot] * kFixInv;
    out[3 * i + 2] = (double)p.fz[slot] * kFixInv;
}

// One block per replica, fixed traversal order -> deterministic sums.
__global__ void k_energy(Params p, double* ekin, long long* epot)
{
    __shared__ double s_k[256];
    __shared__ long long s_u[256];
    const int r = blockIdx.x;
    const int a0 = p.rep_off[r], a1 = p.rep_off[r + 1];
    const int full = *p.kick_full;
    double k = 0.0;
    long long u = 0;
    for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
        const int slot = p.slot_of[i];
        const int s = p.species[i];
        double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
        if (full) {
            double ax, ay, az;
            half_kick(p, s, slot, ax, ay, az);
            vx = vx + ax; vy = vy + ay; vz = vz + az;
        }
        k += 0.5 * p.mass[s] * (vx * vx + vy * vy + vz * vz);
        u += p.epot[slot];
    }
    s_k[threadIdx.x] = k;
    s_u[threadIdx.x] = u;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_k[threadIdx.x] += s_k[threadIdx.x + o];
            s_u[threadIdx.x] += s_u[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ekin[r] = s_k[0];
        epot[r] = s_u[0];
    }
}

__global__ void k_philox(unsigned long long seed, const uint4* ctr, long long n, uint4* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = philox4x32_10(ctr[i], make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

void launch_velocity_out(const Params& p, double* d_v_out, cudaStream_t s)
{
    k_velocity_out<<<(p.n_atoms + 255) / 256, 256, 0, s>>>(p, d_v_out);
}
void launch_force_out(const Params& p, double* d_f_out, cudaStream_t s)
{
    k_force_out<<<(p.n_atoms + 255) / 256, 256, 0, s>>>(p, d_f_out);
}
void launch_energy(const Params& p, double* d_ekin, long long* d_epot, cudaStream_t s)
{
    k_energy<<<p.n_rep, 256, 0, s>>>(p, d_ekin, d_epot);
}
void launch_philox(unsigned long long seed, const uint32_t* ctr, long long n, uint32_t* out,
                   cudaStream_t s)
{
    if (n <= 0) return;
    const long long blocks = (n + 255) / 256;
    k_philox<<<(unsigned)blocks, 256, 0, s>>>(seed, (const uint4*)ctr, n, (uint4*)out);
}

}  // namespace mdg
