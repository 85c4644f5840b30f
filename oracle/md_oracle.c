/*
 * FP64 CPU oracle for the ionising-MD hot path.  TEST INFRASTRUCTURE ONLY:
 * nothing in the product path may call this code; only tests, the smoke
 * check and the benchmark's CPU-baseline leg do.  It shares no source with
 * the CUDA library.
 *
 * Plain, slow, obviously correct:
 *   - forces are all-pairs O(N^2) in double, each atom summing over every
 *     other atom of its replica (no Newton-III shortcut, no cell list);
 *   - the collisional-radiative (CR) update visits atoms one by one in the
 *     order written in the paper's Sec. II.A reading below;
 *   - random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     (seed, atom, step).
 * Build with -ffp-contract=off so that no multiply-add is fused: the CR
 * decisions must reproduce the GPU's IEEE double operations bit for bit.
 *
 * Parity pins of every function are listed in the oracle's Python header
 * (oracle/oracle.py); the one function without a pin is stated there.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with a   */
/* Weyl-sequence key schedule.                                                */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Many blocks at once (tests): counter = (c0[i], c1[i], c2, c3). */
void orc_philox_many(uint64_t seed, const uint32_t* c0, const uint32_t* c1,
                     uint32_t c2, uint32_t c3, int64_t n, uint32_t* out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {c0[i], c1[i], c2, c3};
        orc_philox4x32_10(ctr, key, out + 4 * i);
    }
}

/* 53-bit uniform in [0,1) from two words: (a>>5)*2^26 + (b>>6), times 2^-53. */
double orc_u53(uint32_t a, uint32_t b)
{
    double hi = (double)(a >> 5);
    double lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* p = 1 - exp(-x) for x >= 0, written from the Taylor series with range     */
/* reduction (x = k/16 + r, 0 <= r < 1/16):                                   */
/*   1 - e^{-x} = (1 - E_k) + E_k * (1 - e^{-r}),  E_k = e^{-k/16} (table),  */
/*   1 - e^{-r} = r(1 - (r/2)(1 - (r/3)(1 - ... (1 - r/12)))),               */
/* i.e. the degree-12 Taylor polynomial in nested (Horner) form; the         */
/* truncation error is below r^13/13! < 1e-25.  inv[m] = 1/m (m = 1..12).    */
/* For x >= n_tab/16 the result is 1.                                         */
/* ------------------------------------------------------------------------ */
double orc_one_minus_exp_neg(double x, const double* etab, int n_tab, const double* inv)
{
    if (!(x > 0.0)) return 0.0;
    double xs = x * 16.0;
    if (xs >= (double)n_tab) return 1.0;
    int k = (int)xs;
    double r = x - (double)k * 0.0625;
    double t = 1.0;
    for (int m = 12; m >= 2; --m) {
        double rm = r * inv[m];
        t = 1.0 - rm * t;
    }
    double g = r * t;
    if (k == 0) return g;
    double ek = etab[k];
    return (1.0 - ek) + ek * g;
}

/* ------------------------------------------------------------------------ */
/* Charge-dependent LJ pair table, Sec. II.B, Eq. 11 (reading: the scale      */
/* c_i = 1 - q_i/Z_i multiplies sigma_i, epsilon unchanged), Lorentz-         */
/* Berthelot combination, c6 = 4 eps sigma^6, c12 = 4 eps sigma^12.           */
/* Type state (s, q) is row off[s] + q; off[] has n_species+1 entries.        */
/* ------------------------------------------------------------------------ */
void orc_lj_table(int n_species, const int* z, const double* sigma0, const double* eps0,
                  double* c6, double* c12)
{
    int off[65];
    off[0] = 0;
    for (int s = 0; s < n_species; ++s) off[s + 1] = off[s] + z[s] + 1;
    int nts = off[n_species];
    for (int si = 0; si < n_species; ++si)
        for (int qi = 0; qi <= z[si]; ++qi)
            for (int sj = 0; sj < n_species; ++sj)
                for (int qj = 0; qj <= z[sj]; ++qj) {
                    double sig_i = sigma0[si] * (1.0 - (double)qi / (double)z[si]);
                    double sig_j = sigma0[sj] * (1.0 - (double)qj / (double)z[sj]);
                    double sig = 0.5 * (sig_i + sig_j);
                    double eps = sqrt(eps0[si] * eps0[sj]);
                    double s2 = sig * sig;
                    double s6 = s2 * s2 * s2;
                    int a = off[si] + qi, b = off[sj] + qj;
                    c6[a * nts + b] = 4.0 * eps * s6;
                    c12[a * nts + b] = 4.0 * eps * s6 * s6;
                }
}

/* ------------------------------------------------------------------------ */
/* One pair: screened Coulomb (Sec. II.A, Eq. 2) plus screened LJ (Eq. 8).   */
/*   U_C = f qi qj e^{-k r}/r,  U_LJ = (c12/r^12 - c6/r^6) e^{-k r}           */
/*   F(r) = -dU/dr;  fr = F(r)/r, so the force on i is fr * (x_i - x_j).     */
/* The energy is shifted to zero at the cutoff (reading: the paper is silent */
/* on the cutoff treatment); the force is plainly truncated.                 */
/* ------------------------------------------------------------------------ */
static void pair_terms(double r, double qq_f, double c6, double c12, double kappa,
                       double* fr, double* u)
{
    double e = exp(-kappa * r);
    double ir = 1.0 / r;
    double ir2 = ir * ir;
    double ir6 = ir2 * ir2 * ir2;
    double lj = c12 * ir6 * ir6 - c6 * ir6;               /* c12/r^12 - c6/r^6 */
    double dlj = 12.0 * c12 * ir6 * ir6 - 6.0 * c6 * ir6; /* -r d/dr of lj    */
    double uc = qq_f * ir;
    /* -d/dr [uc e] = e (qq_f/r^2 + kappa qq_f/r);  -d/dr [lj e] = e (dlj/r + kappa lj) */
    double f_c = e * (qq_f * ir2 + kappa * qq_f * ir);
    double f_lj = e * (dlj * ir + kappa * lj);
    *fr = (f_c + f_lj) * ir;
    *u = (uc + lj) * e;
}

void orc_pair(double r, double qi, double qj, double c6, double c12, double kappa,
              double coulomb_f, double rc, int lj_on, double* fr, double* u)
{
    double qq = coulomb_f * qi * qj;
    double a6 = lj_on ? c6 : 0.0, a12 = lj_on ? c12 : 0.0;
    double f, uu, fc, uc;
    pair_terms(r, qq, a6, a12, kappa, &f, &uu);
    pair_terms(rc, qq, a6, a12, kappa, &fc, &uc);
    *fr = f;
    *u = uu - uc;
}

/* ------------------------------------------------------------------------ */
/* Hybrid ion-sphere / Debye potential of one ion (Sec. II.A, Eqs. 4-7).     */
/* Reading (the paper prints neither the coefficients nor the pair form):    */
/*   R  = (3 Q / (4 pi n_e))^{1/3}                          (ion sphere, Eq. 4) */
/*   r' = lambda ((R/lambda)^3 + 1)^{1/3} - lambda,  lambda = 1/kappa  (Eq. 7) */
/*   phi(r) = Q/r + c1 - c2 r^2            for r <  r'  (ion-sphere form)      */
/*   phi(r) = c3 exp(-kappa r) / r         for r >= r'  (Debye form, Eq. 2)    */
/* with c1, c2, c3 fixed by the continuity of phi, phi' and phi'' at r' (the */
/* matching the paper describes; Eq. 6 lists the four terms).  Solving the   */
/* three conditions with x = kappa r' and D = 3 + 3x + x^2:                  */
/*   c3 = 3 Q e^x / D,  c2 = -Q kappa^2 / (2 r' D),                           */
/*   c1 = -Q kappa (3 + 3x/2) / D.                                            */
/* (With Eq. 7, D = kappa^2 R^3 / r', so c2 = -Q/(2R^3) = -2 pi n_e / 3: the  */
/* inner curvature is the uniform electron background's, as in Eq. 5.)      */
/* r' is evaluated as lambda s^3 / (t^2 + t + 1), s = R/lambda,              */
/* t = (1 + s^3)^{1/3}, which equals Eq. 7 without its cancellation.  The    */
/* Debye amplitude is kept at r' (a = c3 e^{-x} = 3Q/D, phi = a             */
/* e^{-kappa (r - r')}/r), which does not overflow as lambda -> 0.           */
/* Without an ion sphere (Q <= 0, n_e <= 0 or kappa <= 0) r' = 0 and        */
/* phi = Q exp(-kappa r)/r (the Debye form; Coulomb when kappa = 0).         */
/* co = {r', c1, c2, a}.                                                      */
/* ------------------------------------------------------------------------ */
void orc_hybrid_coeffs(double Q, double ne, double kappa, double co[4])
{
    if (!(Q > 0.0) || !(ne > 0.0) || !(kappa > 0.0)) {
        co[0] = 0.0; co[1] = 0.0; co[2] = 0.0; co[3] = Q;
        return;
    }
    double lam = 1.0 / kappa;
    double R = cbrt(3.0 * Q / (4.0 * 3.14159265358979323846 * ne));
    double s = R / lam;
    double s3 = s * s * s;
    double t = cbrt(1.0 + s3);
    double rp = lam * s3 / (t * t + t + 1.0);
    double x = kappa * rp;
    double D = 3.0 + 3.0 * x + x * x;
    co[0] = rp;
    co[1] = -Q * kappa * (3.0 + 1.5 * x) / D;
    co[2] = -Q * kappa * kappa / (2.0 * rp * D);
    co[3] = 3.0 * Q / D;
}

/* phi(r) of one ion and -dphi/dr (coefficients from orc_hybrid_coeffs). */
void orc_hybrid_phi(double Q, const double co[4], double kappa, double r, double* phi, double* mdphi)
{
    if (r < co[0]) {
        *phi = Q / r + co[1] - co[2] * r * r;
        *mdphi = Q / (r * r) + 2.0 * co[2] * r;
    } else {
        double e = exp(-kappa * (r - co[0]));
        *phi = co[3] * e / r;
        *mdphi = co[3] * e * (1.0 + kappa * r) / (r * r);
    }
}

/* One pair with the hybrid electrostatics (reading: the pair energy is the  */
/* mean of the two ions' views, U_C = f (q_j phi_i(r) + q_i phi_j(r)) / 2)   */
/* plus the screened LJ of Eq. 8; energy shifted to zero at the cutoff.      */
void orc_pair_hybrid(double r, double qi, double qj, double c6, double c12, double kappa,
                     double ne, double coulomb_f, double rc, int lj_on, double* fr, double* u)
{
    double coi[4], coj[4];
    orc_hybrid_coeffs(qi, ne, kappa, coi);
    orc_hybrid_coeffs(qj, ne, kappa, coj);
    double a6 = lj_on ? c6 : 0.0, a12 = lj_on ? c12 : 0.0;
    double flj, ulj, flj_c, ulj_c;
    pair_terms(r, 0.0, a6, a12, kappa, &flj, &ulj);
    pair_terms(rc, 0.0, a6, a12, kappa, &flj_c, &ulj_c);
    double pi, mi, pj, mj, pic, mic, pjc, mjc;
    orc_hybrid_phi(qi, coi, kappa, r, &pi, &mi);
    orc_hybrid_phi(qj, coj, kappa, r, &pj, &mj);
    orc_hybrid_phi(qi, coi, kappa, rc, &pic, &mic);
    orc_hybrid_phi(qj, coj, kappa, rc, &pjc, &mjc);
    double h = 0.5 * coulomb_f;
    *fr = flj + h * (qj * mi + qi * mj) / r;
    *u = (ulj - ulj_c) + h * ((qj * pi + qi * pj) - (qj * pic + qi * pjc));
}

/* ------------------------------------------------------------------------ */
/* All-pairs forces.  x: [3n] AoS; ts: type-state row; q: charge; frag:       */
/* fragment id (LJ excluded within one fragment, Sec. II.B); rep_off: [R+1]; */
/* box: [3R] (zeros = vacuum, else minimum image); kappa: [R] 1/lambda_D;   */
/* ne: [R] free-electron density (nm^-3) for the hybrid electrostatics, or   */
/* NULL for the Debye-screened Coulomb term.                                  */
/* Output: f [3n], u_atom [n] (half of every pair energy), n_pairs (i<j).    */
/* ------------------------------------------------------------------------ */
void orc_forces(int n, const double* x, const int* ts, const double* q, const int* frag,
                int n_rep, const int* rep_off, const double* box, const double* kappa,
                const double* ne, double rc, double coulomb_f, int nts, const double* c6,
                const double* c12, double* f, double* u_atom, int64_t* n_pairs)
{
    int64_t pairs = 0;
    for (int r = 0; r < n_rep; ++r) {
        int a0 = rep_off[r], a1 = rep_off[r + 1];
        const double* L = box + 3 * r;
        int periodic = (L[0] > 0.0 && L[1] > 0.0 && L[2] > 0.0);
        double kap = kappa[r];
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
        for (int i = a0; i < a1; ++i) {
            double fx = 0.0, fy = 0.0, fz = 0.0, ui = 0.0;
            for (int j = a0; j < a1; ++j) {
                if (j == i) continue;
                double d[3];
                for (int k = 0; k < 3; ++k) {
                    d[k] = x[3 * i + k] - x[3 * j + k];
                    if (periodic) d[k] -= L[k] * nearbyint(d[k] / L[k]);
                }
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < rc * rc)) continue;
                if (j > i) ++pairs;
                double rr = sqrt(r2);
                int lj_on = (frag[i] != frag[j]);
                double fr, u;
                if (ne)
                    orc_pair_hybrid(rr, q[i], q[j], c6[ts[i] * nts + ts[j]], c12[ts[i] * nts + ts[j]],
                                    kap, ne[r], coulomb_f, rc, lj_on, &fr, &u);
                else
                    orc_pair(rr, q[i], q[j], c6[ts[i] * nts + ts[j]], c12[ts[i] * nts + ts[j]],
                             kap, coulomb_f, rc, lj_on, &fr, &u);
                fx += fr * d[0];
                fy += fr * d[1];
                fz += fr * d[2];
                ui += 0.5 * u;
            }
            f[3 * i + 0] = fx;
            f[3 * i + 1] = fy;
            f[3 * i + 2] = fz;
            if (u_atom) u_atom[i] = ui;
        }
    }
    if (n_pairs) *n_pairs = pairs;
}

/* Forces on a subset of atoms (sampled checks of large systems). */
void orc_forces_subset(int n, const double* x, const int* ts, const double* q, const int* frag,
                       const int* rep_of, const int* rep_off, const double* box,
                       const double* kappa, const double* ne, double rc, double coulomb_f, int nts,
                       const double* c6, const double* c12, int n_sel, const int* sel,
                       double* f_sel)
{
    (void)n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int s = 0; s < n_sel; ++s) {
        int i = sel[s];
        int r = rep_of[i];
        const double* L = box + 3 * r;
        int periodic = (L[0] > 0.0 && L[1] > 0.0 && L[2] > 0.0);
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int j = rep_off[r]; j < rep_off[r + 1]; ++j) {
            if (j == i) continue;
            double d[3];
            for (int k = 0; k < 3; ++k) {
                d[k] = x[3 * i + k] - x[3 * j + k];
                if (periodic) d[k] -= L[k] * nearbyint(d[k] / L[k]);
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            double fr, u;
            if (ne)
                orc_pair_hybrid(sqrt(r2), q[i], q[j], c6[ts[i] * nts + ts[j]], c12[ts[i] * nts + ts[j]],
                                kappa[r], ne[r], coulomb_f, rc, frag[i] != frag[j], &fr, &u);
            else
                orc_pair(sqrt(r2), q[i], q[j], c6[ts[i] * nts + ts[j]], c12[ts[i] * nts + ts[j]],
                         kappa[r], coulomb_f, rc, frag[i] != frag[j], &fr, &u);
            fx += fr * d[0];
            fy += fr * d[1];
            fz += fr * d[2];
        }
        f_sel[3 * s + 0] = fx;
        f_sel[3 * s + 1] = fy;
        f_sel[3 * s + 2] = fz;
    }
}

/* ------------------------------------------------------------------------ */
/* Pulse fluence per step.  Photons per nm^2 arriving in [t_n, t_{n+1}],     */
/* t_n = t_start + n dt.  Gaussian pulse: F * (Phi(b) - Phi(a)) with         */
/* sigma_t = FWHM / (2 sqrt(2 ln 2)), written with erfc on the side of the   */
/* centre where it does not cancel.  Flat-top pulse of width FWHM: F times   */
/* the overlap fraction.  Pulses are summed in the order given.              */
/* pulses: [n_pulses][5] = photon keV, FWHM fs, fluence ph/um^2, centre fs,  */
/* shape (0 Gaussian, 1 flat-top).                                            */
/* ------------------------------------------------------------------------ */
void orc_pulse_table(int n_pulses, const double* pulses, double t_start_fs, double dt_fs,
                     int n_steps, double* dF)
{
    for (int n = 0; n < n_steps; ++n) {
        double ta = t_start_fs + (double)n * dt_fs;
        double tb = t_start_fs + (double)(n + 1) * dt_fs;
        double acc = 0.0;
        for (int p = 0; p < n_pulses; ++p) {
            const double* P = pulses + 5 * p;
            double fwhm = P[1], flu = P[2] * 1e-6, t0 = P[3];
            int shape = (int)P[4];
            double frac;
            if (shape == 0) {
                double sig = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
                double s = sig * sqrt(2.0);
                double za = (ta - t0) / s, zb = (tb - t0) / s;
                if (za >= 0.0)
                    frac = 0.5 * (erfc(za) - erfc(zb));
                else if (zb <= 0.0)
                    frac = 0.5 * (erfc(-zb) - erfc(-za));
                else
                    frac = 1.0 - 0.5 * (erfc(-za) + erfc(zb));
            } else {
                double lo = t0 - 0.5 * fwhm, hi = t0 + 0.5 * fwhm;
                double a = ta > lo ? ta : lo;
                double b = tb < hi ? tb : hi;
                frac = b > a ? (b - a) / fwhm : 0.0;
            }
            acc = acc + flu * frac;
        }
        dF[n] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* One collisional-radiative step for all atoms (reading "RCM-1" of Sec.     */
/* II.A: the paper assigns integer charges stochastically from photo- and    */
/* electron-impact ionisation, Auger decay and their inverse processes; the  */
/* rates below are that reading, with at most one event per atom per step).  */
/*                                                                            */
/* Per replica r the caller passes the plasma scalars of the previous step:  */
/*   dF[r] photons/nm^2 this step, ne_dt[r] = n_e dt, and the Te-grid         */
/*   position it0[r], wt[r] (linear interpolation weight).                   */
/* Per atom (species s, charge q, K-hole h, type state ts = off[s]+q):       */
/*   a_PI  = sigma[ts][h] * dF                                                */
/*   a_A   = h ? dt/tau_A[s] : 0                        (auger_dt[s])         */
/*   a_CI  = q < Z ? ne_dt * K_CI(ts, Te) : 0                                 */
/*   a_REC = q > 0 and h == 0 ? ne_dt * K_REC(ts, Te) : 0                     */
/*   lambda = ((a_PI + a_A) + a_CI) + a_REC,  p = 1 - exp(-lambda)            */
/*   (w0..w3) = Philox(ctr = (local id, step, 0, 0), key = seed)             */
/*   u0 = u53(w0, w1), u1 = u53(w2, w3)                                       */
/*   if u0 < p: the first channel whose running sum exceeds u1*lambda fires  */
/*   (order PI, A, CI, REC; if rounding leaves none, the last nonzero one).  */
/* K(ts, Te) = K[i0] + w (K[i0+1] - K[i0]).                                   */
/* Events: PI  q+1, h -> 1 if Z >= 3, h was 0, Z - q' >= 2 (K hole opened),  */
/*             h -> 0 if q' = Z; dE = E_PI[ts][h]                             */
/*         A   q+1, h -> 0; dE = E_A[s]                                       */
/*         CI  q+1, h -> 0 if q' = Z; dE = -IP[ts]                            */
/*         REC q-1; dE = +IP[ts-1]                                            */
/* Outputs: q, h updated; per replica dNe and dE (meV) summed; per-channel   */
/* event counts [R][4].  Returns 0.                                           */
/* ------------------------------------------------------------------------ */
int orc_cr_step(int n, const uint8_t* species, uint8_t* q, uint8_t* h, const int* local_id,
                const int* rep_of, int64_t step, const uint64_t* seed, const double* dF,
                const double* ne_dt, const int* it0, const double* wt, int n_species,
                const int* z, const double* sigma_pi, const double* auger_dt,
                const double* k_ci, const double* k_rec, int n_te, const int64_t* ip_mev,
                const int64_t* e_pi_mev, const int64_t* e_auger_mev, const double* etab,
                int n_etab, const double* inv, int64_t* dNe, int64_t* dE, int64_t* counts)
{
    int off[65];
    off[0] = 0;
    for (int s = 0; s < n_species; ++s) off[s + 1] = off[s] + z[s] + 1;
    for (int i = 0; i < n; ++i) {
        int s = species[i];
        int Z = z[s];
        int qi = q[i], hi = h[i];
        int r = rep_of[i];
        int ts = off[s] + qi;
        double a_pi = sigma_pi[2 * ts + hi] * dF[r];
        double a_a = hi ? auger_dt[s] : 0.0;
        double a_ci = 0.0, a_rec = 0.0;
        int i0 = it0[r];
        double w = wt[r];
        if (qi < Z) {
            const double* K = k_ci + (int64_t)ts * n_te;
            a_ci = ne_dt[r] * (K[i0] + w * (K[i0 + 1] - K[i0]));
        }
        if (qi > 0 && hi == 0) {
            const double* K = k_rec + (int64_t)ts * n_te;
            a_rec = ne_dt[r] * (K[i0] + w * (K[i0 + 1] - K[i0]));
        }
        double c1 = a_pi + a_a;
        double c2 = c1 + a_ci;
        double lam = c2 + a_rec;
        if (!(lam > 0.0)) continue;
        double p = orc_one_minus_exp_neg(lam, etab, n_etab, inv);
        uint32_t key[2] = {(uint32_t)seed[r], (uint32_t)(seed[r] >> 32)};
        uint32_t ctr[4] = {(uint32_t)local_id[i], (uint32_t)step, 0u, 0u};
        uint32_t w4[4];
        orc_philox4x32_10(ctr, key, w4);
        double u0 = orc_u53(w4[0], w4[1]);
        if (!(u0 < p)) continue;
        double u1 = orc_u53(w4[2], w4[3]);
        double t = u1 * lam;
        int ch;
        if (t < a_pi) ch = 0;
        else if (t < c1) ch = 1;
        else if (t < c2) ch = 2;
        else if (t < lam) ch = 3;
        else ch = a_rec > 0.0 ? 3 : (a_ci > 0.0 ? 2 : (a_a > 0.0 ? 1 : 0));
        int qn = qi, hn = hi;
        int64_t de = 0;
        if (ch == 0) {
            qn = qi + 1;
            de = e_pi_mev[2 * ts + hi];
            if (qn == Z) hn = 0;
            else if (Z >= 3 && hi == 0 && Z - qn >= 2) hn = 1;
        } else if (ch == 1) {
            qn = qi + 1;
            hn = 0;
            de = e_auger_mev[s];
        } else if (ch == 2) {
            qn = qi + 1;
            if (qn == Z) hn = 0;
            de = -ip_mev[ts];
        } else {
            qn = qi - 1;
            de = ip_mev[ts - 1];
        }
        q[i] = (uint8_t)qn;
        h[i] = (uint8_t)hn;
        dNe[r] += (ch == 3) ? -1 : 1;
        dE[r] += de;
        counts[4 * r + ch] += 1;
    }
    return 0;
}

/* Tables used by orc_one_minus_exp_neg: etab[k] = e^{-k/16}, inv[m] = 1/m. */
void orc_exp_tables(double* etab, int n_tab, double* inv)
{
    for (int k = 0; k < n_tab; ++k) etab[k] = exp(-(double)k / 16.0);
    inv[0] = 0.0;
    for (int m = 1; m <= 12; ++m) inv[m] = 1.0 / (double)m;
}

/* Vectorised p(x) for tests. */
void orc_one_minus_exp_neg_many(int64_t n, const double* x, double* p, const double* etab,
                                int n_tab, const double* inv)
{
    for (int64_t i = 0; i < n; ++i) p[i] = orc_one_minus_exp_neg(x[i], etab, n_tab, inv);
}

/* Arbitrary counters (tests): ctr4 is [n][4]. */
void orc_philox_blocks(uint64_t seed, const uint32_t* ctr4, int64_t n, uint32_t* out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr4 + 4 * i, key, out + 4 * i);
}
