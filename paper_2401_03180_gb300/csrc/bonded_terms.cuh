// Bonded terms of the native structure (Sec. II.B, Eqs. 9-10; the harmonic
// angle term is the one Sec. III names for the methane clusters):
//
//   bond i-j        V = c D_e (1 - e^{-beta (r - b_e)})^2        (Morse)
//   angle i-j-k     V = c (k_theta / 2) (theta - theta_0)^2      (vertex j)
//   c = max(0, 1 - zbar / N), zbar the summed charge of the term's N atoms (Eq. 9)
//
// One thread per term.  The displacements are formed in FP64 from the FP64
// positions (minimum image of the replica's box), then evaluated in FP32 on
// the mixed path and FP64 on the FP64 path.  Each atom's share is converted
// to 64-bit fixed point (2^-32 kJ/mol/nm) and added with one integer atomic
// per component to the same per-slot sums as the pair forces, so the totals
// are exact integer sums whatever the order of the atomics.  The force
// kernel evaluates them in a prologue (k_pair.cu).
#pragma once

#include "md_internal.cuh"

namespace mdg {
namespace bonded {

__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }

__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * 4294967296.0f); }
__device__ __forceinline__ long long to_fix(double v) { return __double2ll_rn(v * 4294967296.0); }

// Adds v to a fixed-point sum; a value beyond 2^30 (or not finite) raises the
// overflow flag instead.
template <typename T>
__device__ __forceinline__ void add_fix(long long* dst, T v, unsigned* err)
{
    if (!(m_abs(v) < (T)1.073741824e9)) {
        atomicOr(err, ERR_OVERFLOW);
        return;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)to_fix(v));
}

// d minus the nearest box vector (periodic replicas; |d| < L since positions
// are kept inside the box).
__device__ __forceinline__ void min_image(const Params& p, int r, double d[3])
{
    const Grid& g = p.grid_b[r];
    if (!g.periodic) return;
    for (int k = 0; k < 3; ++k) {
        const int o = beyond_half(d[k], g.box[k]);
        if (o > 0) d[k] -= g.box[k];
        else if (o < 0) d[k] += g.box[k];
    }
}

template <typename T>
__device__ __forceinline__ T scale_of(int qsum, int n_atoms)
{
    const T c = (T)1 - (T)qsum / (T)n_atoms;
    return c > (T)0 ? c : (T)0;
}

template <typename T, bool ENERGY>
__device__ void bond_term(const Params& p, const T* par, int t)
{
    const int4 b = __ldg(&p.bonds[t]);
    const int i = b.x, j = b.y;
    double d64[3] = {p.x[i] - p.x[j], p.y[i] - p.y[j], p.z[i] - p.z[j]};
    min_image(p, p.rep[i], d64);
    const T dx = (T)d64[0], dy = (T)d64[1], dz = (T)d64[2];
    const T r = m_sqrt(dx * dx + dy * dy + dz * dz);
    const T De = par[3 * b.z], be = par[3 * b.z + 1], beta = par[3 * b.z + 2];
    const T om = -m_expm1(-beta * (r - be));          // 1 - e^{-beta (r - b_e)}, no cancellation
    const T c = scale_of<T>((int)p.q[i] + (int)p.q[j], 2);
    // F_i = -c dV/dr (d / r), dV/dr = 2 D_e beta e^{-beta (r - b_e)} (1 - e^{-beta (r - b_e)})
    const T fr = -c * ((T)2 * De * beta * ((T)1 - om) * om) / r;
    const int si = p.slot_of[i], sj = p.slot_of[j];
    const T f[3] = {fr * dx, fr * dy, fr * dz};
    long long* sum[3] = {p.fx, p.fy, p.fz};
    for (int k = 0; k < 3; ++k) {
        add_fix(sum[k] + si, f[k], p.err);
        add_fix(sum[k] + sj, -f[k], p.err);
    }
    if constexpr (ENERGY) {
        const T u = (T)0.5 * (c * De * om * om);
        add_fix(p.epot + si, u, p.err);
        add_fix(p.epot + sj, u, p.err);
    }
}

template <typename T, bool ENERGY>
__device__ void angle_term(const Params& p, const T* par, int t)
{
    const int4 a = __ldg(&p.angles[t]);
    const int i = a.x, j = a.y, k = a.z;
    const int r = p.rep[j];
    double u64[3] = {p.x[i] - p.x[j], p.y[i] - p.y[j], p.z[i] - p.z[j]};
    double w64[3] = {p.x[k] - p.x[j], p.y[k] - p.y[j], p.z[k] - p.z[j]};
    min_image(p, r, u64);
    min_image(p, r, w64);
    const T u[3] = {(T)u64[0], (T)u64[1], (T)u64[2]};
    const T w[3] = {(T)w64[0], (T)w64[1], (T)w64[2]};
    const T ru2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T rw2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const T uw = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
    const T cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
    const T sn = m_sqrt(cx * cx + cy * cy + cz * cz);   // |u| |w| sin(theta)
    const T inv = (T)1 / m_sqrt(ru2 * rw2);             // 1 / (|u| |w|)
    const T theta = m_atan2(sn, uw);                    // accurate at every angle
    const T cs = uw * inv;
    T sint = sn * inv;
    if (sint < (T)1e-6) sint = (T)1e-6;                 // collinear: direction undefined, force bounded
    const T kt = par[2 * a.w], th0 = par[2 * a.w + 1];
    const T c = scale_of<T>((int)p.q[i] + (int)p.q[j] + (int)p.q[k], 3);
    const T dth = theta - th0;
    // -dV/dx_i = (c k_theta (theta - theta_0) / sin theta) d(cos theta)/dx_i, likewise for k
    const T g = c * kt * dth / sint;
    const T au = cs / ru2, aw = cs / rw2;
    T fi[3], fk[3];
    for (int d = 0; d < 3; ++d) {
        fi[d] = g * (w[d] * inv - au * u[d]);
        fk[d] = g * (u[d] * inv - aw * w[d]);
    }
    const int si = p.slot_of[i], sj = p.slot_of[j], sk = p.slot_of[k];
    long long* sum[3] = {p.fx, p.fy, p.fz};
    for (int d = 0; d < 3; ++d) {
        add_fix(sum[d] + si, fi[d], p.err);
        add_fix(sum[d] + sk, fk[d], p.err);
        add_fix(sum[d] + sj, -(fi[d] + fk[d]), p.err);
    }
    if constexpr (ENERGY) {
        const T e = c * ((T)0.5 * kt * dth * dth) / (T)3;
        add_fix(p.epot + si, e, p.err);
        add_fix(p.epot + sj, e, p.err);
        add_fix(p.epot + sk, e, p.err);
    }
}


}  // namespace bonded
}  // namespace mdg
