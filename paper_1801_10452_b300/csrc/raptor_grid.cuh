// raptor_grid.cuh -- GRMHD-shaped snapshot sampling on a modified Kerr-Schild grid.
//
// Device layout: snapshots are interleaved per cell, [snap][x2][x1][8] FP32 (32 bytes per
// cell, 32-byte aligned), so one corner of the bilinear stencil is two 16-byte vector loads
// through the read-only path; the host transposes the caller's [snap][field][x2][x1]
// planes into this layout once, at load time.  A 256 x 256 snapshot is 2 MiB and stays
// resident in the 126 MB L2 across the many rays that sample it.
#pragma once

#include "raptor_physics.cuh"

namespace raptor {

template <typename T>
struct NewtonTol;
template <>
struct NewtonTol<double> { static constexpr double v = 1e-14; };
template <>
struct NewtonTol<float> { static constexpr float v = 1e-7f; };

// App. A.2: theta = pi x2 + (1-h)/2 sin(2 pi x2) inverted by Newton-Raphson from
// x2 = theta/pi (FP64: from the FP32 root), resetting to 0.05 outside [0, 1] or where f'
// vanishes, stopping when the update is below tolerance or after 20 iterations.
template <typename T>
RAPTOR_HD T newton_x2(T theta, T h) {
    T xv = theta * T(1.0 / kPi);
    // FP64: start from the FP32 root (tolerance 1e-7), so that one or two FP64 iterations
    // reach the FP64 tolerance; the converged root is the same
    if constexpr (std::is_same<T, double>::value) xv = (double)newton_x2<float>((float)theta, (float)h);
    const T oh = T(1) - h;
    for (int it = 0; it < 20; ++it) {
        T s, c;
        sc(T(2.0 * kPi) * xv, &s, &c);
        const T f = T(kPi) * xv + T(0.5) * oh * s - theta;
        const T fp = T(kPi) * (T(1) + oh * c);
        T xn;
        if (fabs(fp) < T(1e-12)) {
            xn = T(0.05);
        } else {
            xn = xv - dv(f, fp);
            if (xn < T(0) || xn > T(1)) xn = T(0.05);
        }
        const T d = fabs(xn - xv);
        xv = xn;
        if (d < NewtonTol<T>::v) break;
    }
    return xv;
}

// FP32 inversion from a table: x2 at the kX2TabN + 1 angles theta_i = i pi / kX2TabN
// (converged FP64 Newton roots, filled on the host when the plasma is loaded), linear
// interpolation between the two nodes around theta (error ~(pi / kX2TabN)^2 x2'' / 8 < 1e-6),
// then one Newton step (quadratic: below FP32 rounding).  Outside [0, pi]: newton_x2.
constexpr int kX2TabN = 1024;
__device__ __forceinline__ float x2_from_table(const float* tab, float theta, float h) {
    const float u = theta * (float)(kX2TabN / kPi);
    if (!(u >= 0.f && u <= (float)kX2TabN)) return newton_x2<float>(theta, h);
    const int i = min((int)u, kX2TabN - 1);
    const float w = u - (float)i;
    const float x0 = __ldg(tab + i), x1 = __ldg(tab + i + 1);
    const float xv = fmaf(w, x1 - x0, x0);
    float sn, cs;
    sc(2.f * (float)kPi * xv, &sn, &cs);
    const float oh = 1.f - h;
    const float f = (float)kPi * xv + 0.5f * oh * sn - theta;
    const float fp = (float)kPi * (1.f + oh * cs);
    return xv - f * rcp_nr(fp);
}

// Bilinear cell-centred interpolation of the 8 primitives of snapshot s at fractional
// index (fi, fj) (clamped to edge cells).  Vector loads of the interleaved cells.
template <typename T>
RAPTOR_HD void bilinear8(const Params& p, int s, int i0, int j0, T wi, T wj, T out[8]) {
    const float4* g = reinterpret_cast<const float4*>(p.grid) + ((long long)s * p.n2 * p.n1) * 2;
    const long long c00 = ((long long)j0 * p.n1 + i0) * 2, c01 = c00 + (long long)p.n1 * 2;
#ifdef __CUDA_ARCH__
    const float4 a0 = __ldg(g + c00), a1 = __ldg(g + c00 + 1), b0 = __ldg(g + c00 + 2), b1 = __ldg(g + c00 + 3);
    const float4 c0 = __ldg(g + c01), c1 = __ldg(g + c01 + 1), d0 = __ldg(g + c01 + 2), d1 = __ldg(g + c01 + 3);
#else
    const float4 a0 = g[c00], a1 = g[c00 + 1], b0 = g[c00 + 2], b1 = g[c00 + 3];
    const float4 c0 = g[c01], c1 = g[c01 + 1], d0 = g[c01 + 2], d1 = g[c01 + 3];
#endif
    const T w00 = (T(1) - wi) * (T(1) - wj), w10 = wi * (T(1) - wj), w01 = (T(1) - wi) * wj, w11 = wi * wj;
    out[0] = w00 * T(a0.x) + w10 * T(b0.x) + w01 * T(c0.x) + w11 * T(d0.x);
    out[1] = w00 * T(a0.y) + w10 * T(b0.y) + w01 * T(c0.y) + w11 * T(d0.y);
    out[2] = w00 * T(a0.z) + w10 * T(b0.z) + w01 * T(c0.z) + w11 * T(d0.z);
    out[3] = w00 * T(a0.w) + w10 * T(b0.w) + w01 * T(c0.w) + w11 * T(d0.w);
    out[4] = w00 * T(a1.x) + w10 * T(b1.x) + w01 * T(c1.x) + w11 * T(d1.x);
    out[5] = w00 * T(a1.y) + w10 * T(b1.y) + w01 * T(c1.y) + w11 * T(d1.y);
    out[6] = w00 * T(a1.z) + w10 * T(b1.z) + w01 * T(c1.z) + w11 * T(d1.z);
    out[7] = w00 * T(a1.w) + w10 * T(b1.w) + w01 * T(c1.w) + w11 * T(d1.w);
}

// Plasma from the grid at KS point P (x = state position): n_e, Theta_e, B [G], u^mu and
// b^mu [G] in KS components.  Returns 1 emitting, 0 outside the grid or no plasma.
//   HARM primitives: gamma = sqrt(1 + g_ij U^i U^j), u^t = gamma / alpha,
//   u^i = U^i - gamma alpha g^{ti};  b^t = B^i u_i, b^i = (B^i + b^t u^i) / u^t;
//   units (Eq. 45): n_e = rho rho0 / (m_e + m_p), B = |b| c sqrt(4 pi rho0);
//   R-beta (Eq. 46): beta_p = (gamma_ad - 1) u / (b^2/2),
//   T_p/T_e = R_low/(1+beta_p^2) + R_high beta_p^2/(1+beta_p^2),
//   Theta_e = (m_p/m_e) (gamma_ad - 1) (u/rho) / (1 + T_p/T_e).
template <typename T>
RAPTOR_HD int grid_sample(const Params& p, const KSPoint<T>& P, const T x[4], int snap, T& ne, T& the,
                                           T& B, T u[4], T b[4]) {
    const T r = P.r;
    const T x1 = Real<T>::log_(r);
    if (x1 < RAPTOR_P(T, x1_min) || x1 > RAPTOR_P(T, x1_max)) return 0;
    const T h = RAPTOR_P(T, h_mks);
    T x2;
    if constexpr (std::is_same<T, float>::value) x2 = p.x2tab ? x2_from_table(p.x2tab, x[2], h) : newton_x2<T>(x[2], h);
    else x2 = newton_x2<T>(x[2], h);
    T fi = dv(x1 - RAPTOR_P(T, x1_min), RAPTOR_P(T, dx1)) - T(0.5);
    T fj = dv(x2, RAPTOR_P(T, dx2)) - T(0.5);
    int i0 = (int)floor(fi), j0 = (int)floor(fj);
    T wi = fi - T(i0), wj = fj - T(j0);
    if (i0 < 0) { i0 = 0; wi = T(0); }
    if (i0 > p.n1 - 2) { i0 = p.n1 - 2; wi = T(1); }
    if (j0 < 0) { j0 = 0; wj = T(0); }
    if (j0 > p.n2 - 2) { j0 = p.n2 - 2; wj = T(1); }
    T q[8];
    if (p.slow && p.n_snap > 1) {
        T fs = dv(x[0] - RAPTOR_P(T, t0), RAPTOR_P(T, dt_snap));
        fs = fmin(fmax(fs, T(0)), T(p.n_snap - 1));
        int s0 = (int)floor(fs);
        if (s0 > p.n_snap - 2) s0 = p.n_snap - 2;
        const T w = fs - T(s0);
        T q0[8], q1[8];
        bilinear8<T>(p, s0, i0, j0, wi, wj, q0);
        bilinear8<T>(p, s0 + 1, i0, j0, wi, wj, q1);
#pragma unroll
        for (int f = 0; f < 8; ++f) q[f] = (T(1) - w) * q0[f] + w * q1[f];
    } else {
        int s = snap < 0 ? 0 : (snap > p.n_snap - 1 ? p.n_snap - 1 : snap);
        bilinear8<T>(p, s, i0, j0, wi, wj, q);
    }
    const T rho = q[0], uu = q[1];
    if (!(rho > T(0)) || !(uu > T(0))) return 0;
    // MKS Jacobian: dr/dx1 = r, dtheta/dx2 = pi (1 + (1-h) cos 2 pi x2)
    T s2p, c2p;
    sc(T(2.0 * kPi) * x2, &s2p, &c2p);
    const T J1 = r, J2 = T(kPi) * (T(1) + (T(1) - h) * c2p);
    const T U1 = q[2], U2 = q[3], U3 = q[4];
    const T g11 = P.grr * J1 * J1, g22 = P.ghh * J2 * J2, g33 = P.gpp, g13 = P.grp * J1;
    const T qq = g11 * U1 * U1 + g22 * U2 * U2 + g33 * U3 * U3 + T(2) * g13 * U1 * U3;
    const T gam = Real<T>::sqrt_(T(1) + qq);
    const T opz = T(1) + P.z;
    const T alp = rsq(opz);                 // lapse, g^tt = -(1 + z)
    const T gti1 = dv(P.z, J1);                // g^{t x1} in MKS; g^{t x2} = g^{t x3} = 0
    const T ut = dv(gam, alp);
    const T u1 = U1 - gam * alp * gti1, u2 = U2, u3 = U3;
    // covariant spatial u_i (MKS)
    const T uc1 = J1 * (P.gtr * ut + P.grr * J1 * u1 + P.grp * u3);
    const T uc2 = g22 * u2;
    const T uc3 = P.gtp * ut + P.grp * J1 * u1 + P.gpp * u3;
    const T B1 = q[5], B2 = q[6], B3 = q[7];
    const T bt = B1 * uc1 + B2 * uc2 + B3 * uc3;
    const T iut = dv(T(1), ut);
    const T b1 = (B1 + bt * u1) * iut, b2 = (B2 + bt * u2) * iut, b3 = (B3 + bt * u3) * iut;
    // KS components
    u[0] = ut; u[1] = J1 * u1; u[2] = J2 * u2; u[3] = u3;
    T bk[4] = {bt, J1 * b1, J2 * b2, b3};
    T bc[4];
    ks_lower(P, bk, bc);
    const T bsq = bc[0] * bk[0] + bc[1] * bk[1] + bc[2] * bk[2] + bc[3] * bk[3];
    if (!(bsq > T(0))) return 0;
    const T gm1 = RAPTOR_P(T, gam) - T(1);
    ne = rho * RAPTOR_P(T, rho0_ne);
    B = Real<T>::sqrt_(bsq) * RAPTOR_P(T, B_unit);
    const T betap = dv(gm1 * uu, T(0.5) * bsq);
    const T b2p = betap * betap;
    const T R = dv(RAPTOR_P(T, r_low), T(1) + b2p) + dv(RAPTOR_P(T, r_high) * b2p, T(1) + b2p);
    the = dv(T(kMp / kMe) * gm1 * dv(uu, rho), T(1) + R);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = bk[i] * RAPTOR_P(T, B_unit);
    return 1;
}

// Plasma + frequency ratio at state (x, k) in type T.  Returns 1 emitting, 0 no plasma,
// -1 error.  On success fills ne, the, B, g = nu_fluid/nu_obs and sinb.
template <typename T>
RAPTOR_HD int plasma_sample_sc(const Params& p, const T x[4], const T k[4], T sn, T cs, int snap, T& ne, T& the,
                               T& B, T& g, T& sinb, int kepler = -1) {
    KSPoint<T> P;
    ks_point_sc(RAPTOR_P(T, a), x[1], sn, cs, P);
    T u[4], kc[4];
    T kb;  // k . b_hat
    if (p.kind == 0) {
        const int ok = analytic_velocity(RAPTOR_P(T, a), RAPTOR_P(T, r_isco), P, u, kepler);
        if (ok < 0) return -1;
        const T r = x[1];
        if constexpr (std::is_same<T, float>::value) {
            // three power laws of one radius: one logarithm, three exponentials
            const float l2r = log2f(r);
            ne = p.f.n0 * exp2f(p.f.n_pow * l2r);
            the = p.f.the0 * exp2f(p.f.the_pow * l2r);
            B = p.f.B0 * exp2f(p.f.B_pow * l2r);
        } else {
            // one logarithm, three exponentials (r^n = e^{n ln r})
            const T lr = Real<T>::log_(r);
            ne = RAPTOR_P(T, n0) * Real<T>::exp_(RAPTOR_P(T, n_pow) * lr);
            the = RAPTOR_P(T, the0) * Real<T>::exp_(RAPTOR_P(T, the_pow) * lr);
            B = RAPTOR_P(T, B0) * Real<T>::exp_(RAPTOR_P(T, B_pow) * lr);
        }
        ks_lower(P, k, kc);
        g = kc[0] * u[0] + kc[1] * u[1] + kc[2] * u[2] + kc[3] * u[3];
        const T u_phi = P.gtp * u[0] + P.grp * u[1] + P.gpp * u[3];
        const T kv = kc[3] + u_phi * g;
        kb = kv * rsq(P.gpp + u_phi * u_phi);
    } else {
        T b[4];
        const int ok = grid_sample<T>(p, P, x, snap, ne, the, B, u, b);
        if (ok <= 0) return ok;
        ks_lower(P, k, kc);
        g = kc[0] * u[0] + kc[1] * u[1] + kc[2] * u[2] + kc[3] * u[3];
        kb = dv(kc[0] * b[0] + kc[1] * b[1] + kc[2] * b[2] + kc[3] * b[3], B);
    }
    if (!(g > T(0))) return -1;
    // cos theta_B = (k_phys . b) / (g |b|) with k_phys = -k
    T cb = dv(-kb, g);
    cb = fmin(fmax(cb, T(-1)), T(1));
    sinb = Real<T>::sqrt_(T(1) - cb * cb);
    return 1;
}

}  // namespace raptor

namespace raptor {
// plasma_sample_sc with sin and cos of the polar angle computed here.
template <typename T>
RAPTOR_HD int plasma_sample(const Params& p, const T x[4], const T k[4], int snap, T& ne, T& the, T& B, T& g, T& sinb) {
    T sn, cs;
    sc(x[2], &sn, &cs);
    return plasma_sample_sc<T>(p, x, k, sn, cs, snap, ne, the, B, g, sinb);
}
}  // namespace raptor
