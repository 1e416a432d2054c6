// raptor_physics.cuh -- camera, plasma models, emissivity and the backward transfer step.
#pragma once

#include "raptor_math.cuh"

namespace raptor {

// FP32 copies of the scalar parameters, converted once on the host so that the FP32 code
// paths run no double -> float conversion (B300 executes FP64 conversions slowly).
struct ParamsF {
    float a, eps, r_stop, r_esc, Lcm, tau_cut;
    float n0, n_pow, the0, the_pow, B0, B_pow, r_isco, the_min;
    float x1_min, x1_max, dx1, dx2, h_mks, t0, dt_snap, rho0_ne, B_unit, r_high, r_low, gam;
    float r_fp64, turn_kr;
    float2 r_isco_p;  // r_isco as an unevaluated float pair (hi, lo): the ISCO branch decision
    float nu[16];
    // camera parameters as unevaluated float pairs (hi, lo) for the double-float camera
    float2 a_p, sin_i_p, cos_i_p, r_cam_p, incl_p, cam_phi_p, amin_p, da_p, bmin_p, db_p;
};

// Kernel parameters (passed by value; lives in the constant bank).
struct Params {
    // spacetime / camera
    double a, r_cam, incl, sin_i, cos_i;
    double amin, da, bmin, db;
    int nx, ny, row0, n_rows;
    // integration
    double eps, r_stop, r_esc, tau_cut;
    int max_steps;
    unsigned flags;
    // units
    double Lcm;     // GM/c^2 in cm
    double pix_jy;  // dalpha dbeta L^2 / D^2 / 1e-23
    // analytic plasma
    int kind, slow;
    double n0, n_pow, the0, the_pow, B0, B_pow, r_isco;
    double the_min;  // emission only where Theta_e >= the_min (fit-validity mask; 0 = none)
    // grid plasma (MKS, r0 = 0)
    const float* grid;  // [n_snap][8][n2][n1]
    const float* x2tab; // x2 at theta_i = i pi / kX2TabN, i = 0 .. kX2TabN (FP32 inversion start)
    int n1, n2, n_snap, snap;
    double x1_min, x1_max, dx1, dx2, h_mks, t0, dt_snap;
    double rho0_ne;     // rho0 / (m_e + m_p): n_e = rho * rho0_ne
    double B_unit;      // c sqrt(4 pi rho0): B[G] = |b| * B_unit
    double r_high, r_low, gam;
    // mixed precision
    double r_fp64, turn_kr;
    // frequencies
    int nf;
    double nu[16];
    // work decomposition: ray -> (frame, pixel)
    long long n_rays;
    int n_pix;
    const double* t_frames;  // device [n_frames] camera times (t_obs + t_delay applied)
    double t_cam;            // single-image camera time
    int frame_snap0;         // fast-light light curve: snapshot of frame 0
    int lc_fast;             // 1: frame f samples snapshot frame_snap0 + f
    // outputs
    double* image;           // [frame][nf_total][n_rows][nx]
    double2* fwd;            // forward scheme: per thread, (dtau, contribution) [record][freq][thread]
    int fwd_cap;             // records per ray
    long long fwd_stride;    // threads of the launch
    double i_unscale;        // stored intensity = I * i_unscale (1 for FP64; 2^-100 for the FP32 scaling)
    int nf_total, f_off;     // frequency chunking: this launch covers [f_off, f_off + nf)
    int* steps_out;          // optional [n_rows][nx]
    int* status_out;         // optional [n_rows][nx]
    ParamsF f;               // FP32 copies (filled by the host)
    // camera position terms of the BL -> KS map at r_cam (per render, filled by the host):
    // x^0 = (t_cam + cam_logdel) + cam_tterm, x^3 = cam_phi
    double cam_logdel, cam_tterm, cam_phi;
    // learned surrogate (RAPTOR_MIXED_MLP): predicted start states [8][n_rays] (x^mu, k^mu),
    // per-ray fallback flags (start at the camera), the step count of a predicted state,
    // and the outbound exit radius beyond which the transfer is neglected (0 = off)
    const float2* start_xk;  // float pairs (hi, lo)
    const unsigned char* fallback;
    int start_n;
    double r_exit;
    float r_exit_f;
};

// Parameter in the arithmetic type T: the double field for FP64, its FP32 copy for FP32.
template <typename T>
RAPTOR_HD T pv(double d, float f);
template <>
RAPTOR_HD double pv<double>(double d, float) { return d; }
template <>
RAPTOR_HD float pv<float>(double, float f) { return f; }
#define RAPTOR_P(T, name) pv<T>(p.name, p.f.name)

// ------------------------------------------------------------------------------------
// Camera (sec. 2.3, Eqs. 24-28; App. A.1).  Always FP64.
// E = 1, L = -alpha sin i, Q = beta^2 + cos^2 i (alpha^2 - a^2) (carried by k_theta),
// k_theta = sign(beta) sqrt|Q - L^2 cot^2 theta + a^2 cos^2 theta| = beta, k_r from k.k = 0 with
// the physical photon moving outward at the camera; the state is the backward ray -k.
// ------------------------------------------------------------------------------------
// Wave vector of the camera ray through (alpha, beta) (KS components of the backward ray),
// in arithmetic type T (FP64 for the integrator; FP32 for the learned surrogate's baseline).
template <typename T>
RAPTOR_HD void camera_k_t(T a, T sn, T cs, T r, T alpha, T beta, T k[4]) {
    const T a2 = a * a;
    const T L = -alpha * sn;
    const T kt = T(-1), kp = L;
    // At theta = i, Q - L^2 cot^2 + a^2 cos^2 = beta^2 exactly, so the square root of Eq. 28
    // is |beta|: k_theta = beta.  (The printed form cancels two alpha^2 cos^2 i terms, whose
    // rounding residual its square root would magnify to ~1e-8 at beta = 0.)
    const T kh = beta;
    // Boyer-Lindquist inverse metric at the camera
    const T s2 = sn * sn;
    const T Sig = r * r + a2 * cs * cs, Del = r * r - T(2) * r + a2;
    const T A = (r * r + a2) * (r * r + a2) - a2 * Del * s2;
    const T iSD = T(1) / (Sig * Del);
    const T gtt = -A * iSD, gtp = -T(2) * a * r * iSD, grr = Del / Sig, ghh = T(1) / Sig;
    const T gpp = (Del - a2 * s2) * iSD / s2;
    const T rest = gtt * kt * kt + T(2) * gtp * kt * kp + gpp * kp * kp + ghh * kh * kh;
    const T kr = Real<T>::sqrt_(-rest / grr);
    // contravariant BL components of the backward ray
    const T ut = -(gtt * kt + gtp * kp), ur = -(grr * kr), uh = -(ghh * kh), up = -(gtp * kt + gpp * kp);
    // BL -> KS (App. A.1)
    k[0] = ut + T(2) * r / Del * ur;
    k[1] = ur;
    k[2] = uh;
    k[3] = up + a / Del * ur;
}

RAPTOR_HD void camera_k_ai(double a, double sn, double cs, double r, double alpha, double beta, double k[4]) {
    camera_k_t<double>(a, sn, cs, r, alpha, beta, k);
}

// KS position of the camera (the same for every pixel): BL (t_cam, r, incl, 0) -> KS.
RAPTOR_HD void camera_x_ai(double a, double incl, double r, double t_cam, double x[4]) {
    const double a2 = a * a;
    const double Del = r * r - 2.0 * r + a2;
    const double rp = 1.0 + sqrt(1.0 - a2), rm = 1.0 - sqrt(1.0 - a2);
    const double lg = log((r - rp) / (r - rm));
    x[0] = t_cam + log(Del) + 2.0 / (rp - rm) * lg;
    x[1] = r;
    x[2] = incl;
    x[3] = a / (rp - rm) * lg;
}

RAPTOR_HD void camera_ray_ai(double a, double sn, double cs, double incl, double r, double alpha, double beta,
                             double t_cam, double x[4], double k[4]) {
    camera_k_ai(a, sn, cs, r, alpha, beta, k);
    camera_x_ai(a, incl, r, t_cam, x);
}

// The camera position terms that depend on (a, r_cam) only, in the order camera_x_ai adds
// them: x^0 = (t_cam + log Delta) + 2 / (r+ - r-) ln((r - r+)/(r - r-)).
RAPTOR_HD void camera_x_terms(double a, double r, double* logdel, double* tterm, double* phi) {
    const double a2 = a * a;
    const double Del = r * r - 2.0 * r + a2;
    const double rp = 1.0 + sqrt(1.0 - a2), rm = 1.0 - sqrt(1.0 - a2);
    const double lg = log((r - rp) / (r - rm));
    *logdel = log(Del);
    *tterm = 2.0 / (rp - rm) * lg;
    *phi = a / (rp - rm) * lg;
}

// Camera ray of a render: the wave vector per pixel, the position from the per-render terms
// (no logarithm or square root per ray).
RAPTOR_HD void camera_ray(const Params& p, double alpha, double beta, double t_cam, double x[4], double k[4]) {
    camera_k_ai(p.a, p.sin_i, p.cos_i, p.r_cam, alpha, beta, k);
    x[0] = t_cam + p.cam_logdel + p.cam_tterm;
    x[1] = p.r_cam;
    x[2] = p.incl;
    x[3] = p.cam_phi;
}

// ------------------------------------------------------------------------------------
// Plasma sample at a KS point.
// ------------------------------------------------------------------------------------
template <typename T>
struct Sample {
    T ne, the, B;
    T u[4];
    T cosb_num;  // k.v with v = d_phi + u_phi u (toroidal field direction)
    T vnorm;     // |v|
    int ok;      // 1 emitting, 0 no plasma, -1 error (not timelike)
};

// Analytic model of the workload (not in the paper): power-law n_e, Theta_e, B; prograde
// Keplerian rotation Omega = 1/(r^{3/2} + a) at every theta for r >= r_isco; inside, free
// fall from rest at infinity (E = 1, L = 0, Q = 0), written in KS without the 1/Delta
// terms of the BL -> KS transform:
//   u^t = [P (P^2 + 2 r P + 4 r^2)/(P^2 + 2 r s) - a^2 sin^2] / Sigma,
//   u^r = -s / Sigma, u^phi = -2 a r / (Sigma (2 r + s)), P = r^2 + a^2, s = sqrt(2 r P).
template <typename T>
RAPTOR_HD int analytic_velocity(T a, T r_isco, const KSPoint<T>& P, T u[4], int kepler = -1) {
    const T r = P.r;
    u[2] = T(0);
    // kepler: the branch decided by the caller (1: r >= r_isco, 0: inside); -1: decide here.
    // The flow changes discontinuously at r_isco, so the decision is taken with the radius's
    // full precision where the caller has more than T's.
    if (kepler > 0 || (kepler < 0 && r >= r_isco)) {
        const T Om = Real<T>::rcp(r * Real<T>::sqrt_(r) + a);
        const T nrm = P.gtt + T(2) * Om * P.gtp + Om * Om * P.gpp;
        if (!(nrm < T(0))) return -1;
        const T ut = rsq(-nrm);
        u[0] = ut;
        u[1] = T(0);
        u[3] = Om * ut;
    } else {
        const T a2 = a * a;
        const T Pp = r * r + a2;
        const T s = Real<T>::sqrt_(T(2) * r * Pp);
        u[0] = (dv(Pp * (Pp * Pp + T(2) * r * Pp + T(4) * r * r), Pp * Pp + T(2) * r * s) - a2 * P.s2) * P.iSig;
        u[1] = -s * P.iSig;
        u[3] = dv(-T(2) * a * r * P.iSig, T(2) * r + s);
    }
    return 1;
}

// ------------------------------------------------------------------------------------
// Thermal synchrotron (Eqs. 41-44).  j [erg s^-1 cm^-3 Hz^-1 sr^-1], S = B_nu.
// B_nu is written as 2 nu^2 m_e Theta x / expm1(x), x = h nu / (m_e c^2 Theta), which
// equals Eq. 44 and stays inside FP32 range.
// ------------------------------------------------------------------------------------
RAPTOR_HD double bessel_k2_exact(double x) {
    // K_2(x) = int_0^inf exp(-x cosh t) cosh(2 t) dt (DLMF 10.32.9); trapezoidal rule with
    // step 1/4, whose error decays like exp(-pi^2 / h) for this entire integrand.
    const double h = 0.25;
    double sum = 0.5 * exp(-x);
    for (int n = 1; n < 400; ++n) {
        const double t = n * h;
        const double term = exp(-x * cosh(t)) * cosh(2.0 * t);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return h * sum;
}

// `jscale` multiplies j (the FP32 transfer carries emissivities scaled by 2^100 so that the
// exponential tail of Eq. 41 stays inside FP32 range; the FP64 path passes 1).  j = 0 where
// Theta_e < the_min (the fit-validity mask; j = 0 also means no absorption there).
template <typename T>
RAPTOR_HD void synchrotron(T nu, T ne, T the, T B, T sinb, bool k2_exact, T& j, T& S, T jscale = T(1),
                           T the_min = T(0)) {
    const T nu_c_per_G = T(kQe / (2.0 * kPi * kMe * kC));
    const T cj = T(1.4142135623730951 * kPi * kQe * kQe / (3.0 * kC)) * jscale;
    const T hme = T(kH / (kMe * kC * kC));
    const T x = dv(hme * nu, the);
    if constexpr (std::is_same<T, float>::value) S = T(2.0 * kMe) * nu * nu * the * x_over_expm1f(x);
    else if constexpr (std::is_same<T, double>::value) S = T(2.0 * kMe) * nu * nu * the * x_over_expm1(x);
    else S = T(2.0 * kMe) * nu * nu * the * dv(x, Real<T>::expm1_(x));
    j = T(0);
    if (the < the_min) return;  // outside the fit's validity mask: no emission
    const T nu_s = T(2.0 / 9.0) * nu_c_per_G * B * the * the * sinb;
    if (!(nu_s > T(0))) return;
    const T X = dv(nu, nu_s);
    const T X13 = Real<T>::cbrt_(X);
    if (X13 > Real<T>::exp_cut) return;
    const T X16 = Real<T>::sqrt_(X13);
    const T X12 = X13 * X16;  // X^(1/2) = X^(1/3) X^(1/6)
    const T fac = X12 + T(1.8877486253633870) * X16;  // 2^(11/12)
    T K2 = T(2) * the * the;
    if (k2_exact) K2 = T(bessel_k2_exact(1.0 / double(the)));
    j = dv(cj * ne * nu_s, K2) * fac * fac * Real<T>::exp_(-X13);
}

// Backward transfer (Eqs. 35-36, per-step solution of Eq. 34):
//   dtau = (j/S) g dl L;  I += exp(-tau) S (1 - exp(-dtau)) / g^3;  tau += dtau.
template <typename T, typename TT>
RAPTOR_HD void rt_update(T j, T S, T g, T dl_cm, T& I, TT& tau) {
    if (!(j > T(0)) || !(S > T(0))) return;
    const T dtau = j / S * g * dl_cm;
    I += Real<T>::exp_(-T(tau)) * S * (-Real<T>::expm1_(-dtau)) / (g * g * g);
    tau += TT(dtau);
}

}  // namespace raptor
