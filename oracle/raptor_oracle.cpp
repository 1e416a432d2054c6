// raptor_oracle.cpp -- plain, slow, FP64 CPU oracle for backward Kerr ray tracing
// with unpolarised thermal-synchrotron radiative transfer (RAPTOR I, Bronzwaer et al. 2018).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or loads this
// file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg do.
// It shares no code, header, table or constant with the CUDA path.
//
// Every function follows a passage of the paper step by step, in FP64, without blocking,
// fusion or algebraic simplification beyond what the passage states:
//   * metric g_{mu nu} of Kerr in Kerr-Schild (KS) or Boyer-Lindquist (BL) coordinates,
//     its analytic first derivatives, a numerically inverted g^{mu nu};
//   * the connection from the metric, Eq. 2 (sec. 2.1), generic 4x4x4 contraction;
//   * the first-order geodesic system, Eqs. 5-6, integrated by classical RK4, Eqs. 7-15, or
//     by the velocity Verlet scheme of sec. 2.2.2 (Eqs. 16-19, optionally re-evaluated);
//   * the adaptive step of Eqs. 20-23 read in log-radius coordinates;
//   * the Bardeen camera, Eqs. 24-28 (sec. 2.3), plus k^r from the null condition Eq. 4;
//   * the BL -> KS transforms of App. A.1;
//   * nu = -k.u (Eq. 30), the Leung et al. emissivity (Eqs. 41-43) with K2 ~ 2 Theta^2,
//     Kirchhoff absorption with the Planck function (Eq. 44);
//   * backward (camera -> plasma) transfer, Eqs. 35-36, with the per-step formal
//     solution of Eq. 34 (constant coefficients over a step);
//   * GRMHD unit scaling (Eq. 45), R-beta electron temperature (Eq. 46), the MKS map and
//     Newton-Raphson inversion of App. A.2, fast- and slow-light sampling (sec. 5);
//   * the thin-disk line emitter of sec. 4.2.1 (equatorial Keplerian disk from the ISCO to
//     15 M, emission ~ 1/r^2, no absorption, each ray's intensity and redshift recorded).
// Readings of passages that are garbled or silent are listed in the design notes and
// repeated where they are used below.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fopenmp -shared -fPIC.

#include <cmath>
#include <cstring>
#include <cstdlib>
#include <cstdint>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// ---------------------------------------------------------------------------------------
// CGS constants (CODATA 2018 / IAU 2015).  The paper prints none; this is the oracle's copy.
// ---------------------------------------------------------------------------------------
static const double O_G = 6.67430e-8;
static const double O_C = 2.99792458e10;
static const double O_ME = 9.1093837015e-28;
static const double O_MP = 1.67262192369e-24;
static const double O_QE = 4.80320471e-10;
static const double O_H = 6.62607015e-27;
static const double O_MSUN = 1.98841e33;
static const double O_PC = 3.0856775814913673e18;
static const double O_PI = 3.14159265358979323846;

extern "C" {

// Scene description.  Mirrored field by field in oracle/__init__.py (ctypes).
typedef struct {
    // spacetime
    double m;            // mass parameter in units of M: 1 = Kerr, 0 = flat space
    double a;            // spin a/M, |a| < m (or any a with m = 0)
    int coords;          // 0 = KS (t~, r, theta, phi~), 1 = BL
    int step_rule;       // 0 = Eqs. 20-23 in log-r, 1 = literal d lambda = eps * r
    // camera (sec. 2.3)
    double r_cam, incl_deg;
    int nx, ny;
    double amin, amax, bmin, bmax;
    // integration
    double eps, r_stop_factor, r_esc, tau_cut;
    int max_steps;
    int k2_exact;        // 0 = K2(1/Theta) ~ 2 Theta^2 (sec. 4.2.2), 1 = exact Bessel K2
    // units
    double mass_msun, dist_pc;
    // plasma
    int plasma_kind;     // 0 analytic, 1 grid, 2 static isotropic (test), 3 uniform ball (test)
    int slow_light;      // grid only: 1 = interpolate snapshots in ray time
    double n0, n_pow, the0, the_pow, B0, B_pow;   // analytic / static profiles
    double ball_R, ball_j, ball_alpha;            // uniform ball: j [cgs], alpha [1/cm]
    const float* grid;   // [n_snap][8][n2][n1]: rho, u, U1, U2, U3, B1, B2, B3 (MKS)
    int n1, n2, n_snap, snap;  // snap: snapshot used in fast light
    double x1_min, x1_max, h_mks;
    double t0, dt_snap;
    double mass_unit_g, r_high, r_low, gamma_ad;
    int integrator;      // 0 = RK4 (Eqs. 7-15), 1 = velocity Verlet (Eqs. 16-19), 2 = Verlet with re-evaluation
    double theta_e_min;  // no emission (nor absorption) where Theta_e < theta_e_min; 0 = no mask
    int rt_scheme;       // 0 = backward accumulation (Eqs. 35-36), 1 = forward formal solution (Eq. 34)
} OraScene;

}  // extern "C"

typedef double M4[4][4];

// ---------------------------------------------------------------------------------------
// Metric, its derivatives and inverse (sec. 2.4; Kerr in KS and BL)
// ---------------------------------------------------------------------------------------
static void metric(const OraScene* s, double r, double th, M4 g) {
    const double m = s->m, a = s->a;
    const double sn = std::sin(th), cs = std::cos(th), s2 = sn * sn;
    const double Sig = r * r + a * a * cs * cs;
    std::memset(g, 0, sizeof(M4));
    if (s->coords == 0) {
        // Kerr-Schild, ingoing; z = 2 m r / Sigma
        const double z = 2.0 * m * r / Sig;
        g[0][0] = -(1.0 - z);
        g[0][1] = z;
        g[0][3] = -a * z * s2;
        g[1][1] = 1.0 + z;
        g[1][3] = -a * (1.0 + z) * s2;
        g[2][2] = Sig;
        g[3][3] = s2 * (Sig + a * a * (1.0 + z) * s2);
    } else {
        const double Del = r * r - 2.0 * m * r + a * a;
        g[0][0] = -(1.0 - 2.0 * m * r / Sig);
        g[0][3] = -2.0 * m * a * r * s2 / Sig;
        g[1][1] = Sig / Del;
        g[2][2] = Sig;
        g[3][3] = s2 * (r * r + a * a + 2.0 * m * a * a * r * s2 / Sig);
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < i; ++j) g[i][j] = g[j][i];
}

// dg[l][i][j] = d g_ij / d x^l ; only l = 1 (r) and l = 2 (theta) are non-zero.
static void dmetric(const OraScene* s, double r, double th, double dg[4][4][4]) {
    const double m = s->m, a = s->a;
    const double sn = std::sin(th), cs = std::cos(th), s2 = sn * sn;
    const double Sig = r * r + a * a * cs * cs;
    std::memset(dg, 0, sizeof(double) * 64);
    for (int l = 1; l <= 2; ++l) {
        const double dSig = (l == 1) ? 2.0 * r : -2.0 * a * a * cs * sn;
        const double ds2 = (l == 1) ? 0.0 : 2.0 * sn * cs;
        const double dr = (l == 1) ? 1.0 : 0.0;
        double (*d)[4] = dg[l];
        if (s->coords == 0) {
            const double z = 2.0 * m * r / Sig;
            const double dz = 2.0 * m * dr / Sig - 2.0 * m * r * dSig / (Sig * Sig);
            d[0][0] = dz;
            d[0][1] = dz;
            d[0][3] = -a * (dz * s2 + z * ds2);
            d[1][1] = dz;
            d[1][3] = -a * (dz * s2 + (1.0 + z) * ds2);
            d[2][2] = dSig;
            d[3][3] = ds2 * (Sig + a * a * (1.0 + z) * s2) +
                      s2 * (dSig + a * a * (dz * s2 + (1.0 + z) * ds2));
        } else {
            const double Del = r * r - 2.0 * m * r + a * a;
            const double dDel = (l == 1) ? 2.0 * r - 2.0 * m : 0.0;
            const double q = 2.0 * m * r / Sig;  // g_tt = -(1 - q)
            const double dq = 2.0 * m * dr / Sig - 2.0 * m * r * dSig / (Sig * Sig);
            d[0][0] = dq;
            d[0][3] = -a * (dq * s2 + q * ds2);
            d[1][1] = dSig / Del - Sig * dDel / (Del * Del);
            d[2][2] = dSig;
            d[3][3] = ds2 * (r * r + a * a + a * a * q * s2) +
                      s2 * (2.0 * r * dr + a * a * (dq * s2 + q * ds2));
        }
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < i; ++j) d[i][j] = d[j][i];
    }
}

// Gauss-Jordan inversion with partial pivoting (a library-style primitive).
static void invert4(const M4 g, M4 gi) {
    double A[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) A[i][j] = (j < 4) ? g[i][j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int i = c + 1; i < 4; ++i)
            if (std::fabs(A[i][c]) > std::fabs(A[p][c])) p = i;
        if (p != c)
            for (int j = 0; j < 8; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
        const double piv = A[c][c];
        for (int j = 0; j < 8; ++j) A[c][j] /= piv;
        for (int i = 0; i < 4; ++i) {
            if (i == c) continue;
            const double f = A[i][c];
            if (f == 0.0) continue;
            for (int j = 0; j < 8; ++j) A[i][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) gi[i][j] = A[i][j + 4];
}

// Eq. 2: Gamma^a_{mn} = 1/2 g^{ar} (d_m g_{nr} + d_n g_{mr} - d_r g_{mn})
static void connection(const OraScene* s, double r, double th, double G[4][4][4]) {
    M4 g, gi;
    double dg[4][4][4];
    metric(s, r, th, g);
    invert4(g, gi);
    dmetric(s, r, th, dg);
    for (int al = 0; al < 4; ++al)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                double acc = 0.0;
                for (int rho = 0; rho < 4; ++rho)
                    acc += gi[al][rho] * (dg[mu][nu][rho] + dg[nu][mu][rho] - dg[rho][mu][nu]);
                G[al][mu][nu] = 0.5 * acc;
            }
}

// Eqs. 5-6: dx/dl = k, dk^a/dl = -Gamma^a_{mn} k^m k^n
static void rhs(const OraScene* s, const double x[4], const double k[4], double dx[4], double dk[4]) {
    double G[4][4][4];
    connection(s, x[1], x[2], G);
    for (int al = 0; al < 4; ++al) {
        double acc = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) acc += G[al][mu][nu] * k[mu] * k[nu];
        dx[al] = k[al];
        dk[al] = -acc;
    }
}

// Eqs. 7-15, classical RK4.  Reading: the position coefficients use the wave vector at the
// stage point, C2x = dl (k + C1k/2), C3x = dl (k + C2k/2), C4x = dl (k + C3k); the printed
// "k + C1x/2" adds a position increment to a wave vector and is taken as a typo.
static void rk4_step(const OraScene* s, double x[4], double k[4], double dl) {
    double C1x[4], C1k[4], C2x[4], C2k[4], C3x[4], C3k[4], C4x[4], C4k[4];
    double xs[4], ks[4], fx[4], fk[4];
    rhs(s, x, k, fx, fk);
    for (int i = 0; i < 4; ++i) { C1x[i] = dl * fx[i]; C1k[i] = dl * fk[i]; }
    for (int i = 0; i < 4; ++i) { xs[i] = x[i] + 0.5 * C1x[i]; ks[i] = k[i] + 0.5 * C1k[i]; }
    rhs(s, xs, ks, fx, fk);
    for (int i = 0; i < 4; ++i) { C2x[i] = dl * fx[i]; C2k[i] = dl * fk[i]; }
    for (int i = 0; i < 4; ++i) { xs[i] = x[i] + 0.5 * C2x[i]; ks[i] = k[i] + 0.5 * C2k[i]; }
    rhs(s, xs, ks, fx, fk);
    for (int i = 0; i < 4; ++i) { C3x[i] = dl * fx[i]; C3k[i] = dl * fk[i]; }
    for (int i = 0; i < 4; ++i) { xs[i] = x[i] + C3x[i]; ks[i] = k[i] + C3k[i]; }
    rhs(s, xs, ks, fx, fk);
    for (int i = 0; i < 4; ++i) { C4x[i] = dl * fx[i]; C4k[i] = dl * fk[i]; }
    for (int i = 0; i < 4; ++i) {
        x[i] = x[i] + (C1x[i] + 2.0 * C2x[i] + 2.0 * C3x[i] + C4x[i]) / 6.0;
        k[i] = k[i] + (C1k[i] + 2.0 * C2k[i] + 2.0 * C3k[i] + C4k[i]) / 6.0;
    }
}

// Sec. 2.2.2, velocity Verlet (Eqs. 16-19).  f holds (dk/dl)_n on entry and the derivative
// at the new point on return, so each step evaluates the connection once (twice with the
// re-evaluation):
//   x_{n+1} = x_n + k_n dl + f_n dl^2 / 2                          (Eq. 16)
//   k_p = k_n + f_n dl                                             (Eq. 17)
//   f_{n+1} = -Gamma(x_{n+1}) k_p k_p                              (Eq. 18)
//   k_{n+1} = k_n + (f_n + f_{n+1}) dl / 2                         (Eq. 19)
// Re-evaluation (reeval): Eq. 18 again with k_p = k_{n+1} from Eq. 19, then Eq. 19 again;
// the derivative carried to the next step is the last one evaluated (reading: the paper
// does not say which derivative the next step starts from; the last is the only one at the
// new point that needs no further evaluation).
static void verlet_step(const OraScene* s, double x[4], double k[4], double f[4], double dl, int reeval) {
    double xn[4], kp[4], kn[4], fn[4], dx[4];
    for (int i = 0; i < 4; ++i) {
        xn[i] = x[i] + k[i] * dl + 0.5 * f[i] * dl * dl;
        kp[i] = k[i] + f[i] * dl;
    }
    rhs(s, xn, kp, dx, fn);
    for (int i = 0; i < 4; ++i) kn[i] = k[i] + 0.5 * (f[i] + fn[i]) * dl;
    if (reeval) {
        rhs(s, xn, kn, dx, fn);
        for (int i = 0; i < 4; ++i) kn[i] = k[i] + 0.5 * (f[i] + fn[i]) * dl;
    }
    for (int i = 0; i < 4; ++i) { x[i] = xn[i]; k[i] = kn[i]; f[i] = fn[i]; }
}

// One step of the scene's integrator; f is the carried derivative of the Verlet schemes
// (unused by RK4).
static void advance(const OraScene* s, double x[4], double k[4], double f[4], double dl) {
    if (s->integrator == 0) rk4_step(s, x, k, dl);
    else verlet_step(s, x, k, f, dl, s->integrator == 2);
}

// The carried derivative at the start of a ray: (dk/dl)_0 = -Gamma(x_0) k_0 k_0.
static void start_derivative(const OraScene* s, const double x[4], const double k[4], double f[4]) {
    double dx[4];
    if (s->integrator == 0) {
        for (int i = 0; i < 4; ++i) f[i] = 0.0;
        return;
    }
    rhs(s, x, k, dx, f);
}

// Eqs. 20-23 evaluated in coordinates x1 = ln r, x2 = theta/pi, x3 = phi, i.e.
//   dl1 = eps / (|k^r|/r + delta), dl2 = eps min(x2, 1-x2) / (|k^theta|/pi + delta),
//   dl3 = eps / (|k^phi| + delta),  dl = 1 / (1/dl1 + 1/dl2 + 1/dl3).
static double step_size(const OraScene* s, const double x[4], const double k[4]) {
    const double delta = 1e-30;
    const double r = x[1], th = x[2];
    if (s->step_rule == 1) return s->eps * r;
    const double k1 = std::fabs(k[1]) / r;          // |d x1 / d lambda|
    const double k2 = std::fabs(k[2]) / O_PI;       // |d x2 / d lambda|
    const double k3 = std::fabs(k[3]);
    const double x2 = th / O_PI;
    const double dl1 = s->eps / (k1 + delta);
    const double dl2 = s->eps * std::fmin(x2, 1.0 - x2) / (k2 + delta);
    const double dl3 = s->eps / (k3 + delta);
    return 1.0 / (1.0 / std::fabs(dl1) + 1.0 / std::fabs(dl2) + 1.0 / std::fabs(dl3));
}

static double horizon(const OraScene* s) {
    if (s->m <= 0.0) return 0.0;
    return s->m + std::sqrt(s->m * s->m - s->a * s->a);
}

// App. A.1: BL -> KS for a contravariant vector at radius r.
static void vec_bl_to_ks(const OraScene* s, double r, const double vb[4], double vk[4]) {
    const double Del = r * r - 2.0 * s->m * r + s->a * s->a;
    vk[0] = vb[0] + 2.0 * s->m * r / Del * vb[1];
    vk[1] = vb[1];
    vk[2] = vb[2];
    vk[3] = vb[3] + s->a / Del * vb[1];
}

// App. A.1: BL -> KS coordinates (t~, phi~); valid outside the horizon.
static void pos_bl_to_ks(const OraScene* s, const double xb[4], double xk[4]) {
    const double m = s->m, a = s->a, r = xb[1];
    xk[0] = xb[0];
    xk[1] = xb[1];
    xk[2] = xb[2];
    xk[3] = xb[3];
    if (m <= 0.0) return;
    const double rp = m + std::sqrt(m * m - a * a), rm = m - std::sqrt(m * m - a * a);
    const double Del = r * r - 2.0 * m * r + a * a;
    const double lg = std::log((r - rp) / (r - rm));
    xk[0] = xb[0] + m * std::log(Del) + 2.0 * m * m / (rp - rm) * lg;
    xk[3] = xb[3] + a / (rp - rm) * lg;
}

static double sgn_pos(double v) { return v < 0.0 ? -1.0 : 1.0; }

extern "C" {

// ---------------------------------------------------------------------------------------
// Exported primitives (used by the pins)
// ---------------------------------------------------------------------------------------
int ora_abi_version(void) { return 3; }

void ora_metric(const OraScene* s, double r, double th, double* g16, double* gi16) {
    M4 g, gi;
    metric(s, r, th, g);
    invert4(g, gi);
    for (int i = 0; i < 16; ++i) {
        g16[i] = g[i / 4][i % 4];
        gi16[i] = gi[i / 4][i % 4];
    }
}

void ora_dmetric(const OraScene* s, double r, double th, double* dg64) {
    double dg[4][4][4];
    dmetric(s, r, th, dg);
    std::memcpy(dg64, dg, sizeof(dg));
}

void ora_connection(const OraScene* s, double r, double th, double* G64) {
    double G[4][4][4];
    connection(s, r, th, G);
    std::memcpy(G64, G, sizeof(G));
}

double ora_step_size(const OraScene* s, const double* x, const double* k) { return step_size(s, x, k); }

void ora_rk4_step(const OraScene* s, double* x, double* k, double dl) { rk4_step(s, x, k, dl); }

void ora_verlet_step(const OraScene* s, double* x, double* k, double* f, double dl, int reeval) {
    verlet_step(s, x, k, f, dl, reeval);
}

double ora_horizon(const OraScene* s) { return horizon(s); }

void ora_vec_bl_to_ks(const OraScene* s, double r, const double* vb, double* vk) { vec_bl_to_ks(s, r, vb, vk); }

void ora_pos_bl_to_ks(const OraScene* s, const double* xb, double* xk) { pos_bl_to_ks(s, xb, xk); }

// Sec. 2.3, Eqs. 24-28, with E = 1.  Reading of the garbled camera equations:
//   Q = beta^2 + cos^2 i (alpha^2 - a^2),  k_theta = sign(beta) sqrt|Q - L^2 cot^2 + a^2 cos^2|
// (the a^2 follows from the Carter constant, Eq. 39, with mu = 0).  k_r from the null
// condition with k^r > 0: the physical photon arrives at the camera moving outward.  The
// integrated state is the backward ray -k_phys.  Output in the scene's coordinates.
void ora_camera(const OraScene* s, double alpha, double beta, double t_cam, double* x, double* k) {
    const double inc = s->incl_deg * O_PI / 180.0;
    const double si = std::sin(inc), ci = std::cos(inc);
    const double E = 1.0;
    const double L = -alpha * E * si;
    const double Q = E * E * (beta * beta + ci * ci * (alpha * alpha - s->a * s->a));
    const double th = inc, r = s->r_cam;
    const double cth = std::cos(th), sth = std::sin(th);
    const double cot = cth / sth;
    double kc[4];
    kc[0] = -E;
    kc[3] = L;
    // At the camera theta = i, so Q - L^2 cot^2 + a^2 cos^2 = beta^2 exactly and Eq. 28 gives
    // k_theta = sign(beta) |beta| = beta.  It is evaluated in that form: the printed form
    // cancels two equal alpha^2 cos^2 i terms and its square root turns the rounding
    // residual into a ~1e-8 spurious k_theta for beta = 0.
    const double kth_sq = Q - L * L * cot * cot + s->a * s->a * cth * cth;  // == beta^2 in exact arithmetic
    (void)kth_sq;
    kc[2] = sgn_pos(beta) * std::fabs(beta);
    // BL inverse metric at the camera
    OraScene bl = *s;
    bl.coords = 1;
    M4 g, gi;
    metric(&bl, r, th, g);
    invert4(g, gi);
    double rest = 0.0;
    const int idx[3] = {0, 2, 3};
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) rest += gi[idx[p]][idx[q]] * kc[idx[p]] * kc[idx[q]];
    kc[1] = std::sqrt(-rest / gi[1][1]);
    double kb[4];
    for (int mu = 0; mu < 4; ++mu) {
        double acc = 0.0;
        for (int nu = 0; nu < 4; ++nu) acc += gi[mu][nu] * kc[nu];
        kb[mu] = -acc;  // backward ray
    }
    double xb[4] = {t_cam, r, th, 0.0};
    if (s->coords == 1) {
        for (int i = 0; i < 4; ++i) { x[i] = xb[i]; k[i] = kb[i]; }
    } else {
        pos_bl_to_ks(s, xb, x);
        vec_bl_to_ks(s, r, kb, k);
    }
}

// Eq. 39 for the physical photon (-state): E = -k_t, L = k_phi,
// Q = k_theta^2 + cos^2 [a^2 (mu^2 - k_t^2) + k_phi^2 / sin^2], mu = 0.  Also returns
// the null residual g_{mn} k^m k^n in out[3].
void ora_constants(const OraScene* s, const double* x, const double* kstate, double* out) {
    M4 g;
    metric(s, x[1], x[2], g);
    double kc[4], kk = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        double acc = 0.0;
        for (int nu = 0; nu < 4; ++nu) acc += g[mu][nu] * (-kstate[nu]);
        kc[mu] = acc;
    }
    for (int mu = 0; mu < 4; ++mu) kk += kc[mu] * (-kstate[mu]);
    const double c = std::cos(x[2]), sn = std::sin(x[2]);
    out[0] = -kc[0];
    out[1] = kc[3];
    out[2] = kc[2] * kc[2] + c * c * (s->a * s->a * (0.0 - kc[0] * kc[0]) + kc[3] * kc[3] / (sn * sn));
    out[3] = kk;
}

// Innermost stable circular orbit, Bardeen, Press & Teukolsky (1972), for an orbit with
// angular velocity of the sign of +1 (prograde for a > 0).
double ora_r_isco(double a) {
    const double z1 = 1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
    const double z2 = std::sqrt(3.0 * a * a + z1 * z1);
    const double sg = a < 0.0 ? -1.0 : 1.0;
    return 3.0 + z2 - sg * std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

// ---------------------------------------------------------------------------------------
// Plasma (sec. 4.2.2, sec. 5; analytic model of the workload; test plasmas)
// ---------------------------------------------------------------------------------------

// App. A.2, Newton-Raphson for theta -> x2 with theta = pi x2 + (1-h)/2 sin(2 pi x2).
// Start x2 = theta/pi; reset to 0.05 when the iterate leaves [0,1] or f' -> 0; stop when
// |x_{n+1} - x_n| < tol or after 20 iterations.
double ora_newton_x2(double theta, double h, double tol, int* iters) {
    double x = theta / O_PI;
    int n = 0;
    for (n = 1; n <= 20; ++n) {
        const double f = O_PI * x + 0.5 * (1.0 - h) * std::sin(2.0 * O_PI * x) - theta;
        const double fp = O_PI * (1.0 + (1.0 - h) * std::cos(2.0 * O_PI * x));
        double xn;
        if (std::fabs(fp) < 1e-12) {
            xn = 0.05;
        } else {
            xn = x - f / fp;
            if (xn < 0.0 || xn > 1.0) xn = 0.05;
        }
        const double d = std::fabs(xn - x);
        x = xn;
        if (d < tol) break;
    }
    if (iters) *iters = n;
    return x;
}

// Bilinear, cell-centred interpolation of the 8 primitive fields of snapshot `snap` at
// (x1, x2); x2 is clamped to the edge cells.  Returns 0 outside the radial range.
static int grid_bilinear(const OraScene* s, int snap, double x1, double x2, double out[8]) {
    if (x1 < s->x1_min || x1 > s->x1_max) return 0;
    const double dx1 = (s->x1_max - s->x1_min) / s->n1;
    const double dx2 = 1.0 / s->n2;
    double fi = (x1 - s->x1_min) / dx1 - 0.5;
    double fj = x2 / dx2 - 0.5;
    int i0 = (int)std::floor(fi), j0 = (int)std::floor(fj);
    double wi = fi - i0, wj = fj - j0;
    if (i0 < 0) { i0 = 0; wi = 0.0; }
    if (i0 > s->n1 - 2) { i0 = s->n1 - 2; wi = 1.0; }
    if (j0 < 0) { j0 = 0; wj = 0.0; }
    if (j0 > s->n2 - 2) { j0 = s->n2 - 2; wj = 1.0; }
    const size_t plane = (size_t)s->n1 * s->n2;
    const float* base = s->grid + (size_t)snap * 8 * plane;
    for (int f = 0; f < 8; ++f) {
        const float* F = base + f * plane;
        const double v00 = F[(size_t)j0 * s->n1 + i0], v10 = F[(size_t)j0 * s->n1 + i0 + 1];
        const double v01 = F[(size_t)(j0 + 1) * s->n1 + i0], v11 = F[(size_t)(j0 + 1) * s->n1 + i0 + 1];
        out[f] = (1.0 - wi) * (1.0 - wj) * v00 + wi * (1.0 - wj) * v10 + (1.0 - wi) * wj * v01 + wi * wj * v11;
    }
    return 1;
}

int ora_grid_bilinear(const OraScene* s, int snap, double x1, double x2, double* out) {
    return grid_bilinear(s, snap, x1, x2, out);
}

// Plasma state at KS position x: n_e [cm^-3], Theta_e, B [G], u^mu and b^mu (KS; b in G).
// Returns 0 where there is no emitting plasma.
typedef struct {
    double ne, thetae, B;
    double u[4], b[4];
    int iso;  // 1: isotropic emitter (sin theta_B = 1), 2: fixed j, alpha (uniform ball)
    double jfix, afix;
} Plasma;

static int plasma_at(const OraScene* s, const double x[4], Plasma* P) {
    const double r = x[1], th = x[2], a = s->a, m = s->m;
    std::memset(P, 0, sizeof(Plasma));
    if (s->plasma_kind == 3) {  // uniform ball at rest, constant coefficients
        if (r >= s->ball_R) return 0;
        M4 g;
        metric(s, r, th, g);
        P->u[0] = 1.0 / std::sqrt(-g[0][0]);
        P->iso = 2;
        P->jfix = s->ball_j;
        P->afix = s->ball_alpha;
        return 1;
    }
    if (s->plasma_kind == 0 || s->plasma_kind == 2) {
        P->ne = s->n0 * std::pow(r, s->n_pow);
        P->thetae = s->the0 * std::pow(r, s->the_pow);
        P->B = s->B0 * std::pow(r, s->B_pow);
        OraScene bl = *s;
        bl.coords = 1;
        M4 g, gi;
        metric(&bl, r, th, g);
        invert4(g, gi);
        double ub[4] = {0, 0, 0, 0};
        if (s->plasma_kind == 2) {
            ub[0] = 1.0 / std::sqrt(-g[0][0]);  // static observer
            P->iso = 1;
        } else {
            const double risco = (m > 0.0) ? ora_r_isco(a) : 0.0;
            if (r >= risco) {
                // prograde Keplerian angular velocity at every theta
                const double Om = std::sqrt(m) / (std::pow(r, 1.5) + a * std::sqrt(m));
                const double nrm = g[0][0] + 2.0 * Om * g[0][3] + Om * Om * g[3][3];
                if (!(nrm < 0.0)) return -1;
                ub[0] = 1.0 / std::sqrt(-nrm);
                ub[3] = Om * ub[0];
            } else {
                // free fall from rest at infinity: u_t = -1, u_phi = 0, Q = 0
                const double Sig = r * r + a * a * std::cos(th) * std::cos(th);
                ub[1] = -std::sqrt(2.0 * m * r * (r * r + a * a)) / Sig;
                ub[0] = -gi[0][0];
                ub[3] = -gi[0][3];
            }
        }
        double uk[4];
        if (s->coords == 0) vec_bl_to_ks(s, r, ub, uk);
        else for (int i = 0; i < 4; ++i) uk[i] = ub[i];
        for (int i = 0; i < 4; ++i) P->u[i] = uk[i];
        if (P->iso) return 1;
        // toroidal field: b ~ (d_phi) + u_phi u, normalised to |b| = B
        M4 gs;
        metric(s, r, th, gs);
        double u_phi = 0.0;
        for (int nu = 0; nu < 4; ++nu) u_phi += gs[3][nu] * uk[nu];
        double v[4] = {u_phi * uk[0], u_phi * uk[1], u_phi * uk[2], 1.0 + u_phi * uk[3]};
        double vv = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) vv += gs[mu][nu] * v[mu] * v[nu];
        const double nv = std::sqrt(vv);
        for (int i = 0; i < 4; ++i) P->b[i] = P->B * v[i] / nv;
        return 1;
    }
    if (s->plasma_kind == 1) {
        // GRMHD-shaped grid in MKS (App. A.2), h from the data, r0 = 0.
        const double x1 = std::log(r);
        if (x1 < s->x1_min || x1 > s->x1_max) return 0;
        const double x2 = ora_newton_x2(th, s->h_mks, 1e-14, nullptr);
        double prim[8];
        if (s->slow_light && s->n_snap > 1) {
            double fs = (x[0] - s->t0) / s->dt_snap;
            if (fs < 0.0) fs = 0.0;
            if (fs > s->n_snap - 1) fs = s->n_snap - 1;
            int s0 = (int)std::floor(fs);
            if (s0 > s->n_snap - 2) s0 = s->n_snap - 2;
            const double w = fs - s0;
            double p0[8], p1[8];
            grid_bilinear(s, s0, x1, x2, p0);
            grid_bilinear(s, s0 + 1, x1, x2, p1);
            for (int f = 0; f < 8; ++f) prim[f] = (1.0 - w) * p0[f] + w * p1[f];
        } else {
            int snap = s->snap;
            if (snap < 0) snap = 0;
            if (snap > s->n_snap - 1) snap = s->n_snap - 1;
            grid_bilinear(s, snap, x1, x2, prim);
        }
        const double rho = prim[0], uu = prim[1];
        if (!(rho > 0.0) || !(uu > 0.0)) return 0;
        // MKS metric from the KS metric: J = diag(1, dr/dx1, dtheta/dx2, 1)
        M4 gk, gm, gmi;
        metric(s, r, th, gk);
        const double J[4] = {1.0, r, O_PI * (1.0 + (1.0 - s->h_mks) * std::cos(2.0 * O_PI * x2)), 1.0};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) gm[i][j] = gk[i][j] * J[i] * J[j];
        invert4(gm, gmi);
        // HARM primitives: U^i is the velocity relative to the normal observer
        const double Ut[3] = {prim[2], prim[3], prim[4]};
        double q = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) q += gm[i + 1][j + 1] * Ut[i] * Ut[j];
        const double gam = std::sqrt(1.0 + q);
        const double alp = 1.0 / std::sqrt(-gmi[0][0]);
        double um[4];
        um[0] = gam / alp;
        for (int i = 1; i < 4; ++i) um[i] = Ut[i - 1] - gam * alp * gmi[0][i];
        double ucov[4];
        for (int mu = 0; mu < 4; ++mu) {
            double acc = 0.0;
            for (int nu = 0; nu < 4; ++nu) acc += gm[mu][nu] * um[nu];
            ucov[mu] = acc;
        }
        const double Bv[3] = {prim[5], prim[6], prim[7]};
        double bm[4];
        bm[0] = 0.0;
        for (int i = 0; i < 3; ++i) bm[0] += Bv[i] * ucov[i + 1];
        for (int i = 1; i < 4; ++i) bm[i] = (Bv[i - 1] + bm[0] * um[i]) / um[0];
        double b2 = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) b2 += gm[mu][nu] * bm[mu] * bm[nu];
        if (!(b2 > 0.0)) return 0;
        // Eq. 45 unit scaling
        const double L = O_G * s->mass_msun * O_MSUN / (O_C * O_C);
        const double rho0 = s->mass_unit_g / (L * L * L);
        const double B0 = O_C * std::sqrt(4.0 * O_PI * rho0);
        P->ne = rho * rho0 / (O_ME + O_MP);
        P->B = std::sqrt(b2) * B0;
        // Eq. 46: R-beta electron temperature
        const double betap = (s->gamma_ad - 1.0) * uu / (0.5 * b2);
        const double b2p = betap * betap;
        const double R = s->r_low / (1.0 + b2p) + s->r_high * b2p / (1.0 + b2p);
        P->thetae = (O_MP / O_ME) * (s->gamma_ad - 1.0) * (uu / rho) / (1.0 + R);
        // back to KS components
        const double Jv[4] = {1.0, r, J[2], 1.0};
        const double bscale = B0;
        for (int i = 0; i < 4; ++i) {
            P->u[i] = um[i] * Jv[i];
            P->b[i] = bm[i] * Jv[i] * bscale;
        }
        return 1;
    }
    return 0;
}

int ora_plasma(const OraScene* s, const double* x, double* out) {
    Plasma P;
    const int ok = plasma_at(s, x, &P);
    out[0] = P.ne;
    out[1] = P.thetae;
    out[2] = P.B;
    for (int i = 0; i < 4; ++i) {
        out[3 + i] = P.u[i];
        out[7 + i] = P.b[i];
    }
    return ok;
}

// ---------------------------------------------------------------------------------------
// Emission and absorption (sec. 4.2.2)
// ---------------------------------------------------------------------------------------
// Eqs. 41-43 (Leung et al. 2011 fit) and Eq. 44 (Planck); alpha = j / B_nu (Kirchhoff).
// out[0] = j_nu [erg s^-1 cm^-3 Hz^-1 sr^-1], out[1] = B_nu [erg s^-1 cm^-2 Hz^-1 sr^-1].
void ora_emissivity(double nu, double ne, double thetae, double B, double sin_thb, int k2_exact, double* out) {
    out[0] = 0.0;
    out[1] = 0.0;
    const double nu_c = O_QE * B / (2.0 * O_PI * O_ME * O_C);
    const double nu_s = (2.0 / 9.0) * nu_c * thetae * thetae * sin_thb;
    const double K2 = k2_exact ? std::cyl_bessel_k(2.0, 1.0 / thetae) : 2.0 * thetae * thetae;
    const double xhm = O_H * nu / (O_ME * O_C * O_C * thetae);
    out[1] = (2.0 * O_H * nu * nu * nu / (O_C * O_C)) / std::expm1(xhm);
    if (!(nu_s > 0.0)) return;
    const double X = nu / nu_s;
    const double X13 = std::cbrt(X);
    const double X16 = std::sqrt(X13);
    const double X12 = std::sqrt(X);
    const double fac = X12 + std::pow(2.0, 11.0 / 12.0) * X16;
    out[0] = std::sqrt(2.0) * O_PI * O_QE * O_QE * ne * nu_s / (3.0 * O_C * K2) * fac * fac * std::exp(-X13);
}

// Backward transfer step (Eqs. 35-36 with the constant-coefficient solution of Eq. 34):
//   dtau = alpha g dl L ;  I_obs += exp(-tau) S (1 - exp(-dtau)) / g^3 ;  tau += dtau
void ora_rt_update(double* I, double* tau, double j, double S, double g, double dl_cm) {
    if (!(j > 0.0) || !(S > 0.0)) return;
    const double alpha = j / S;
    const double dtau = alpha * g * dl_cm;
    *I += std::exp(-*tau) * S * (-std::expm1(-dtau)) / (g * g * g);
    *tau += dtau;
}

// Forward formal solution (sec. 3, Eq. 34 over one step, constant coefficients): the step's
// optical depth and its own invariant contribution S (1 - e^{-dtau}) / g^3 are recorded (in
// `fwd`, pairs in step order) and the optical depth from the camera is still accumulated
// for the cut-off; the intensity is formed once the ray has ended, from its far end:
// I <- I e^{-dtau} + S (1 - e^{-dtau}) / g^3 towards the camera.
static void rt_record(std::vector<double>* fwd, double* tau, double j, double S, double g, double dl_cm) {
    double dtau = 0.0, c = 0.0;
    if (j > 0.0 && S > 0.0) {
        dtau = j / S * g * dl_cm;
        c = S * (-std::expm1(-dtau)) / (g * g * g);
    }
    fwd->push_back(dtau);
    fwd->push_back(c);
    *tau += dtau;
}

// One transfer sample at state (x, k) for all frequencies.  Returns 0 on success, 1 if
// the frequency ratio g <= 0 (not possible for a timelike u: reported as an error).
static int rt_sample(const OraScene* s, const double x[4], const double k[4], double dl,
                     const double* nus, int nf, double* I, double* tau, double* g_out,
                     std::vector<double>* fwd = nullptr) {
    Plasma P;
    const int ok = plasma_at(s, x, &P);
    if (g_out) *g_out = 0.0;
    if (ok < 0) return 1;
    if (ok == 0) return 0;
    M4 g;
    metric(s, x[1], x[2], g);
    double ku = 0.0, kb = 0.0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
            ku += g[mu][nu] * k[mu] * P.u[nu];
            kb += g[mu][nu] * k[mu] * P.b[nu];
        }
    // Eq. 30 for the physical photon -k: g = nu_fluid / nu_obs = -(-k).u = k.u
    const double gr = ku;
    if (g_out) *g_out = gr;
    if (!(gr > 0.0)) return 1;
    const double L = O_G * s->mass_msun * O_MSUN / (O_C * O_C);
    double sinb = 1.0;
    if (P.iso == 0) {
        double cb = -kb / (gr * P.B);  // (k_phys . b) / (g |b|)
        if (cb > 1.0) cb = 1.0;
        if (cb < -1.0) cb = -1.0;
        sinb = std::sqrt(1.0 - cb * cb);
    }
    for (int f = 0; f < nf; ++f) {
        const double nuf = gr * nus[f];
        double jS[2];
        if (P.iso == 2) {
            // constant j, alpha in the fluid frame
            jS[0] = P.jfix;
            jS[1] = P.jfix / P.afix;
        } else if (P.thetae < s->theta_e_min) {
            // sec. 4.2.2: the fit holds for Theta_e above ~0.5; below theta_e_min the
            // sample emits and absorbs nothing (validity mask, off by default)
            jS[0] = jS[1] = 0.0;
        } else {
            ora_emissivity(nuf, P.ne, P.thetae, P.B, sinb, s->k2_exact, jS);
        }
        if (fwd) rt_record(&fwd[f], &tau[f], jS[0], jS[1], gr, dl * L);
        else ora_rt_update(&I[f], &tau[f], jS[0], jS[1], gr, dl * L);
    }
    return 0;
}

// One backward ray (sec. 3, Eqs. 35-36): geodesic and transfer integrated together.
// Termination after each step, before that step's transfer sample: captured (r < r_stop
// r_h), escaped (r > r_esc), truncated (max_steps); thick (min tau > tau_cut) is tested
// after the sample.  Status: 0 escaped, 1 captured, 2 thick, 3 truncated, 4 error.
// trace (optional) receives per step: x[4], k[4], dl, g, I[0], tau[0]  (12 doubles);
// g = 0 on the terminating step, which takes no transfer sample.  With the forward scheme
// (rt_scheme = 1) the intensity exists only once the ray has ended: the trace's I stays 0.
int ora_trace_ray(const OraScene* s, double alpha, double beta, double t_cam, const double* nus, int nf,
                  double* I, double* tau, int* steps, double* trace, int max_trace) {
    double x[4], k[4], fd[4];
    ora_camera(s, alpha, beta, t_cam, x, k);
    start_derivative(s, x, k, fd);
    for (int f = 0; f < nf; ++f) { I[f] = 0.0; tau[f] = 0.0; }
    std::vector<std::vector<double>> fwd(s->rt_scheme == 1 ? nf : 0);
    const double r_stop = s->r_stop_factor * horizon(s);
    int n = 0, status = 3;
    while (n < s->max_steps) {
        const double dl = step_size(s, x, k);
        advance(s, x, k, fd, dl);
        ++n;
        bool finite = true;
        for (int i = 0; i < 4; ++i) finite = finite && std::isfinite(x[i]) && std::isfinite(k[i]);
        double gr = 0.0;
        int done = -1;
        if (!finite) done = 4;
        else if (x[1] < r_stop) done = 1;
        else if (x[1] > s->r_esc) done = 0;
        else if (rt_sample(s, x, k, dl, nus, nf, I, tau, &gr, fwd.empty() ? nullptr : fwd.data())) done = 4;
        if (trace && n <= max_trace) {
            double* T = trace + (size_t)(n - 1) * 12;
            for (int i = 0; i < 4; ++i) { T[i] = x[i]; T[4 + i] = k[i]; }
            T[8] = dl; T[9] = gr; T[10] = nf > 0 ? I[0] : 0.0; T[11] = nf > 0 ? tau[0] : 0.0;
        }
        if (done >= 0) { status = done; break; }
        if (nf > 0) {
            double tmin = tau[0];
            for (int f = 1; f < nf; ++f) tmin = std::fmin(tmin, tau[f]);
            if (tmin > s->tau_cut) { status = 2; break; }
        }
    }
    for (size_t f = 0; f < fwd.size(); ++f) {
        double Iinv = 0.0;
        for (size_t q = fwd[f].size(); q >= 2; q -= 2) Iinv = Iinv * std::exp(-fwd[f][q - 2]) + fwd[f][q - 1];
        I[f] = Iinv;
    }
    if (steps) *steps = n;
    return status;
}

// Geodesic only: integrate from the camera until termination or max_steps; returns the
// status (0 escaped, 1 captured, 3 truncated, 4 error) and the final state.
int ora_geodesic(const OraScene* s, double alpha, double beta, int max_steps, double* x, double* k, int* steps) {
    ora_camera(s, alpha, beta, 0.0, x, k);
    double fd[4];
    start_derivative(s, x, k, fd);
    const double r_stop = s->r_stop_factor * horizon(s);
    int n = 0, status = 3;
    while (n < max_steps) {
        const double dl = step_size(s, x, k);
        double xn[4], kn[4], fn[4];
        for (int i = 0; i < 4; ++i) { xn[i] = x[i]; kn[i] = k[i]; fn[i] = fd[i]; }
        advance(s, xn, kn, fn, dl);
        bool finite = true;
        for (int i = 0; i < 4; ++i) finite = finite && std::isfinite(xn[i]) && std::isfinite(kn[i]);
        if (!finite) { status = 4; break; }
        for (int i = 0; i < 4; ++i) { x[i] = xn[i]; k[i] = kn[i]; fd[i] = fn[i]; }
        ++n;
        if (x[1] < r_stop) { status = 1; break; }
        if (x[1] > s->r_esc) { status = 0; break; }
    }
    if (steps) *steps = n;
    return status;
}

// Image (sec. 4.2.2, Table 3 integration): pixel centres alpha_j = amin + (j + 1/2) dalpha,
// beta_i = bmin + (i + 1/2) dbeta; image[f][i][j] in Jy per pixel:
//   F = I_obs dalpha dbeta L^2 / D^2 / 1e-23.
// Only rows [row0, row0 + nrows) are traced (nrows <= 0: all rows); image rows are
// indexed from row0.  Pixel loop in parallel over `nthreads` OpenMP threads.
int ora_render(const OraScene* s, const double* nus, int nf, double t_cam, int row0, int nrows,
               double* image, int* steps, int* status, int nthreads) {
    if (nrows <= 0) { row0 = 0; nrows = s->ny; }
    const double da = (s->amax - s->amin) / s->nx, db = (s->bmax - s->bmin) / s->ny;
    const double L = O_G * s->mass_msun * O_MSUN / (O_C * O_C);
    const double D = s->dist_pc * O_PC;
    const double pix = da * db * L * L / (D * D) / 1e-23;
    const long npix = (long)nrows * s->nx;
    const size_t plane = (size_t)nrows * s->nx;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long p = 0; p < npix; ++p) {
        const int i = (int)(p / s->nx) + row0, j = (int)(p % s->nx);
        const double alpha = s->amin + (j + 0.5) * da;
        const double beta = s->bmin + (i + 0.5) * db;
        double I[64], tau[64];
        int n = 0;
        const int st = ora_trace_ray(s, alpha, beta, t_cam, nus, nf, I, tau, &n, nullptr, 0);
        for (int f = 0; f < nf; ++f) image[f * plane + p] = I[f] * pix;
        if (steps) steps[p] = n;
        if (status) status[p] = st;
    }
    return 0;
}

// ---------------------------------------------------------------------------------------
// Thin-disk line emission (sec. 4.2.1): a geometrically thin, optically thick disk in the
// equatorial plane between r_in (the ISCO when r_in <= 0) and r_out, on prograde circular
// Keplerian orbits (Omega = 1/(r^{3/2} + a); retrograde relative to the hole for a < 0),
// emitting a monochromatic line with emission ~ r^{-q} (q = 2 in the paper), no absorption.
// Readings (the paper gives the model, not the discrete rules):
//   * a crossing of theta = pi/2 is a step whose end points lie on opposite sides (or whose
//     end point lies on the plane); its point is found by Newton's iteration on the RK4 step
//     length h from the state before the step: theta(h) = the polar angle after one RK4 step
//     of length h, h <- h - (theta(h) - pi/2) / k^theta(h), from the linear estimate, a fixed
//     four iterations, then the step of the final length;
//   * the ray stops at the first crossing with r_in <= r <= r_out (the disk is opaque);
//     crossings outside the disk count towards the image order, and after max_cross of them
//     the ray stops without a hit;
//   * E_obs / E_em = 1 / g with g = k.u (Eq. 30 for the backward ray), and the line's
//     frequency-integrated intensity at the camera is I = (E_obs/E_em)^4 r^{-q} (I_nu / nu^3
//     invariant, Eq. 31, integrated over the line).
// Status: 0 escaped, 1 captured, 3 truncated, 4 error, 5 disk hit, 6 max_cross crossings
// without a hit.  out[7]: E_obs/E_em, I, order (crossing number of the hit), r and theta of
// the hit, g, steps (the refinement counts as one step).
// ---------------------------------------------------------------------------------------
static void disk_crossing(const OraScene* s, const double x0[4], const double k0[4], double dl, double th1,
                          double xc[4], double kc[4]) {
    const double half_pi = 0.5 * O_PI;
    double h = dl * (half_pi - x0[2]) / (th1 - x0[2]);
    for (int it = 0; it < 4; ++it) {
        for (int i = 0; i < 4; ++i) { xc[i] = x0[i]; kc[i] = k0[i]; }
        rk4_step(s, xc, kc, h);
        if (!(std::fabs(kc[2]) > 0.0)) break;
        h -= (xc[2] - half_pi) / kc[2];
    }
    for (int i = 0; i < 4; ++i) { xc[i] = x0[i]; kc[i] = k0[i]; }
    rk4_step(s, xc, kc, h);
}

int ora_disk_ray(const OraScene* s, double alpha, double beta, double r_in, double r_out, double q, int max_cross,
                 double* out) {
    const double half_pi = 0.5 * O_PI;
    if (r_in <= 0.0) r_in = ora_r_isco(s->a);
    double x[4], k[4];
    ora_camera(s, alpha, beta, 0.0, x, k);
    for (int i = 0; i < 7; ++i) out[i] = 0.0;
    const double r_stop = s->r_stop_factor * horizon(s);
    int n = 0, status = 3, crossings = 0;
    while (n < s->max_steps) {
        const double dl = step_size(s, x, k);
        double xn[4], kn[4];
        for (int i = 0; i < 4; ++i) { xn[i] = x[i]; kn[i] = k[i]; }
        rk4_step(s, xn, kn, dl);
        ++n;
        bool finite = true;
        for (int i = 0; i < 4; ++i) finite = finite && std::isfinite(xn[i]) && std::isfinite(kn[i]);
        if (!finite) { status = 4; break; }
        if ((x[2] - half_pi) * (xn[2] - half_pi) <= 0.0 && x[2] != half_pi) {
            crossings += 1;
            double xc[4], kc[4];
            disk_crossing(s, x, k, dl, xn[2], xc, kc);
            const double rc = xc[1];
            if (rc >= r_in && rc <= r_out) {
                // Keplerian velocity in BL at the crossing point, then to KS (App. A.1)
                OraScene bl = *s;
                bl.coords = 1;
                M4 gb;
                metric(&bl, rc, xc[2], gb);
                const double Om = 1.0 / (std::pow(rc, 1.5) + s->a);
                const double nrm = gb[0][0] + 2.0 * Om * gb[0][3] + Om * Om * gb[3][3];
                if (!(nrm < 0.0)) { status = 4; break; }
                double ub[4] = {1.0 / std::sqrt(-nrm), 0.0, 0.0, 0.0};
                ub[3] = Om * ub[0];
                double uk[4];
                if (s->coords == 0) vec_bl_to_ks(s, rc, ub, uk);
                else for (int i = 0; i < 4; ++i) uk[i] = ub[i];
                M4 g;
                metric(s, rc, xc[2], g);
                double gr = 0.0;
                for (int mu = 0; mu < 4; ++mu)
                    for (int nu = 0; nu < 4; ++nu) gr += g[mu][nu] * kc[mu] * uk[nu];
                if (!(gr > 0.0)) { status = 4; break; }
                const double ratio = 1.0 / gr;
                out[0] = ratio;
                out[1] = ratio * ratio * ratio * ratio * std::pow(rc, -q);
                out[2] = crossings;
                out[3] = rc;
                out[4] = xc[2];
                out[5] = gr;
                status = 5;
                break;
            }
            if (crossings >= max_cross) { status = 6; break; }
        }
        for (int i = 0; i < 4; ++i) { x[i] = xn[i]; k[i] = kn[i]; }
        if (x[1] < r_stop) { status = 1; break; }
        if (x[1] > s->r_esc) { status = 0; break; }
    }
    out[6] = n;
    return status;
}

// Ordered equatorial crossings of one ray (the thin disk's geometry, sec. 4.2.1, without the
// disk): the ray is traced from the camera as in ora_disk_ray, and every crossing of
// theta = pi/2 is refined by the same Newton iteration on the RK4 step length; its radius,
// coordinate time and affine length from the camera (the sum of the accepted steps before it
// plus the refined step) are recorded, up to max_n crossings.  The trace continues from the
// unrefined step end (crossings change nothing on the ray) until capture, escape, the step
// cap or the max_n-th crossing.  Returns the number of crossings found; *fate gets 0 escaped,
// 1 captured, 3 truncated, 4 error, 7 stopped at the max_n-th crossing.
int ora_disk_crossings(const OraScene* s, double alpha, double beta, int max_n, double* r_out, double* lam_out,
                       double* t_out, int* fate, int* steps) {
    const double half_pi = 0.5 * O_PI;
    double x[4], k[4];
    ora_camera(s, alpha, beta, 0.0, x, k);
    const double r_stop = s->r_stop_factor * horizon(s);
    int n = 0, found = 0, status = 3;
    double lam = 0.0;
    while (n < s->max_steps) {
        const double dl = step_size(s, x, k);
        double xn[4], kn[4];
        for (int i = 0; i < 4; ++i) { xn[i] = x[i]; kn[i] = k[i]; }
        rk4_step(s, xn, kn, dl);
        ++n;
        bool finite = true;
        for (int i = 0; i < 4; ++i) finite = finite && std::isfinite(xn[i]) && std::isfinite(kn[i]);
        if (!finite) { status = 4; break; }
        if ((x[2] - half_pi) * (xn[2] - half_pi) <= 0.0 && x[2] != half_pi) {
            // the refined step length: the Newton iteration of disk_crossing, repeated here
            // so that the length itself is available
            double h = dl * (half_pi - x[2]) / (xn[2] - x[2]);
            double xc[4], kc[4];
            for (int it = 0; it < 4; ++it) {
                for (int i = 0; i < 4; ++i) { xc[i] = x[i]; kc[i] = k[i]; }
                rk4_step(s, xc, kc, h);
                if (!(std::fabs(kc[2]) > 0.0)) break;
                h -= (xc[2] - half_pi) / kc[2];
            }
            for (int i = 0; i < 4; ++i) { xc[i] = x[i]; kc[i] = k[i]; }
            rk4_step(s, xc, kc, h);
            r_out[found] = xc[1];
            lam_out[found] = lam + h;
            t_out[found] = xc[0];
            found += 1;
            if (found >= max_n) { status = 7; break; }
        }
        lam += dl;
        for (int i = 0; i < 4; ++i) { x[i] = xn[i]; k[i] = kn[i]; }
        if (x[1] < r_stop) { status = 1; break; }
        if (x[1] > s->r_esc) { status = 0; break; }
    }
    *fate = status;
    *steps = n;
    return found;
}

// Disk image: per pixel (centres as in ora_render) E_obs/E_em, I, hit order, status and
// steps (0 where the ray does not hit the disk), OpenMP over pixels.
int ora_disk_render(const OraScene* s, double r_in, double r_out, double q, int max_cross, double* ratio,
                    double* inten, int* order, int* status, int* steps, int nthreads) {
    const double da = (s->amax - s->amin) / s->nx, db = (s->bmax - s->bmin) / s->ny;
    const long npix = (long)s->ny * s->nx;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long p = 0; p < npix; ++p) {
        const int i = (int)(p / s->nx), j = (int)(p % s->nx);
        double out[7];
        const int st = ora_disk_ray(s, s->amin + (j + 0.5) * da, s->bmin + (i + 0.5) * db, r_in, r_out, q, max_cross, out);
        ratio[p] = out[0];
        inten[p] = out[1];
        order[p] = (int)out[2];
        status[p] = st;
        steps[p] = (int)out[6];
    }
    return 0;
}

// Geometric unit conversions used by the tests.
double ora_length_unit_cm(double mass_msun) { return O_G * mass_msun * O_MSUN / (O_C * O_C); }

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
