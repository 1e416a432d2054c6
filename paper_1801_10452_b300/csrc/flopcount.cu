// flopcount.cu -- source-level operation count of one geodesic step and its transfer
// sample, obtained by instantiating the kernels' templated arithmetic (raptor_math.cuh,
// raptor_physics.cuh, raptor_grid.cuh) on the host with a number type that counts every
// operation.  A fused multiply-add in the compiled kernel is a multiply plus an add here,
// so the count is the algorithmic flop count with FMA = 2.  Prints one JSON object.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <vector>

namespace raptor {
namespace count {
struct Ops {
    unsigned long long add = 0, mul = 0, div = 0, sqrt = 0, rsqrt = 0, cbrt = 0, exp = 0, expm1 = 0, log = 0, pow = 0,
                       sincos = 0, cmp = 0;
};
static Ops g_ops;

struct Cnt {
    double v;
    Cnt() : v(0.0) {}
    Cnt(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    explicit operator float() const { return (float)v; }
};
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline bool operator<(Cnt a, Cnt b) { g_ops.cmp++; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { g_ops.cmp++; return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { g_ops.cmp++; return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { g_ops.cmp++; return a.v >= b.v; }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }
inline Cnt fmin(Cnt a, Cnt b) { g_ops.cmp++; return Cnt(std::fmin(a.v, b.v)); }
inline Cnt fmax(Cnt a, Cnt b) { g_ops.cmp++; return Cnt(std::fmax(a.v, b.v)); }
inline Cnt floor(Cnt a) { return Cnt(std::floor(a.v)); }
inline void sc(Cnt v, Cnt* s, Cnt* c) { g_ops.sincos++; *s = Cnt(std::sin(v.v)); *c = Cnt(std::cos(v.v)); }
inline Cnt rsq(Cnt v) { g_ops.rsqrt++; return Cnt(1.0 / std::sqrt(v.v)); }
}  // namespace count
using count::Cnt;
using count::Ops;
using count::g_ops;
template <typename T> struct Real;
template <>
struct Real<Cnt> {
    static Cnt sqrt_(Cnt v) { g_ops.sqrt++; return Cnt(std::sqrt(v.v)); }
    static Cnt cbrt_(Cnt v) { g_ops.cbrt++; return Cnt(std::cbrt(v.v)); }
    static Cnt exp_(Cnt v) { g_ops.exp++; return Cnt(std::exp(v.v)); }
    static Cnt expm1_(Cnt v) { g_ops.expm1++; return Cnt(std::expm1(v.v)); }
    static Cnt pow_(Cnt b, Cnt e) { g_ops.pow++; return Cnt(std::pow(b.v, e.v)); }
    static Cnt log_(Cnt v) { g_ops.log++; return Cnt(std::log(v.v)); }
    static Cnt rcp(Cnt v) { g_ops.div++; return Cnt(1.0 / v.v); }
    static constexpr double exp_cut = 700.0;
};
}  // namespace raptor

#include "raptor_grid.cuh"

namespace raptor {
template <>
struct NewtonTol<Cnt> { static constexpr double v = 1e-14; };
template <>
Cnt pv<Cnt>(double d, float) { return Cnt(d); }
}  // namespace raptor

using namespace raptor;

static void print_ops(const char* name, const Ops& o, bool last) {
    const unsigned long long flops = o.add + o.mul + o.div + o.sqrt + o.rsqrt + o.cbrt + o.exp + o.expm1 + o.log + o.pow + o.sincos;
    std::printf("\"%s\": {\"flops\": %llu, \"add\": %llu, \"mul\": %llu, \"div\": %llu, \"sqrt\": %llu, \"rsqrt\": %llu, "
                "\"cbrt\": %llu, \"exp\": %llu, \"expm1\": %llu, \"log\": %llu, \"pow\": %llu, \"sincos\": %llu, \"cmp\": %llu}%s\n",
                name, flops, o.add, o.mul, o.div, o.sqrt, o.rsqrt, o.cbrt, o.exp, o.expm1, o.log, o.pow, o.sincos, o.cmp,
                last ? "" : ",");
}

int main() {
    Params p;
    std::memset(&p, 0, sizeof(p));
    p.a = 0.9375;
    p.eps = 0.05;
    p.kind = 0;
    p.n0 = 1e6; p.n_pow = -1.5; p.the0 = 10.0; p.the_pow = -1.0; p.B0 = 20.0; p.B_pow = -1.0;
    p.r_isco = 2.0445;
    p.Lcm = 5.9e11;
    // a representative emitting state: the ray of pixel (alpha, beta) = (3, 2) of the
    // a = 0.9375, i = 60 deg camera, integrated in double until r < 4
    p.r_cam = 1000.0;
    p.incl = 60.0 * kPi / 180.0;
    p.sin_i = std::sin(p.incl);
    p.cos_i = std::cos(p.incl);
    double xd[4], kd[4];
    camera_ray(p, 3.0, 2.0, 0.0, xd, kd);
    for (int n = 0; n < 10000 && xd[1] >= 4.0; ++n) rk4_step<double>(p.a, xd, kd, step_size<double>(p.eps, false, xd, kd));
    Cnt x[4], k[4];
    for (int i = 0; i < 4; ++i) { x[i] = Cnt(xd[i]); k[i] = Cnt(kd[i]); }
    std::printf("{\n");
    // geodesic: step size + RK4 (4 right-hand sides)
    g_ops = Ops();
    Cnt dl = step_size<Cnt>(Cnt(p.eps), false, x, k);
    rk4_step<Cnt>(Cnt(p.a), x, k, dl);
    print_ops("geodesic_step", g_ops, false);
    // one right-hand side alone
    g_ops = Ops();
    Cnt f[4];
    geodesic_force<Cnt>(Cnt(p.a), x[1], x[2], k, f);
    print_ops("geodesic_rhs", g_ops, false);
    // velocity Verlet (sec. 2.2.2): step size + one step, without and with the re-evaluation
    {
        Cnt xv[4], kv[4], fv[4];
        for (int i = 0; i < 4; ++i) { xv[i] = x[i]; kv[i] = k[i]; fv[i] = f[i]; }
        g_ops = Ops();
        Cnt dv = step_size<Cnt>(Cnt(p.eps), false, xv, kv);
        verlet_step<Cnt>(Cnt(p.a), xv, kv, fv, dv, false);
        print_ops("verlet_step", g_ops, false);
        for (int i = 0; i < 4; ++i) { xv[i] = x[i]; kv[i] = k[i]; fv[i] = f[i]; }
        g_ops = Ops();
        dv = step_size<Cnt>(Cnt(p.eps), false, xv, kv);
        verlet_step<Cnt>(Cnt(p.a), xv, kv, fv, dv, true);
        print_ops("verlet_reeval_step", g_ops, false);
    }
    // analytic plasma sample (Keplerian branch) and the free-fall branch
    Cnt ne, the, B, g, sinb;
    g_ops = Ops();
    plasma_sample<Cnt>(p, x, k, 0, ne, the, B, g, sinb);
    print_ops("sample_analytic", g_ops, false);
    Cnt xi[4] = {x[0], Cnt(1.8), x[2], x[3]};
    g_ops = Ops();
    plasma_sample<Cnt>(p, xi, k, 0, ne, the, B, g, sinb);
    print_ops("sample_analytic_freefall", g_ops, false);
    // per frequency: emissivity + transfer update
    g_ops = Ops();
    plasma_sample<Cnt>(p, x, k, 0, ne, the, B, g, sinb);
    g_ops = Ops();
    Cnt j, S, I(0.0), tau(0.0);
    synchrotron<Cnt>(g * Cnt(2.3e11), ne, the, B, sinb, false, j, S);
    rt_update<Cnt, Cnt>(j, S, g, dl * Cnt(p.Lcm), I, tau);
    print_ops("per_frequency", g_ops, false);
    // grid plasma sample: a 4 x 4 uniform grid around the state, one snapshot
    std::vector<float> grid(4 * 4 * 8);
    for (int c = 0; c < 16; ++c) {
        float* q = &grid[c * 8];
        q[0] = 1.0f; q[1] = 0.1f; q[2] = 0.0f; q[3] = 0.0f; q[4] = 0.05f; q[5] = 0.01f; q[6] = 0.0f; q[7] = 0.0f;
    }
    p.kind = 1;
    p.grid = grid.data();
    p.n1 = 4; p.n2 = 4; p.n_snap = 1;
    p.x1_min = std::log(1.3); p.x1_max = std::log(50.0);
    p.dx1 = (p.x1_max - p.x1_min) / 4; p.dx2 = 0.25; p.h_mks = 0.3;
    p.rho0_ne = 1e6; p.B_unit = 100.0; p.r_high = 1.0; p.r_low = 1.0; p.gam = 4.0 / 3.0;
    g_ops = Ops();
    plasma_sample<Cnt>(p, x, k, 0, ne, the, B, g, sinb);
    print_ops("sample_grid_fast", g_ops, false);
    p.slow = 1; p.n_snap = 1;
    std::vector<float> grid2(2 * 4 * 4 * 8);
    for (size_t i = 0; i < grid2.size(); ++i) grid2[i] = grid[i % grid.size()];
    p.grid = grid2.data(); p.n_snap = 2; p.t0 = -1000.0; p.dt_snap = 10.0;
    g_ops = Ops();
    plasma_sample<Cnt>(p, x, k, 0, ne, the, B, g, sinb);
    print_ops("sample_grid_slow", g_ops, true);
    std::printf("}\n");
    return 0;
}
