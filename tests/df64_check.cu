// df64_check.cu (test harness, built by tests/test_df64.py) -- host check of the double-float arithmetic against long double: prints
// the largest relative errors of add, mul, div, sqrt and sincos over seeded random operands.
#include <cmath>
#include <cstdio>
#include <random>

#include "raptor_df64.cuh"

using namespace raptor;

static long double LD(df64 v) { return (long double)v.hi + (long double)v.lo; }
static df64 mk(double d) { return df64(d); }

int main() {
    std::mt19937_64 g(1801104520ull);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    double e_add = 0, e_mul = 0, e_div = 0, e_sqrt = 0, e_sin = 0, e_cos = 0, e_tab = 0;
    for (int i = 0; i < 200000; ++i) {
        const double a = u(g) * std::pow(10.0, 3 * u(g)), b = u(g) * std::pow(10.0, 3 * u(g));
        const df64 A = mk(a), B = mk(b);
        const long double la = LD(A), lb = LD(B);
        auto rel = [](long double x, long double ref) { return (double)(fabsl(x - ref) / fmaxl(fabsl(ref), 1e-300L)); };
        // add: error relative to the magnitude of the operands (cancellation is exact in df64)
        e_add = std::fmax(e_add, (double)(fabsl(LD(A + B) - (la + lb)) / fmaxl(fabsl(la) + fabsl(lb), 1e-300L)));
        e_mul = std::fmax(e_mul, rel(LD(A * B), la * lb));
        e_div = std::fmax(e_div, rel(LD(A / B), la / lb));
        const df64 P = mk(std::fabs(a));
        e_sqrt = std::fmax(e_sqrt, rel(LD(df_sqrt(P)), sqrtl(LD(P))));
        const double th = 3.14159265358979 * (0.5 + 0.5 * u(g));
        const df64 T = mk(th);
        df64 s, c;
        df_sincos(T, &s, &c);
        e_sin = std::fmax(e_sin, (double)fabsl(LD(s) - sinl(LD(T))));
        e_cos = std::fmax(e_cos, (double)fabsl(LD(c) - cosl(LD(T))));
        // the table-based form used by the geodesic steps (theta in [0, pi]) and its fallback
        const df64 T2 = mk(3.14159265358979 * 0.5 * (1.0 + 1.04 * u(g)));
        df64 s2, c2;
        df_sincos_tab(T2, &s2, &c2);
        e_tab = std::fmax(e_tab, (double)std::fmax(fabsl(LD(s2) - sinl(LD(T2))), fabsl(LD(c2) - cosl(LD(T2)))));
    }
    std::printf("{\"add\": %.3e, \"mul\": %.3e, \"div\": %.3e, \"sqrt\": %.3e, \"sin_abs\": %.3e, \"cos_abs\": %.3e, "
                "\"sincos_table_abs\": %.3e}\n", e_add, e_mul, e_div, e_sqrt, e_sin, e_cos, e_tab);
    return 0;
}
