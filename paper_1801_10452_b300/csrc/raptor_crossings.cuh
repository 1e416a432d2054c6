// raptor_crossings.cuh -- the learned surrogate's equatorial outputs: (alpha, beta, a, i) ->
// the first four crossings of the plane theta = pi/2 by the backward ray (sec. 4.2.1's thin
// disk geometry), each with its radius, affine length and the energy ratio E_obs/E_em of a
// Keplerian emitter there.  Training data from the FP64 integrator, a loss for the network's
// 16 outputs, and the learned thin-disk image: the network's first crossing inside the disk
// gives a pixel's hit, and the exact integrator (k_disk_fp64 over a pixel list) takes the
// pixels near the critical curve.
#pragma once

#include "raptor_df64.cuh"
#include "raptor_kernels_fp64.cuh"
#include "raptor_surrogate.cuh"

namespace raptor {

constexpr int kCross = 4;              // crossings per ray
constexpr int kXOut = 4 * kCross;      // per crossing: presence logit, ln r, affine length, E_obs/E_em
using XLayout = MlpLayoutT<kXOut>;

// Quiet NaN: the mark of an absent target.
__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7FF8000000000000ll); }

// The straight camera ray (flat space, FP32) as the baseline of the first crossing: its
// affine length to the plane, the camera's height r cos i over the ray's downward rate, and
// the log of its radius there, softened as ln sqrt(r_flat^2 + 9) so that it stays finite for
// rays aimed at the centre.  The network learns the first crossing against these (the
// gravitational delay and deflection).  A ray that never descends: 0 and ln 3.
RAPTOR_HD void crossing_flat(float a, float sn_i, float cs_i, float r_cam, float alpha, float beta, float* lam_flat,
                             float* lnr_flat) {
    float k0[4];
    camera_k_t<float>(a, sn_i, cs_i, r_cam, alpha, beta, k0);
    // camera at (r sin i, 0, r cos i); velocity from (k^r, k^theta, k^phi) at phi = 0
    const float vx = k0[1] * sn_i + r_cam * k0[2] * cs_i;
    const float vy = r_cam * sn_i * k0[3];
    const float vz = k0[1] * cs_i - r_cam * k0[2] * sn_i;
    const float lam = vz < 0.f ? -r_cam * cs_i / vz : 0.f;
    const float X = r_cam * sn_i + vx * lam, Y = vy * lam;
    *lam_flat = lam;
    *lnr_flat = 0.5f * logf(X * X + Y * Y + 9.f);
}

// E_obs/E_em of a prograde Keplerian equatorial emitter at radius r for a photon of E = 1 and
// angular momentum L (Eq. 30 with u = u^t (1, 0, 0, Omega) in BL, Omega = 1/(r^{3/2} + a)):
// 1 / (u^t (1 - Omega L)); 0 where the orbit is not timelike or the energy not positive.
__device__ __forceinline__ double kepler_ratio(double r, double a, double L) {
    const double om = 1.0 / (r * sqrt(r) + a);
    const double gtt = -(1.0 - 2.0 / r), gtp = -2.0 * a / r, gpp = r * r + a * a + 2.0 * a * a / r;
    const double nrm = gtt + 2.0 * om * gtp + om * om * gpp;
    if (!(nrm < 0.0)) return 0.0;
    const double e = (1.0 - om * L) / sqrt(-nrm);
    return e > 0.0 ? 1.0 / e : 0.0;
}

// E_obs/E_em of an equatorial emitter on a prograde Keplerian orbit at the crossing (xc, kc)
// (the thin disk's Eq. 30 ratio, as k_disk_fp64 takes it); NaN when the orbit is not
// timelike or the energy is not positive.
__device__ __forceinline__ double crossing_ratio(double a, const double xc[4], const double kc[4]) {
    KSPoint<double> P;
    ks_point<double>(a, xc[1], xc[2], P);
    double u[4], kcov[4];
    if (analytic_velocity<double>(a, 0.0, P, u) < 0) return qnan();
    ks_lower(P, kc, kcov);
    const double g = kcov[0] * u[0] + kcov[1] * u[1] + kcov[2] * u[2] + kcov[3] * u[3];
    return g > 0.0 ? 1.0 / g : qnan();
}

// The integrator's crossings of one ray and the network's targets.  The ray is traced from
// the camera with the FP64 RK4 step of the renders; each step whose end lies on the other
// side of the plane is refined by disk_crossing (Newton on the step length) and the crossing
// recorded; the trace goes on from the unrefined step end until capture (r < r_stop),
// escape (r > r_esc), the step cap, a non-finite state or the fourth crossing.
//   targets[4n]     1 if crossing n exists, else 0
//   targets[4n + 1] ln r_n, minus the straight ray's ln r for n = 0 (NaN if absent)
//   targets[4n + 2] lambda_n - lambda_{n-1}, lambda_{-1} = the straight ray's length (NaN if absent)
//   targets[4n + 3] E_obs/E_em at r_n for r_n >= r_isco      (NaN if absent or inside)
//   raw (optional)  per crossing: presence, r_n, lambda_n, E_obs/E_em (NaN for absent; the
//                   ratio at every radius where the orbit is timelike)
// Returns the number of steps taken.
__device__ int crossing_targets(double a, double incl_deg, double r_cam, double eps, double r_stop_factor, double r_esc,
                                int max_steps, double alpha, double beta, double* targets, double* raw) {
    const double inc = incl_deg * (kPi / 180.0);
    const double sn = sin(inc), cs = cos(inc);
    double x[4], k[4];
    camera_ray_ai(a, sn, cs, inc, r_cam, alpha, beta, 0.0, x, k);
    const double r_h = 1.0 + sqrt(1.0 - a * a);
    const double r_stop = r_stop_factor * r_h;
    double r_isco;
    {
        // Bardeen-Press-Teukolsky ISCO of the emitter's orbit (prograde for a >= 0)
        const double z1 = 1.0 + cbrt(1.0 - a * a) * (cbrt(1.0 + a) + cbrt(1.0 - a));
        const double z2 = sqrt(3.0 * a * a + z1 * z1);
        r_isco = 3.0 + z2 - (a < 0.0 ? -1.0 : 1.0) * sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
    }
    float lam_flat_f, lnr_flat_f;
    crossing_flat((float)a, (float)sn, (float)cs, (float)r_cam, (float)alpha, (float)beta, &lam_flat_f, &lnr_flat_f);
    const double lam_flat = (double)lam_flat_f;
    for (int q = 0; q < kXOut; ++q) {
        targets[q] = (q % 4 == 0) ? 0.0 : qnan();
        if (raw) raw[q] = (q % 4 == 0) ? 0.0 : qnan();
    }
    const double half_pi = 0.5 * kPi;
    double lam = 0.0, lam_prev = lam_flat;
    int n = 0, found = 0;
    while (n < max_steps) {
        const double dl = step_size<double>(eps, false, x, k);
        double xo[4], ko[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { xo[i] = x[i]; ko[i] = k[i]; }
        rk4_step<double>(a, x, k, dl);
        n += 1;
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) fin = fin && isfinite(x[i]) && isfinite(k[i]);
        if (!fin) break;
        if ((xo[2] - half_pi) * (x[2] - half_pi) <= 0.0 && xo[2] != half_pi) {
            double xc[4], kc[4], h = 0.0;
            disk_crossing(a, xo, ko, dl, x[2], xc, kc, &h);
            const double rc = xc[1], lc = lam + h;
            const double ratio = crossing_ratio(a, xc, kc);
            targets[4 * found] = 1.0;
            targets[4 * found + 1] = log(rc) - (found == 0 ? (double)lnr_flat_f : 0.0);
            targets[4 * found + 2] = lc - lam_prev;
            targets[4 * found + 3] = rc >= r_isco ? ratio : qnan();
            if (raw) {
                raw[4 * found] = 1.0;
                raw[4 * found + 1] = rc;
                raw[4 * found + 2] = lc;
                raw[4 * found + 3] = ratio;
            }
            lam_prev = lc;
            found += 1;
            if (found >= kCross) break;
        }
        lam += dl;
        if (x[1] < r_stop || x[1] > r_esc) break;
    }
    return n;
}

// Training data: counter-based inputs as k_surrogate_data draws them (rounded to FP32 before
// the targets are computed), targets [n][16], raw [n][16] optional.
__global__ void __launch_bounds__(128) k_crossing_data(SurrogateRange R, double r_stop_factor, double r_esc, int max_steps,
                                                       uint64_t seed, long long n, float* __restrict__ inputs,
                                                       double* __restrict__ targets, double* __restrict__ raw) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double al = (double)(float)(R.amin + (R.amax - R.amin) * u01(seed, i, 0));
        const double be = (double)(float)(R.bmin + (R.bmax - R.bmin) * u01(seed, i, 1));
        const double a = (double)(float)(R.smin + (R.smax - R.smin) * u01(seed, i, 2));
        const double inc = (double)(float)(R.imin + (R.imax - R.imin) * u01(seed, i, 3));
        inputs[i * kIn + 0] = (float)al;
        inputs[i * kIn + 1] = (float)be;
        inputs[i * kIn + 2] = (float)a;
        inputs[i * kIn + 3] = (float)inc;
        crossing_targets(a, inc, R.r_cam, R.eps, r_stop_factor, r_esc, max_steps, al, be, targets + i * kXOut,
                         raw ? raw + i * kXOut : nullptr);
    }
}

// Loss of the crossing network, per row and output averaged over rows x 16: the logistic
// loss log(1 + e^z) - y z on the presence logits (o % 4 == 0), (z - (y - mu)/sigma)^2 on the
// others, nothing where the target is NaN.  dout = d loss / d out; per-block partial sums
// of the loss in loss_acc (fixed order).
// Floats as unsigned integers whose order is the floats' order (sign bit flipped for
// non-negative values, all bits flipped for negative ones), for atomicMin / atomicMax.
__host__ __device__ __forceinline__ unsigned float_to_ordered(float v) {
    unsigned u;
    memcpy(&u, &v, sizeof(u));
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ordered_to_float(unsigned o) {
    const unsigned u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    float v;
    memcpy(&v, &u, sizeof(v));
    return v;
}

// Smallest and largest spin (column 2) and inclination (column 3) of n network inputs [n][4]:
// mm = {min a, max a, min i, max i} as ordered integers (initialised by the caller to
// {UINT_MAX, 0, UINT_MAX, 0}).
__global__ void __launch_bounds__(256) k_input_range(const float* __restrict__ x, long long n, unsigned* __restrict__ mm) {
    unsigned lo_a = 0xFFFFFFFFu, hi_a = 0u, lo_i = 0xFFFFFFFFu, hi_i = 0u;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
        const unsigned oa = float_to_ordered(x[m * 4 + 2]), oi = float_to_ordered(x[m * 4 + 3]);
        lo_a = min(lo_a, oa);
        hi_a = max(hi_a, oa);
        lo_i = min(lo_i, oi);
        hi_i = max(hi_i, oi);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo_a = min(lo_a, __shfl_down_sync(0xffffffffu, lo_a, o));
        hi_a = max(hi_a, __shfl_down_sync(0xffffffffu, hi_a, o));
        lo_i = min(lo_i, __shfl_down_sync(0xffffffffu, lo_i, o));
        hi_i = max(hi_i, __shfl_down_sync(0xffffffffu, hi_i, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm + 0, lo_a);
        atomicMax(mm + 1, hi_a);
        atomicMin(mm + 2, lo_i);
        atomicMax(mm + 3, hi_i);
    }
}

__global__ void k_cross_grad(const float* __restrict__ P, const float* __restrict__ out, const double* __restrict__ y,
                             long long rows, float* __restrict__ dout, double* __restrict__ loss_acc) {
    __shared__ double sh[256];
    double part = 0.0;
    const float inv = 1.f / (float)(rows * kXOut);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * kXOut; e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e % kXOut);
        const double t = y[e];
        const float z = out[e];
        float g = 0.f;
        if (!isnan(t)) {
            if ((o & 3) == 0) {
                const float tf = (float)t;
                const float sig = 1.f / (1.f + expf(-z));
                part += (double)(fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - tf * z);
                g = (sig - tf) * inv;
            } else {
                const float yn = (float)((t - P[XLayout::MU + o]) / P[XLayout::SD + o]);
                const float d = z - yn;
                part += (double)d * d;
                g = 2.f * d * inv;
            }
        }
        dout[e] = g;
    }
    sh[threadIdx.x] = part;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_acc[blockIdx.x] = sh[0];
}

// Decoded predictions [n][16] from the network outputs: per crossing the presence
// probability, r, the affine length from the camera (the straight ray's length plus the
// predicted increments) and E_obs/E_em.
__global__ void k_crossings_decode(const float* __restrict__ P, const float* __restrict__ x, const float* __restrict__ out,
                                   long long n, float r_cam, double* __restrict__ pred) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float al = x[i * kIn], be = x[i * kIn + 1], a = x[i * kIn + 2], inc = x[i * kIn + 3] * (float)(kPi / 180.0);
        float lam_f, lnr_f;
        crossing_flat(a, sinf(inc), cosf(inc), r_cam, al, be, &lam_f, &lnr_f);
        double lam = (double)lam_f;
        for (int c = 0; c < kCross; ++c) {
            const float* o = out + i * kXOut + 4 * c;
            double* d = pred + i * kXOut + 4 * c;
            const int q = 4 * c;
            d[0] = 1.0 / (1.0 + exp(-(double)o[0]));
            d[1] = exp((double)o[1] * P[XLayout::SD + q + 1] + P[XLayout::MU + q + 1] + (c == 0 ? (double)lnr_f : 0.0));
            lam += (double)o[2] * P[XLayout::SD + q + 2] + P[XLayout::MU + q + 2];
            d[2] = lam;
            d[3] = (double)o[3] * P[XLayout::SD + q + 3] + P[XLayout::MU + q + 3];
        }
    }
}

// Learned thin-disk image: pixels outside the fallback set take the first predicted crossing
// (presence logit > 0, in order; the first absent one ends the search) whose radius lies in
// [r_in, r_out]: E_obs/E_em of the Keplerian emitter at that radius (kepler_ratio, exact
// given the radius), I = (E_obs/E_em)^4 r^-q, order = its crossing number; no such crossing:
// no hit.  Fallback pixels are appended to `list` (its unused tail holds -1) for
// k_disk_fp64.
// Pixels whose decoded hit is uncertain also join the fallback list: a presence logit within
// z_margin of 0 on a crossing the decoding reads (the network cannot tell whether the ray
// crosses there), or a predicted radius within a factor exp(lnr_margin) of r_in or r_out
// (a small radius error would move the hit onto or off the disk).  There a wrong decision
// is an O(1) intensity error, not a small one.
__global__ void __launch_bounds__(256) k_disk_learned(const Params p, const DiskArgs d, const float* __restrict__ P,
                                                      const float* __restrict__ out, const unsigned char* __restrict__ fallback,
                                                      int* __restrict__ list, unsigned int* __restrict__ n_list,
                                                      float z_margin, float lnr_margin) {
    float mu[kCross], sd[kCross];
#pragma unroll
    for (int c = 0; c < kCross; ++c) {
        mu[c] = P[XLayout::MU + 4 * c + 1];
        sd[c] = P[XLayout::SD + 4 * c + 1];
    }
    const float sif = (float)p.sin_i, cif = (float)p.cos_i, rcf = (float)p.r_cam;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < p.n_rays;
         id += (long long)gridDim.x * blockDim.x) {
        const int pix = (int)id;
        if (fallback[id]) {
            list[atomicAdd(n_list, 1u)] = pix;
            continue;
        }
        const int row = pix / p.nx, col = pix - (pix / p.nx) * p.nx;
        const double al = p.amin + (col + 0.5) * p.da, be = p.bmin + (row + 0.5) * p.db;
        float lam_f, lnr_f;
        crossing_flat(p.f.a, sif, cif, rcf, (float)al, (float)be, &lam_f, &lnr_f);
        double ratio = 0.0, inten = 0.0;
        int order = 0;
        bool unsure = false;
        const float4* o4 = reinterpret_cast<const float4*>(out + id * kXOut);
        const double ln_in = log(d.r_in), ln_out = log(d.r_out);
#pragma unroll
        for (int c = 0; c < kCross; ++c) {
            const float4 o = o4[c];
            if (fabsf(o.x) < z_margin) { unsure = true; break; }
            if (!(o.x > 0.f)) break;
            const double lnr = (double)(o.y * sd[c] + mu[c]) + (c == 0 ? (double)lnr_f : 0.0);
            if (fabs(lnr - ln_in) < lnr_margin || fabs(lnr - ln_out) < lnr_margin) { unsure = true; break; }
            const double r = exp(lnr);
            if (r >= d.r_in && r <= d.r_out) {
                ratio = kepler_ratio(r, p.a, -al * p.sin_i);
                inten = ratio * ratio * ratio * ratio * pow(r, -d.q);
                order = ratio > 0.0 ? c + 1 : 0;
                break;
            }
        }
        if (unsure) {
            list[atomicAdd(n_list, 1u)] = pix;
            continue;
        }
        d.ratio[pix] = ratio;
        d.inten[pix] = inten;
        d.order[pix] = order;
        if (d.status) d.status[pix] = order ? kDiskHit : kDiskNone;
        if (d.steps) d.steps[pix] = 0;
    }
}


// ---------------------------------------------------------------------------------------
// Fallback pixels of the learned disk in double-float arithmetic (float pairs on the FP32
// pipe, ~48-bit significands): the disk ray of k_disk_fp64 with the state, the RK4 steps and
// the Newton refinement of a crossing in df64, the step length from the FP32 view of the
// state (as the mixed path's double-float phase takes it), and E_obs/E_em at a hit in FP64
// (once per ray).  FP64 issues at a small fraction of the FP32 rate on this GPU, so the
// exact fallback integration, the learned disk's largest cost, moves to the FP32 pipe.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void disk_crossing_df(df64 a, const df64 x0[4], const df64 k0[4], df64 dl, df64 th1,
                                                 df64 xc[4], df64 kc[4]) {
    const df64 hp(0.5 * kPi);
    df64 h = dl * (hp - x0[2]) / (th1 - x0[2]);
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) { xc[i] = x0[i]; kc[i] = k0[i]; }
        rk4_step_rolled<df64>(a, xc, kc, h);
        if (!(fabsf(kc[2].hi) > 0.f)) break;
        h = h - (xc[2] - hp) / kc[2];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) { xc[i] = x0[i]; kc[i] = k0[i]; }
    rk4_step_rolled<df64>(a, xc, kc, h);
}

__device__ __forceinline__ int disk_step_df(const Params& p, const DiskArgs& d, df64 a, df64 x[4], df64 k[4], int& n,
                                            int& crossings, double& ratio, double& inten) {
    const df64 hp(0.5 * kPi);
    float xf[4], kf[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { xf[i] = x[i].hi + x[i].lo; kf[i] = k[i].hi + k[i].lo; }
    const df64 dl(step_size<float>(p.f.eps, (p.flags & kFlagLinearR) != 0, xf, kf), 0.f);
    df64 xo[4], ko[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { xo[i] = x[i]; ko[i] = k[i]; }
    rk4_step_rolled<df64>(a, x, k, dl);
    n += 1;
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) fin = fin && isfinite(x[i].hi) && isfinite(x[i].lo) && isfinite(k[i].hi) && isfinite(k[i].lo);
    if (!fin) return kError;
    const df64 s0 = xo[2] - hp, s1 = x[2] - hp;
    // the plane is crossed when theta - pi/2 changes sign (or reaches 0), not starting on it
    if (s0.hi != 0.f && ((s0.hi > 0.f) != (s1.hi > 0.f) || s1.hi == 0.f)) {
        crossings += 1;
        // far from [r_in, r_out] the crossing cannot hit the disk: no refinement (as in
        // disk_step; a step changes r by at most ~eps r)
        const float grow = 1.f + 4.f * p.f.eps + 0.05f;
        const float r0 = xf[1], r1 = x[1].hi + x[1].lo;
        if (fmaxf(r0, r1) * grow < (float)d.r_in || fminf(r0, r1) > (float)d.r_out * grow) {
            if (crossings >= d.max_cross) return kDiskNone;
            const float r = r1;
            if (r < p.f.r_stop) return kCaptured;
            if (r > p.f.r_esc) return kEscaped;
            if (n >= p.max_steps) return kTruncated;
            return -1;
        }
        df64 xc[4], kc[4];
        disk_crossing_df(a, xo, ko, dl, x[2], xc, kc);
        const double rc = (double)xc[1];
        if (rc >= d.r_in && rc <= d.r_out) {
            double xd[4], kd[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { xd[i] = (double)xc[i]; kd[i] = (double)kc[i]; }
            KSPoint<double> P;
            ks_point<double>(p.a, rc, xd[2], P);
            double u[4], kcov[4];
            if (analytic_velocity<double>(p.a, 0.0, P, u) < 0) return kError;
            ks_lower(P, kd, kcov);
            const double g = kcov[0] * u[0] + kcov[1] * u[1] + kcov[2] * u[2] + kcov[3] * u[3];
            if (!(g > 0.0)) return kError;
            ratio = 1.0 / g;
            inten = ratio * ratio * ratio * ratio * pow(rc, -d.q);
            return kDiskHit;
        }
        if (crossings >= d.max_cross) return kDiskNone;
    }
    const float r = x[1].hi + x[1].lo;
    if (r < p.f.r_stop) return kCaptured;
    if (r > p.f.r_esc) return kEscaped;
    if (n >= p.max_steps) return kTruncated;
    return -1;
}

// Persistent over the fallback list (ray id -> d.list[id], -1 entries skipped), one ray per
// lane, refilled from the counter; outputs and statistics as k_disk_fp64.
__global__ void __launch_bounds__(128, 4) k_disk_df(const Params p, const DiskArgs d, unsigned long long* counter,
                                                    unsigned long long* stats) {
    const df64 a(p.f.a_p.x, p.f.a_p.y);
    df64 x[4], k[4];
    double ratio = 0.0, inten = 0.0;
    int n = 0, crossings = 0, pix = 0;
    long long id = -1;
    bool drained = false;
    unsigned long long c_rays = 0, c_steps = 0, c_trunc = 0, c_err = 0;
    for (;;) {
        const long long nid = warp_fetch(counter, p.n_rays, id < 0, drained);
        const int npix = nid >= 0 ? (d.list ? d.list[nid] : (int)nid) : -1;
        if (id < 0 && npix >= 0) {
            id = nid;
            pix = npix;
            const int row = pix / p.nx, col = pix % p.nx;
            double xd[4], kd[4];
            camera_ray(p, p.amin + (col + 0.5) * p.da, p.bmin + (row + 0.5) * p.db, p.t_cam, xd, kd);
#pragma unroll
            for (int i = 0; i < 4; ++i) { x[i] = df64(xd[i]); k[i] = df64(kd[i]); }
            n = 0;
            crossings = 0;
            ratio = 0.0;
            inten = 0.0;
        }
        if (!__any_sync(0xffffffffu, id >= 0)) break;
        if (id >= 0) {
            const int st = disk_step_df(p, d, a, x, k, n, crossings, ratio, inten);
            if (st >= 0) {
                const bool hit = st == kDiskHit;
                d.ratio[pix] = hit ? ratio : 0.0;
                d.inten[pix] = hit ? inten : 0.0;
                d.order[pix] = hit ? crossings : 0;
                if (d.status) d.status[pix] = st;
                if (d.steps) d.steps[pix] = n;
                c_rays += 1;
                c_steps += (unsigned long long)n;
                c_trunc += (st == kTruncated);
                c_err += (st == kError);
                id = -1;
            }
        }
    }
    warp_add_stats(stats, c_rays, c_steps, c_steps, c_trunc, c_err);
}

}  // namespace raptor
