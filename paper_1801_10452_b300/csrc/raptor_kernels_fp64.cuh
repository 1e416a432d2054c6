// raptor_kernels_fp64.cuh -- persistent FP64 ray-tracing kernel, single-ray trace kernel and
// the deterministic flux reduction.
#pragma once

#include "raptor_physics.cuh"
#include "raptor_grid.cuh"

namespace raptor {

constexpr unsigned kFlagK2Exact = 0x1u;
constexpr unsigned kFlagLinearR = 0x2u;
constexpr unsigned kFlagInnerDf64 = 0x4u;
constexpr unsigned kFlagVerlet = 0x8u;         // velocity Verlet (sec. 2.2.2) instead of RK4
constexpr unsigned kFlagVerletReeval = 0x10u;  // ... with the re-evaluation of Eqs. 18-19
constexpr unsigned kFlagForwardRT = 0x20u;     // forward formal-solution transfer (FP64 path)
constexpr int kForwardCap = 2048;              // forward scheme: transfer records per ray
constexpr int kForwardMaxFreq = 4;             // forward scheme: frequencies per call

enum : int { kEscaped = 0, kCaptured = 1, kThick = 2, kTruncated = 3, kError = 4, kDiskHit = 5, kDiskNone = 6 };

// Per-kernel profiling slots (raptor_profile_read).
enum : int { kProfRenderFp64 = 0, kProfMixedA = 1, kProfMixedB = 2, kProfMixedC = 3, kProfReduce = 4, kProfTrace = 5,
             kProfLoad = 6, kProfPeak = 7, kProfSurrogate = 8, kProfTrain = 9, kProfSurrogateMlp = 10,
             kProfDisk = 11, kProfMixedBLong = 12, kProfSlots = 13 };

// Stats slots (device unsigned long long[kNumStats]).
enum : int { kStatRays = 0, kStatSteps = 1, kStatFp64Steps = 2, kStatTrunc = 3, kStatErr = 4, kStatFallback = 5,
             kStatReentry = 6, kStatClamp = 7, kStatFp64Long = 8, kStatFp32In = 9, kStatFp32Out = 10,
             kNumStats = 16 };

template <int NF>
struct RayD {
    double x[4], k[4];
    double f[4];  // carried derivative of the Verlet integrator (unused by RK4)
    double I[NF], tau[NF];
    int n;
    int snap;
    int ns;       // forward scheme: transfer records of this ray
};

// Forward formal solution (sec. 3, Eq. 34 with constant coefficients over each step): the
// thread's records of this ray, (dtau, S (1 - e^{-dtau}) / g^3) in step order, combined from
// the far end: I <- I e^{-dtau} + contribution, towards the camera.
__device__ __forceinline__ double forward_intensity(const Params& p, long long tid, int ns, int f) {
    double I = 0.0;
    for (int q = ns - 1; q >= 0; --q) {
        const double2 rec = p.fwd[((long long)q * p.nf + f) * p.fwd_stride + tid];
        I = I * exp(-rec.x) + rec.y;
    }
    return I;
}

// One FP64 step of a ray: adaptive step, RK4 (VERLET = false) or velocity Verlet,
// termination, transfer sample.  Returns the termination code or -1 to continue.
// dl_out / g_out feed the trace recorder.
template <int NF, bool VERLET = false>
__device__ __forceinline__ int step_fp64(const Params& p, RayD<NF>& R, double& dl_out, double& g_out) {
    const double dl = step_size<double>(p.eps, (p.flags & kFlagLinearR) != 0, R.x, R.k);
    if constexpr (VERLET) verlet_step<double>(p.a, R.x, R.k, R.f, dl, (p.flags & kFlagVerletReeval) != 0);
    else rk4_step<double>(p.a, R.x, R.k, dl);
    R.n += 1;
    dl_out = dl;
    g_out = 0.0;
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) fin = fin && isfinite(R.x[i]) && isfinite(R.k[i]);
    if (!fin) return kError;
    if (R.x[1] < p.r_stop) return kCaptured;
    if (R.x[1] > p.r_esc) return kEscaped;
    double ne, the, B, g, sinb;
    const int ok = plasma_sample<double>(p, R.x, R.k, R.snap, ne, the, B, g, sinb);
    if (ok < 0) return kError;
    if (ok > 0) {
        g_out = g;
        const double dlcm = dl * p.Lcm;
        const bool k2x = (p.flags & kFlagK2Exact) != 0;
        const bool fwd = (p.flags & kFlagForwardRT) != 0;
        if (fwd && R.ns >= p.fwd_cap) return kError;  // this ray's records are full
        const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f < p.nf) {
                double j, S;
                synchrotron<double>(g * p.nu[f], ne, the, B, sinb, k2x, j, S, 1.0, p.the_min);
                if (fwd) {
                    double dtau = 0.0, c = 0.0;
                    if (j > 0.0 && S > 0.0) {
                        dtau = j / S * g * dlcm;
                        c = S * (-expm1(-dtau)) / (g * g * g);
                    }
                    p.fwd[((long long)R.ns * p.nf + f) * p.fwd_stride + tid] = make_double2(dtau, c);
                    R.tau[f] += dtau;
                } else {
                    rt_update<double, double>(j, S, g, dlcm, R.I[f], R.tau[f]);
                }
            }
        }
        if (fwd) R.ns += 1;
    }
    double tmin = R.tau[0];
#pragma unroll
    for (int f = 1; f < NF; ++f)
        if (f < p.nf) tmin = fmin(tmin, R.tau[f]);
    if (tmin > p.tau_cut) return kThick;
    if (R.n >= p.max_steps) return kTruncated;
    return -1;
}

// Ray id -> (frame, pixel, row, col); initial state (and, for Verlet, the derivative there).
template <int NF, bool VERLET = false>
__device__ __forceinline__ void init_ray(const Params& p, long long id, RayD<NF>& R, int& frame, int& pix) {
    frame = (int)(id / p.n_pix);
    pix = (int)(id - (long long)frame * p.n_pix);
    const int row = p.row0 + pix / p.nx, col = pix % p.nx;
    const double alpha = p.amin + (col + 0.5) * p.da;
    const double beta = p.bmin + (row + 0.5) * p.db;
    const double tc = p.t_frames ? p.t_frames[frame] : p.t_cam;
    camera_ray(p, alpha, beta, tc, R.x, R.k);
    if constexpr (VERLET) geodesic_force<double>(p.a, R.x[1], R.x[2], R.k, R.f);
#pragma unroll
    for (int f = 0; f < NF; ++f) { R.I[f] = 0.0; R.tau[f] = 0.0; }
    R.n = 0;
    R.ns = 0;
    R.snap = p.lc_fast ? p.frame_snap0 + frame : p.snap;
}

template <int NF>
__device__ __forceinline__ void write_ray(const Params& p, int frame, int pix, const double* I, int n, int status) {
    const long long plane = (long long)p.n_rows * p.nx;
#pragma unroll
    for (int f = 0; f < NF; ++f)
        if (f < p.nf) p.image[((long long)frame * p.nf_total + p.f_off + f) * plane + pix] = I[f] * p.i_unscale * p.pix_jy;
    if (p.steps_out) p.steps_out[pix] = n;
    if (p.status_out) p.status_out[pix] = status;
}

__device__ __forceinline__ void warp_add_stats(unsigned long long* stats, unsigned long long rays, unsigned long long steps,
                                               unsigned long long s64, unsigned long long trunc, unsigned long long err) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rays += __shfl_down_sync(0xffffffffu, rays, o);
        steps += __shfl_down_sync(0xffffffffu, steps, o);
        s64 += __shfl_down_sync(0xffffffffu, s64, o);
        trunc += __shfl_down_sync(0xffffffffu, trunc, o);
        err += __shfl_down_sync(0xffffffffu, err, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&stats[kStatRays], rays);
        atomicAdd(&stats[kStatSteps], steps);
        if (s64) atomicAdd(&stats[kStatFp64Steps], s64);
        if (trunc) atomicAdd(&stats[kStatTrunc], trunc);
        if (err) atomicAdd(&stats[kStatErr], err);
    }
}

// Warp-aggregated fetch from the global ray counter: lanes whose `need` is set receive
// consecutive ray ids (or -1 once the queue is drained).  Returns false once drained.
__device__ __forceinline__ long long warp_fetch(unsigned long long* counter, long long n_total, bool need, bool& drained) {
    const unsigned m = __ballot_sync(0xffffffffu, need && !drained);
    long long id = -1;
    if (m) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (base + __popc(m) >= (unsigned long long)n_total) drained = true;
        if (need) {
            const long long cand = (long long)base + __popc(m & ((1u << lane) - 1u));
            if (cand < n_total) id = cand;
        }
    }
    return id;
}

// Persistent FP64 kernel: each warp keeps 32 rays in flight and refills a lane from the
// global work counter as soon as its ray terminates (per-warp compaction of uneven ray
// lengths).  Blocks must be a multiple of 32 threads.  VERLET: the velocity-Verlet integrator.
template <int NF, bool VERLET = false>
__global__ void __launch_bounds__(128) k_render_fp64(const Params p, unsigned long long* counter, unsigned long long* stats) {
    RayD<NF> R;
    long long id = -1;
    int frame = 0, pix = 0;
    bool drained = false;
    unsigned long long c_rays = 0, c_steps = 0, c_trunc = 0, c_err = 0;
    for (;;) {
        const long long nid = warp_fetch(counter, p.n_rays, id < 0, drained);
        if (id < 0 && nid >= 0) {
            id = nid;
            init_ray<NF, VERLET>(p, id, R, frame, pix);
        }
        if (!__any_sync(0xffffffffu, id >= 0)) break;
        if (id >= 0) {
            double dl, g;
            const int st = step_fp64<NF, VERLET>(p, R, dl, g);
            if (st >= 0) {
                if (p.flags & kFlagForwardRT) {
                    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        if (f < p.nf) R.I[f] = forward_intensity(p, tid, R.ns, f);
                }
                write_ray<NF>(p, frame, pix, R.I, R.n, st);
                c_rays += 1;
                c_steps += (unsigned long long)R.n;
                c_trunc += (st == kTruncated);
                c_err += (st == kError);
                id = -1;
            }
        }
    }
    warp_add_stats(stats, c_rays, c_steps, c_steps, c_trunc, c_err);
}

// ------------------------------------------------------------------------------------
// Thin-disk line emitter (sec. 4.2.1): an opaque equatorial disk between r_in and r_out on
// circular Keplerian orbits (Omega = 1/(r^{3/2} + a)), emission ~ r^{-q}, no absorption.  Each
// ray is integrated with the FP64 step of k_render_fp64 until it crosses theta = pi/2 inside
// the disk (a hit), is captured or escapes, or has crossed the plane max_cross times.  The
// crossing point: Newton's iteration on the length h of one RK4 step from the state before
// the crossing step, h <- h - (theta(h) - pi/2) / k^theta(h), from the linear estimate, a
// fixed four iterations, then the step of the final length.  At a hit: E_obs/E_em = 1 / g,
// g = k.u (Eq. 30), and the line intensity I = (E_obs/E_em)^4 r^{-q}.
// ------------------------------------------------------------------------------------
struct DiskArgs {
    double r_in, r_out, q;
    int max_cross;
    double* ratio;    // [n_pix] E_obs/E_em (0: no hit)
    double* inten;    // [n_pix] line intensity (0: no hit)
    int* order;       // [n_pix] crossing number of the hit (0: no hit)
    int* status;      // [n_pix] or nullptr
    int* steps;       // [n_pix] or nullptr
    const int* list;  // nullptr: ray id = pixel; else the pixel of each ray id (-1: none)
};

__device__ __forceinline__ void disk_crossing(double a, const double x0[4], const double k0[4], double dl, double th1,
                                              double xc[4], double kc[4], double* h_out = nullptr) {
    const double half_pi = 0.5 * kPi;
    double h = dl * (half_pi - x0[2]) / (th1 - x0[2]);
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) { xc[i] = x0[i]; kc[i] = k0[i]; }
        rk4_step<double>(a, xc, kc, h);
        if (!(fabs(kc[2]) > 0.0)) break;
        h -= (xc[2] - half_pi) / kc[2];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) { xc[i] = x0[i]; kc[i] = k0[i]; }
    rk4_step<double>(a, xc, kc, h);
    if (h_out) *h_out = h;
}

// One step of a disk ray: returns the termination code or -1; on a hit fills ratio, I.
__device__ __forceinline__ int disk_step(const Params& p, const DiskArgs& d, double x[4], double k[4], int& n,
                                         int& crossings, double& ratio, double& inten) {
    const double half_pi = 0.5 * kPi;
    const double dl = step_size<double>(p.eps, (p.flags & kFlagLinearR) != 0, x, k);
    double xo[4], ko[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { xo[i] = x[i]; ko[i] = k[i]; }
    rk4_step<double>(p.a, x, k, dl);
    n += 1;
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) fin = fin && isfinite(x[i]) && isfinite(k[i]);
    if (!fin) return kError;
    if ((xo[2] - half_pi) * (x[2] - half_pi) <= 0.0 && xo[2] != half_pi) {
        crossings += 1;
        // A step changes r by at most ~eps r (the step rule), so the crossing's radius lies
        // within that of the step's end radii: a crossing far outside [r_in, r_out] cannot
        // hit the disk and skips the refinement (same hits, same values).
        const double grow = 1.0 + 4.0 * p.eps + 0.05;
        const bool near = fmax(xo[1], x[1]) * grow >= d.r_in && fmin(xo[1], x[1]) <= d.r_out * grow;
        double xc[4], kc[4];
        if (near) disk_crossing(p.a, xo, ko, dl, x[2], xc, kc);
        const double rc = near ? xc[1] : -1.0;
        if (near && rc >= d.r_in && rc <= d.r_out) {
            KSPoint<double> P;
            ks_point<double>(p.a, rc, xc[2], P);
            double u[4], kcov[4];
            if (analytic_velocity<double>(p.a, 0.0, P, u) < 0) return kError;  // Keplerian at every r
            ks_lower(P, kc, kcov);
            const double g = kcov[0] * u[0] + kcov[1] * u[1] + kcov[2] * u[2] + kcov[3] * u[3];
            if (!(g > 0.0)) return kError;
            ratio = 1.0 / g;
            inten = ratio * ratio * ratio * ratio * pow(rc, -d.q);
            return kDiskHit;
        }
        if (crossings >= d.max_cross) return kDiskNone;
    }
    if (x[1] < p.r_stop) return kCaptured;
    if (x[1] > p.r_esc) return kEscaped;
    if (n >= p.max_steps) return kTruncated;
    return -1;
}

// Persistent: each warp keeps 32 rays in flight and refills lanes from the counter (a ray
// id is a pixel, or indexes d.list, whose -1 entries are skipped).
__global__ void __launch_bounds__(128) k_disk_fp64(const Params p, const DiskArgs d, unsigned long long* counter,
                                                   unsigned long long* stats) {
    double x[4], k[4], ratio = 0.0, inten = 0.0;
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
            camera_ray(p, p.amin + (col + 0.5) * p.da, p.bmin + (row + 0.5) * p.db, p.t_cam, x, k);
            n = 0;
            crossings = 0;
            ratio = 0.0;
            inten = 0.0;
        }
        if (!__any_sync(0xffffffffu, id >= 0)) break;
        if (id >= 0) {
            const int st = disk_step(p, d, x, k, n, crossings, ratio, inten);
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

// Line spectrum of the disk image: pixels whose hit has crossing number `sel_order` (0: any)
// add I * pixel area to bin floor((ratio - x_min) / dx) when it lies in [0, n_bins).  The
// weights are summed as 64-bit fixed-point integers (w * 2^scale_log2, rounded), so the
// spectrum does not depend on the order of the atomic additions.
__global__ void __launch_bounds__(256) k_disk_profile(const double* __restrict__ ratio, const double* __restrict__ inten,
                                                      const int* __restrict__ order, long long n, int sel_order,
                                                      double x_min, double dx, int n_bins, double pix_area,
                                                      double scale, unsigned long long* __restrict__ hist) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int o = order[i];
        if (o == 0 || (sel_order > 0 && o != sel_order)) continue;
        const double b = floor((ratio[i] - x_min) / dx);
        if (!(b >= 0.0 && b < (double)n_bins)) continue;
        atomicAdd(&hist[(int)b], (unsigned long long)llrint(inten[i] * pix_area * scale));
    }
}

// Single-ray trace with per-step records (same arithmetic as k_render_fp64).
template <int NF, bool VERLET = false>
__global__ void k_trace_fp64(const Params p, double alpha, double beta, double t_cam, int max_rec, double* rec, int* out_n,
                             int* out_status, double* out_I) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    RayD<NF> R;
    camera_ray(p, alpha, beta, t_cam, R.x, R.k);
    if constexpr (VERLET) geodesic_force<double>(p.a, R.x[1], R.x[2], R.k, R.f);
#pragma unroll
    for (int f = 0; f < NF; ++f) { R.I[f] = 0.0; R.tau[f] = 0.0; }
    R.n = 0;
    R.ns = 0;
    R.snap = p.snap;
    int st = -1;
    while (st < 0) {
        double dl, g;
        st = step_fp64<NF, VERLET>(p, R, dl, g);
        if (R.n <= max_rec) {
            double* T = rec + (long long)(R.n - 1) * 12;
            for (int i = 0; i < 4; ++i) { T[i] = R.x[i]; T[4 + i] = R.k[i]; }
            T[8] = dl;
            T[9] = g;
            T[10] = R.I[0];
            T[11] = R.tau[0];
        }
    }
    if (p.flags & kFlagForwardRT)
        for (int f = 0; f < NF; ++f)
            if (f < p.nf) R.I[f] = forward_intensity(p, 0, R.ns, f);
    *out_n = R.n;
    *out_status = st;
    for (int f = 0; f < NF; ++f)
        if (f < p.nf) out_I[f] = R.I[f];
}

// Deterministic two-pass sum of `planes` arrays of `len` doubles: pass 1 (grid chunks x
// planes) writes fixed-order partial sums, pass 2 (one block per plane) adds them in order.
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum_fixed(double v) {
    __shared__ double sh[kRedThreads];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_partial(const double* __restrict__ data, long long len, int chunks,
                                                                double* __restrict__ partial) {
    const int plane = blockIdx.y, c = blockIdx.x;
    const long long per = (len + chunks - 1) / chunks;
    const long long b = (long long)c * per, e = min(len, b + per);
    const double* d = data + (long long)plane * len;
    double acc = 0.0;
    for (long long i = b + threadIdx.x; i < e; i += kRedThreads) acc += d[i];
    const double s = block_sum_fixed(acc);
    if (threadIdx.x == 0) partial[(long long)plane * chunks + c] = s;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double* __restrict__ partial, int chunks, double* __restrict__ out) {
    const int plane = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < chunks; i += kRedThreads) acc += partial[(long long)plane * chunks + i];
    const double s = block_sum_fixed(acc);
    if (threadIdx.x == 0) out[plane] = s;
}

// FMA-chain microbenchmark: 16 independent dependent chains per thread.
// Self-check of the FP32 code paths' own primitives.  Per primitive, the largest distance in
// ulps (of the float bit patterns) from a reference rounded to float: rcp_nr and sqrt_nr
// against the correctly rounded 1/v and sqrtf, cbrt_nr against the FP64 cube root rounded
// to float, x_over_expm1f and one_minus_exp_over_f against FP64 x / expm1(x) and
// -expm1(-d) / d rounded to float.  Inputs: m 2^e, m from a Weyl sequence in [1, 2), e in
// [-100, 100] (both signs for the reciprocal); x and d = m 2^e with e in [-40, 4], and
// 1 + 35 m for the series' other branch.
__global__ void k_check_fp32_math(long long n, unsigned int* max_ulp) {
    unsigned int worst[5] = {0, 0, 0, 0, 0};
    auto ulps = [](float a, float b) {
        const int d = __float_as_int(a) - __float_as_int(b);
        return (unsigned int)(d < 0 ? -d : d);
    };
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float m = 1.0f + (float)((i * 0x9E3779B9ull) & 0xFFFFFF) * (1.0f / 16777216.0f);
        const int e = (int)(i % 201) - 100;
        const float v = ldexpf(m, e);
        const float vs = (i & 1) ? -v : v;
        worst[0] = max(worst[0], ulps(rcp_nr(vs), 1.0f / vs));
        worst[1] = max(worst[1], ulps(sqrt_nr(v), sqrtf(v)));
        worst[2] = max(worst[2], ulps(cbrt_nr(v), (float)cbrt((double)v)));
        const float x = (i % 3 == 0) ? 1.0f + 35.0f * (m - 1.0f) : ldexpf(m, (int)(i % 45) - 40);
        worst[3] = max(worst[3], ulps(x_over_expm1f(x), (float)((double)x / expm1((double)x))));
        worst[4] = max(worst[4], ulps(one_minus_exp_over_f(x), (float)(-expm1(-(double)x) / (double)x)));
    }
    for (int k = 0; k < 5; ++k) atomicMax(&max_ulp[k], worst[k]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T seed) {
    T a[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] = seed + T(threadIdx.x + c) * T(1e-7);
    const T m = T(0.9999999), d = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 16; ++c) a[c] = fma(a[c], m, d);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 16; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace raptor
