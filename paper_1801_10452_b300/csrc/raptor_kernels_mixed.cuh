// raptor_kernels_mixed.cuh -- mixed FP32/FP64 integration as a three-phase wavefront.
//
// B300 executes FP64 at a small fraction of its FP32 rate, and a warp that holds one FP64
// ray pays the FP64 price for all 32 lanes.  So rays are sorted by precision through device
// queues instead of switching precision per lane:
//   phase A (FP32, persistent): fresh camera rays, integrated while r >= r_fp64 and away
//     from radial turning points (|k^r| >= turn_kr |k^t|); a ray entering that region is
//     pushed to the FP64 queue with its state promoted to FP64, and the lane refills.
//   phase B (FP64, persistent): rays from the FP64 queue, geodesic steps in FP64 (their
//     transfer samples in FP32) until they terminate or leave the region; leavers are
//     pushed to an FP32 queue.
//   phase C (FP32, persistent): rays from the FP32 queues, integrated to termination (an
//     outgoing photon has no further radial turning point; re-entries are counted).
// Rays near the critical curve orbit the photon sphere and need ~10^3 sequential FP64
// steps: their chain of steps, not the total work, bounds the frame.  They are selected
// first (phase A1), and their FP64 phase runs on a second stream (B-long) while the other
// rays go through phases A2, B and C on the first.  The other rays' FP64 passes end in a
// ragged tail each; after the first few passes, the rays still in the FP64 region move to
// the second stream (B-tail, after B-long) and the first stream goes on with phase C.
// Every launch works on a range of a queue fixed before it starts (a snapshot of the push
// counter, or a queue completed earlier in stream order), so no kernel waits on another.
// The optical depth of a frequency beyond 10 is accumulated with a 48-bit significand
// (compensated float pair), so the per-step loops of all phases issue no FP64 instruction
// for the transfer: on B300 one FP64 compare or conversion occupies the FP64 pipe for as
// long as ~70 FP32 instructions.
#pragma once

#include "raptor_kernels_fp64.cuh"
#include "raptor_surrogate.cuh"
#include "raptor_df64.cuh"

namespace raptor {

struct RayQueue {
    float2* xk;       // [8][cap]: x^0..x^3, k^0..k^3 as unevaluated float pairs (hi, lo)
    double* I;        // [nf_cap][cap]
    double* tau;      // [nf_cap][cap]
    int* n;           // [cap] steps so far
    long long* id;    // [cap] ray id
};

struct MixedQueues {
    RayQueue q64;         // phase A -> FP64 (A1's rays first, then A2's)
    RayQueue q64b, q64c;  // re-queue targets of the FP64 passes (alternating)
    RayQueue q32;         // FP64 passes -> phase C
    RayQueue q32l;        // B-long -> phase C (its own queue: B-long runs concurrently with C)
    size_t cap = 0;
    int nf_cap = 0;
};

// Counter slots in the context's device counter array (kNumCounters entries).
enum : int {
    kCntListCrit = 0,    // length of the near-critical id list (phase A1)
    kCntListRest = 1,    // length of the other id list (phase A2)
    kCntFreshCrit = 2,   // fetch counters of the two lists
    kCntFreshRest = 3,
    kCntPush64 = 4,      // q64 push counter of A2 (entries from the bottom of q64)
    kCntPush64C = 5,     // q64 push counter of A1 (entries from cap - cnt[kCntListCrit] up)
    kCntPush32L = 7,     // q32l push counter
    kCntPush32 = 8,      // q32 push counter
    kCntFetch32 = 9,
    kCntFetch32L = 10,
    kCntTailFetch = 11,  // B-tail's fetch counter
    kCntPassFetch = 16,  // per pass of the first stream: fetch counters
    kCntPassOut = 24,    // per pass of the first stream: re-queue push counters
    kCntLPassFetch = 32, // per pass of the second stream (near-critical rays): fetch counters
    kCntLPassOut = 40,   // per pass of the second stream: re-queue push counters
    kMaxPasses = 8,
    kNumCounters = 48
};

// Input, outputs and counter slots of one launch of the mixed kernels.
struct PhaseIO {
    const int* fresh;     // phase A: ray ids to start (nullptr: rays come from `in`)
    RayQueue in;          // queued input
    RayQueue push;        // phase A: FP64 queue; FP64 launches: leavers (FP32 queue)
    RayQueue requeue;     // FP64 passes: rays still in the region after `budget` steps
    int fetch, total;     // fetch counter slot; slot holding the number of input entries
    int push_cnt;         // push counter slot of `push` (phase C: -1, re-entries are counted)
    int requeue_cnt;      // push counter slot of `requeue` (-1: no re-queue)
    int budget;           // FP64 launches: steps per ray in this launch
    int in_exact;         // FP64 launches: `in` holds re-queued states in the exact format
    int push_top = -1;    // counter slot c: `push` entries start at cap - cnt[c] (-1: at 0)
    int in_top = -1;      // the same for `in`
    int requeue_top = -1; // and for `requeue`
    int long_lane = 0;    // FP64 launches on the second stream: their FP64 steps also go to kStatFp64Long
};

inline cudaError_t alloc_queue(RayQueue& q, size_t cap, int nf) {
    cudaError_t e = cudaMalloc((void**)&q.xk, sizeof(float2) * 8 * cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&q.I, sizeof(double) * nf * cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&q.tau, sizeof(double) * nf * cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&q.n, sizeof(int) * cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&q.id, sizeof(long long) * cap);
    return e;
}

inline void free_queue(RayQueue& q) {
    cudaFree(q.xk);
    cudaFree(q.I);
    cudaFree(q.tau);
    cudaFree(q.n);
    cudaFree(q.id);
    q = RayQueue{nullptr, nullptr, nullptr, nullptr, nullptr};
}

inline void free_mixed_queues(MixedQueues& m) {
    RayQueue* all[] = {&m.q64, &m.q64b, &m.q64c, &m.q32, &m.q32l};
    for (RayQueue* q : all) free_queue(*q);
    m.cap = 0;
    m.nf_cap = 0;
}

inline cudaError_t alloc_mixed_queues(MixedQueues& m, size_t cap, int nf) {
    RayQueue* all[] = {&m.q64, &m.q64b, &m.q64c, &m.q32, &m.q32l};
    for (RayQueue* q : all) *q = RayQueue{nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (RayQueue* q : all)
        if (e == cudaSuccess) e = alloc_queue(*q, cap, nf);
    if (e == cudaSuccess) {
        m.cap = cap;
        m.nf_cap = nf;
    } else {
        free_mixed_queues(m);
    }
    return e;
}

// Warp-aggregated push: lanes with `push` set receive consecutive slots.
__device__ __forceinline__ long long warp_push_slot(unsigned long long* count, bool push) {
    const unsigned m = __ballot_sync(0xffffffffu, push);
    long long slot = -1;
    if (m) {
        const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (push) slot = (long long)base + __popc(m & ((1u << lane) - 1u));
    }
    return slot;
}

template <typename T>
__device__ __forceinline__ bool in_fp64_region(const Params& p, const T x[4], const T k[4]) {
    return x[1] < RAPTOR_P(T, r_fp64) || fabs(k[1]) < RAPTOR_P(T, turn_kr) * fabs(k[0]);
}

template <int NF>
struct RayF {
    float x[4], k[4];
    float xl[4], kl[4];  // low parts of the compensated state (rk4_step_comp)
    float I[NF], tau[NF];
    df64 tau_hi[NF];  // optical depth beyond 10, compensated sum (zero while unused)
    int n, snap;
};

// Split a queued optical depth into the float part (<= 10) and the compensated high part.
__device__ __forceinline__ void split_f(double v, float& hi, float& lo) {
    hi = float(v);
    lo = float(v - double(hi));
}

__device__ __forceinline__ void tau_split(double t, float& lo, df64& hi) {
    if (t > 10.0) { lo = 0.f; hi = df64(t); }
    else { lo = float(t); hi = df64(0.f, 0.f); }
}

// FP32 transfer sample at (x, k) after a step of length dl (Eqs. 30, 34-36, 41-44).
// Intensities are carried scaled by kIScale = 2^100: the emissivity's exponential tail
// reaches ~1e-60 cgs, far below FP32's smallest normal number.  The per-step increment of
// the formal solution, exp(-tau) S (1 - exp(-dtau)) / g^3, is written as
// exp(-tau) j dl L F(dtau) / g^2 with F(x) = (1 - exp(-x)) / x, so no factor underflows.
// A frequency's optical depth moves to the compensated accumulator once above 10.
constexpr float kIScale = 1.2676506002282294e30f;      // 2^100
constexpr double kIUnscale = 7.888609052210118e-31;    // 2^-100

// (sn, cs): sin and cos of x[2], when the caller has them (sn > 1: compute them here).
// r_lo: the radius's low part (the radius is x[1] + r_lo): the analytic flow changes from
// Keplerian to free fall at r_isco, and that branch is decided on the radius to ~48 bits
// against r_isco as a float pair, as the FP64 path decides it (a sample within FP32
// rounding of r_isco would otherwise take the other branch).
template <int NF, typename TI>
__device__ __forceinline__ int rt_sample_fp32(const Params& p, const float x[4], const float k[4], float dl, int snap,
                                              TI* I, float* tau, df64* tau_hi, float r_lo, float sn = 2.f, float cs = 0.f) {
    float ne, the, B, g, sinb;
    if (sn > 1.f) sc(x[2], &sn, &cs);
    const int kepler = ((x[1] - p.f.r_isco_p.x) + (r_lo - p.f.r_isco_p.y)) >= 0.f ? 1 : 0;
    const int ok = plasma_sample_sc<float>(p, x, k, sn, cs, snap, ne, the, B, g, sinb, kepler);
    if (ok <= 0) return ok;
    const float dlcm = dl * p.f.Lcm;
    const float gdl_unscaled = g * dlcm * float(kIUnscale);
    const float ig2 = rcp_nr(g * g);
    const bool k2x = (p.flags & kFlagK2Exact) != 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f < p.nf) {
            float j, S;
            synchrotron<float>(g * p.f.nu[f], ne, the, B, sinb, k2x, j, S, kIScale, p.f.the_min);
            if (j > 0.f && S > 0.f) {
                const float dtau = j * rcp_nr(S) * gdl_unscaled;
                const float F = one_minus_exp_over_f(dtau);
                const float tau_now = tau[f] + tau_hi[f].hi;
                I[f] += TI(expf(-tau_now) * j * dlcm * F * ig2);
                if (tau_hi[f].hi > 0.f || tau[f] + dtau > 10.f) tau_hi[f] = tau_hi[f] + df64(dtau, 0.f);
                else tau[f] += dtau;
            }
        }
    }
    return 1;
}

template <int NF>
__device__ __forceinline__ int thick_or_capped(const Params& p, const float* tau, const df64* tau_hi, int n) {
    float tmin = tau[0] + (tau_hi[0].hi + tau_hi[0].lo);
#pragma unroll
    for (int f = 1; f < NF; ++f)
        if (f < p.nf) tmin = fminf(tmin, tau[f] + (tau_hi[f].hi + tau_hi[f].lo));
    if (tmin > p.f.tau_cut) return kThick;
    if (n >= p.max_steps) return kTruncated;
    return -1;
}

// One FP32 step (same scheme as step_fp64).  Returns termination code or -1.
template <int NF>
__device__ __forceinline__ int step_fp32(const Params& p, RayF<NF>& R) {
    const float dl = step_size<float>(p.f.eps, (p.flags & kFlagLinearR) != 0, R.x, R.k);
    float sn, cs;
    rk4_step_comp(p.f.a, R.x, R.xl, R.k, R.kl, dl, &sn, &cs);
    R.n += 1;
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) fin = fin && isfinite(R.x[i]) && isfinite(R.k[i]);
    if (!fin) return kError;
    if (R.x[1] < p.f.r_stop) return kCaptured;
    if (R.x[1] > p.f.r_esc) return kEscaped;
    if (p.r_exit_f > 0.f && R.x[1] > p.r_exit_f && R.k[1] > 0.f) return kEscaped;  // surrogate path only
    if (rt_sample_fp32<NF, float>(p, R.x, R.k, dl, R.snap, R.I, R.tau, R.tau_hi, R.xl[1], sn, cs) < 0) return kError;
    return thick_or_capped<NF>(p, R.tau, R.tau_hi, R.n);
}

// Mixed FP64 phase: the geodesic step in FP64 (S = double) or in double-float arithmetic
// on the FP32 pipe (S = df64, RAPTOR_FLAG_INNER_DF64), its transfer sample in FP32 (optical
// depth beyond 10 in the compensated accumulator).
template <typename S>
struct StateT;
// Queue slots hold float pairs.  A state handed from the FP64 phase to another FP64 pass is
// stored exactly: the double's bits in the slot (from_exact / to_exact), so re-queueing
// never rounds and the result of a ray does not depend on how often it is re-queued; a
// double-float state is exact as a pair anyway.
template <>
struct StateT<double> {
    static __device__ __forceinline__ double from(double d) { return d; }
    static __device__ __forceinline__ double from2(float2 v) { return double(v.x) + double(v.y); }
    static __device__ __forceinline__ float2 to2(double v) {
        const float hi = float(v);
        return make_float2(hi, float(v - double(hi)));
    }
    static __device__ __forceinline__ double from_exact(float2 v) {
        return __hiloint2double(__float_as_int(v.y), __float_as_int(v.x));
    }
    static __device__ __forceinline__ float2 to_exact(double v) {
        return make_float2(__int_as_float(__double2loint(v)), __int_as_float(__double2hiint(v)));
    }
    static __device__ __forceinline__ float f(double v) { return (float)v; }
    static __device__ __forceinline__ bool finite(double v) { return isfinite(v); }
};
template <>
struct StateT<df64> {
    static __device__ __forceinline__ df64 from(double d) { return df64(d); }
    static __device__ __forceinline__ df64 from2(float2 v) { return df64(v.x, v.y); }
    static __device__ __forceinline__ float2 to2(df64 v) { return make_float2(v.hi, v.lo); }
    static __device__ __forceinline__ df64 from_exact(float2 v) { return df64(v.x, v.y); }
    static __device__ __forceinline__ float2 to_exact(df64 v) { return make_float2(v.hi, v.lo); }
    static __device__ __forceinline__ float f(df64 v) { return v.hi + v.lo; }
    static __device__ __forceinline__ bool finite(df64 v) { return isfinite(v.hi) && isfinite(v.lo); }
};

// Intensity accumulator of the FP64 phase: FP64 next to FP64 steps (one FP64 add per sample
// beside hundreds of FP64 step instructions), FP32 next to double-float steps, which issue
// no FP64 instruction at all.
template <typename S>
using AccI = typename std::conditional<std::is_same<S, double>::value, double, float>::type;

template <int NF, typename S = double>
struct RayM {
    S x[4], k[4];
    AccI<S> I[NF];
    float tau[NF];
    df64 tau_hi[NF];
    int n, snap;
};

template <int NF, typename S>
__device__ __forceinline__ int step_mixed64(const Params& p, RayM<NF, S>& R, S a) {
    float xf[4], kf[4];
    if constexpr (std::is_same<S, double>::value) {
        const double dl = step_size<double>(p.eps, (p.flags & kFlagLinearR) != 0, R.x, R.k);
        rk4_step<double>(p.a, R.x, R.k, dl);
        R.n += 1;
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) fin = fin && isfinite(R.x[i]) && isfinite(R.k[i]);
        if (!fin) return kError;
        if (R.x[1] < p.r_stop) return kCaptured;
        if (R.x[1] > p.r_esc) return kEscaped;
#pragma unroll
        for (int i = 0; i < 4; ++i) { xf[i] = float(R.x[i]); kf[i] = float(R.k[i]); }
        if (rt_sample_fp32<NF, double>(p, xf, kf, float(dl), R.snap, R.I, R.tau, R.tau_hi, float(R.x[1] - double(xf[1]))) < 0)
            return kError;
    } else {
        // step size from the FP32 view of the state (the rule is a heuristic; its value only
        // needs to be a smooth function of the state), RK4 in df64
#pragma unroll
        for (int i = 0; i < 4; ++i) { xf[i] = StateT<S>::f(R.x[i]); kf[i] = StateT<S>::f(R.k[i]); }
        const float dl = step_size<float>(p.f.eps, (p.flags & kFlagLinearR) != 0, xf, kf);
        rk4_step_rolled<S>(a, R.x, R.k, S(dl, 0.f));
        R.n += 1;
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) fin = fin && StateT<S>::finite(R.x[i]) && StateT<S>::finite(R.k[i]);
        if (!fin) return kError;
#pragma unroll
        for (int i = 0; i < 4; ++i) { xf[i] = StateT<S>::f(R.x[i]); kf[i] = StateT<S>::f(R.k[i]); }
        if (xf[1] < p.f.r_stop) return kCaptured;
        if (xf[1] > p.f.r_esc) return kEscaped;
        const float r_lo = (R.x[1].hi - xf[1]) + R.x[1].lo;  // the first difference is exact
        if (rt_sample_fp32<NF, float>(p, xf, kf, dl, R.snap, R.I, R.tau, R.tau_hi, r_lo) < 0) return kError;
    }
    return thick_or_capped<NF>(p, R.tau, R.tau_hi, R.n);
}

// Queue entry `slot`: the state as float pairs (FP32 phases store their compensated state as
// is; the FP64 phase splits FP64 values, which keeps 48 of their 53 bits, the precision of
// the double-float arithmetic), per-frequency I and tau in FP64, step count, ray id.
template <int NF, typename TI>
__device__ __forceinline__ void store_ray(const RayQueue& q, size_t cap, long long slot, long long id, const float2 x[4],
                                          const float2 k[4], const TI* I, const double* tau, int n, int nf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        q.xk[(size_t)i * cap + slot] = x[i];
        q.xk[(size_t)(4 + i) * cap + slot] = k[i];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
        if (f < nf) {
            q.I[(size_t)f * cap + slot] = double(I[f]);
            q.tau[(size_t)f * cap + slot] = tau[f];
        }
    q.n[slot] = n;
    q.id[slot] = id;
}

// A camera ray of phase A in double-float arithmetic (the FP64 camera's construction, ~10x
// cheaper than FP64 on B300, 48-bit accurate), straight into the compensated FP32 state.
template <int NF>
__device__ __forceinline__ void init_ray_pair(const Params& p, long long id, RayF<NF>& R, int& frame, int& pix) {
    frame = (int)(id / p.n_pix);
    pix = (int)(id - (long long)frame * p.n_pix);
    const int row = p.row0 + pix / p.nx, col = pix % p.nx;
    auto D = [](float2 v) { return df64(v.x, v.y); };
    const df64 alpha = D(p.f.amin_p) + df64((float)col + 0.5f, 0.f) * D(p.f.da_p);
    const df64 beta = D(p.f.bmin_p) + df64((float)row + 0.5f, 0.f) * D(p.f.db_p);
    df64 k[4];
    camera_k_t<df64>(D(p.f.a_p), D(p.f.sin_i_p), D(p.f.cos_i_p), D(p.f.r_cam_p), alpha, beta, k);
    const double tc = p.t_frames ? p.t_frames[frame] : p.t_cam;
    split_f(tc + p.cam_logdel + p.cam_tterm, R.x[0], R.xl[0]);
    R.x[1] = p.f.r_cam_p.x;
    R.xl[1] = p.f.r_cam_p.y;
    R.x[2] = p.f.incl_p.x;
    R.xl[2] = p.f.incl_p.y;
    R.x[3] = p.f.cam_phi_p.x;
    R.xl[3] = p.f.cam_phi_p.y;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        R.k[i] = k[i].hi;
        R.kl[i] = k[i].lo;
    }
    R.n = 0;
    R.snap = p.lc_fast ? p.frame_snap0 + frame : p.snap;
}

// Load queued ray `nid` of q into FP32 lane state (compensated pairs from the FP64 state).
template <int NF>
__device__ __forceinline__ long long load_ray_f(const Params& p, const RayQueue& q, size_t cap, long long nid, RayF<NF>& R) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 xv = q.xk[(size_t)i * cap + nid], kv = q.xk[(size_t)(4 + i) * cap + nid];
        R.x[i] = xv.x;
        R.xl[i] = xv.y;
        R.k[i] = kv.x;
        R.kl[i] = kv.y;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f < p.nf) {
            R.I[f] = float(q.I[(size_t)f * cap + nid]);
            tau_split(q.tau[(size_t)f * cap + nid], R.tau[f], R.tau_hi[f]);
        } else {
            R.I[f] = 0.f; R.tau[f] = 0.f; R.tau_hi[f] = df64(0.f, 0.f);
        }
    }
    R.n = q.n[nid];
    return q.id[nid];
}

// FP32 phases.  Phase A (io.fresh set): camera rays (or the surrogate's predicted states)
// from the id list; rays entering the FP64 region go to io.push.  Phase C: rays from io.in,
// integrated to termination (re-entries into the region are counted, not moved).
// The FP32 step is issue-bound and more resident warps hide its latencies: one frequency
// at most 102 registers (five 128-thread blocks, 20 warps per SM), two to four at most 128
// (four blocks).
template <int NF>
constexpr int kMixed32MinBlocks = NF == 1 ? 5 : (NF <= 4 ? 4 : 1);

template <int NF>
__global__ void __launch_bounds__(128, kMixed32MinBlocks<NF>) k_mixed_fp32(const Params p, PhaseIO io, size_t cap, unsigned long long* cnt,
                                                    unsigned long long* stats) {
    RayF<NF> R;
    long long id = -1;
    int frame = 0, pix = 0;
    bool drained = false;
    const bool fresh = io.fresh != nullptr;
    const long long n_total = (long long)cnt[io.total];
    const long long push_off = io.push_top >= 0 ? (long long)cap - (long long)cnt[io.push_top] : 0;
    unsigned long long c_rays = 0, c_steps = 0, c_trunc = 0, c_err = 0, c_re = 0;
    unsigned c_ph = 0;  // steps taken in this launch: the step count at exit minus that at entry
    for (;;) {
        const long long nid = warp_fetch(&cnt[io.fetch], n_total, id < 0, drained);
        if (id < 0 && nid >= 0) {
            if (fresh) {
                id = io.fresh[nid];
                if (p.start_xk && !p.fallback[id]) {
                    // learned surrogate: start from the predicted state after start_n steps
                    frame = (int)(id / p.n_pix);
                    pix = (int)(id - (long long)frame * p.n_pix);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 xv = p.start_xk[(long long)i * p.n_rays + id];
                        const float2 kv = p.start_xk[(long long)(4 + i) * p.n_rays + id];
                        R.x[i] = xv.x;
                        R.xl[i] = xv.y;
                        R.k[i] = kv.x;
                        R.kl[i] = kv.y;
                    }
                    R.n = p.start_n;
                    R.snap = p.lc_fast ? p.frame_snap0 + frame : p.snap;
                } else {
                    init_ray_pair<NF>(p, id, R, frame, pix);
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) { R.I[f] = 0.f; R.tau[f] = 0.f; R.tau_hi[f] = df64(0.f, 0.f); }
            } else {
                id = load_ray_f<NF>(p, io.in, cap, nid, R);
                frame = (int)(id / p.n_pix);
                pix = (int)(id - (long long)frame * p.n_pix);
                R.snap = p.lc_fast ? p.frame_snap0 + frame : p.snap;
            }
            c_ph -= (unsigned)R.n;
        }
        if (!__any_sync(0xffffffffu, id >= 0)) break;
        int st = -1;
        bool push = false;
        if (id >= 0) {
            st = step_fp32<NF>(p, R);
            if (st < 0 && in_fp64_region<float>(p, R.x, R.k)) {
                if (fresh) push = true;
                else c_re += 1;
            }
        }
        const long long slot = fresh ? warp_push_slot(&cnt[io.push_cnt], push) : -1;
        if (push) {
            float2 x[4], k[4];
            double tau[NF];
#pragma unroll
            for (int i = 0; i < 4; ++i) { x[i] = make_float2(R.x[i], R.xl[i]); k[i] = make_float2(R.k[i], R.kl[i]); }
#pragma unroll
            for (int f = 0; f < NF; ++f) tau[f] = double(R.tau[f]) + double(R.tau_hi[f]);
            store_ray<NF>(io.push, cap, slot + push_off, id, x, k, R.I, tau, R.n, p.nf);
            c_ph += (unsigned)R.n;
            id = -1;
        } else if (id >= 0 && st >= 0) {
            double I[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) I[f] = R.I[f];
            write_ray<NF>(p, frame, pix, I, R.n, st);
            c_rays += 1;
            c_steps += (unsigned long long)R.n;
            c_ph += (unsigned)R.n;
            c_trunc += (st == kTruncated);
            c_err += (st == kError);
            id = -1;
        }
    }
    warp_add_stats(stats, c_rays, c_steps, 0, c_trunc, c_err);
    if (c_re) atomicAdd(&stats[kStatReentry], c_re);
    // FP32 steps taken in this launch, per phase (inbound A, outbound C)
    unsigned long long c_ph64 = c_ph;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c_ph64 += __shfl_down_sync(0xffffffffu, c_ph64, o);
    if ((threadIdx.x & 31) == 0 && c_ph64) atomicAdd(&stats[fresh ? kStatFp32In : kStatFp32Out], c_ph64);
}

// FP64 phase: rays from io.in; FP64 (or double-float) geodesic steps, FP32 transfer samples.
// A ray runs at most io.budget steps in this launch; if it is still in the FP64 region then,
// it goes to io.requeue for the next pass.  Each pass therefore starts with full warps and
// its ragged end lasts at most `budget` steps.  Leavers go to io.push (an FP32 queue).
// Double-float steps are FP32-issue bound: ask for at least 4 resident blocks (16 warps)
// per SM so that latency is hidden; the FP64 variant is FP64-pipe bound and needs no cap.
template <typename S>
constexpr int kMixed64MinBlocks = std::is_same<S, df64>::value ? 4 : 1;

template <int NF, typename S = double>
__global__ void __launch_bounds__(128, kMixed64MinBlocks<S>) k_mixed_fp64(const Params p, PhaseIO io, size_t cap,
                                                                          unsigned long long* cnt, unsigned long long* stats) {
    RayM<NF, S> R;
    const S a_s = StateT<S>::from(p.a);
    long long id = -1;
    int frame = 0, pix = 0, n_in = 0;
    bool drained = false;
    const long long n_total = (long long)cnt[io.total];
    const long long in_off = io.in_top >= 0 ? (long long)cap - (long long)cnt[io.in_top] : 0;
    const long long rq_off = io.requeue_top >= 0 ? (long long)cap - (long long)cnt[io.requeue_top] : 0;
    const bool can_requeue = io.requeue_cnt >= 0;
    unsigned long long c_rays = 0, c_steps = 0, c_64 = 0, c_trunc = 0, c_err = 0;
    for (;;) {
        const long long nid = warp_fetch(&cnt[io.fetch], n_total, id < 0, drained);
        if (id < 0 && nid >= 0) {
            const RayQueue& q = io.in;
            const long long e = nid + in_off;
            id = q.id[e];
            frame = (int)(id / p.n_pix);
            pix = (int)(id - (long long)frame * p.n_pix);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 xv = q.xk[(size_t)i * cap + e], kv = q.xk[(size_t)(4 + i) * cap + e];
                R.x[i] = io.in_exact ? StateT<S>::from_exact(xv) : StateT<S>::from2(xv);
                R.k[i] = io.in_exact ? StateT<S>::from_exact(kv) : StateT<S>::from2(kv);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                R.I[f] = f < p.nf ? AccI<S>(q.I[(size_t)f * cap + e]) : AccI<S>(0);
                tau_split(f < p.nf ? q.tau[(size_t)f * cap + e] : 0.0, R.tau[f], R.tau_hi[f]);
            }
            R.n = q.n[e];
            n_in = R.n;
            R.snap = p.lc_fast ? p.frame_snap0 + frame : p.snap;
        }
        if (!__any_sync(0xffffffffu, id >= 0)) break;
        int st = -1;
        bool push = false, requeue = false;
        if (id >= 0) {
            st = step_mixed64<NF, S>(p, R, a_s);
            if (st < 0) {
                float xf[4], kf[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { xf[i] = StateT<S>::f(R.x[i]); kf[i] = StateT<S>::f(R.k[i]); }
                if (!in_fp64_region<float>(p, xf, kf)) push = true;
                else if (can_requeue && R.n - n_in >= io.budget) requeue = true;
            }
        }
        const long long slot = warp_push_slot(&cnt[io.push_cnt], push);
        const long long rslot = can_requeue ? warp_push_slot(&cnt[io.requeue_cnt], requeue) : -1;
        if (push || requeue) {
            double tau[NF];
            float2 xd[4], kd[4];
#pragma unroll
            for (int f = 0; f < NF; ++f) tau[f] = double(R.tau[f]) + double(R.tau_hi[f]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                xd[i] = push ? StateT<S>::to2(R.x[i]) : StateT<S>::to_exact(R.x[i]);
                kd[i] = push ? StateT<S>::to2(R.k[i]) : StateT<S>::to_exact(R.k[i]);
            }
            store_ray<NF>(push ? io.push : io.requeue, cap, push ? slot : rslot + rq_off, id, xd, kd, R.I, tau, R.n, p.nf);
            c_64 += (unsigned long long)(R.n - n_in);
            id = -1;
        } else if (id >= 0 && st >= 0) {
            double I[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) I[f] = R.I[f];
            write_ray<NF>(p, frame, pix, I, R.n, st);
            c_rays += 1;
            c_steps += (unsigned long long)R.n;
            c_64 += (unsigned long long)(R.n - n_in);
            c_trunc += (st == kTruncated);
            c_err += (st == kError);
            id = -1;
        }
    }
    warp_add_stats(stats, c_rays, c_steps, c_64, c_trunc, c_err);
    if (io.long_lane) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c_64 += __shfl_down_sync(0xffffffffu, c_64, o);
        if ((threadIdx.x & 31) == 0 && c_64) atomicAdd(&stats[kStatFp64Long], c_64);
    }
}

// Split the rays of a render into the near-critical list (pixel centre within `band` M of
// the critical curve, n_curve <= kMaxCurve FP32 vertices; `box` its bounding box grown by the
// band) and the rest, as id lists of counts cnt[kCntListCrit] and cnt[kCntListRest].
// Warp-aggregated appends: the order within a list is not deterministic, and nothing
// downstream depends on it (every ray's arithmetic is its own).
__global__ void __launch_bounds__(256) k_select_critical(const Params p, const float2* __restrict__ curve, int n_curve,
                                                         float band, float4 box, int* __restrict__ crit,
                                                         int* __restrict__ rest, unsigned long long* cnt) {
    __shared__ float2 sc[kMaxCurve];
    for (int c = threadIdx.x; c < n_curve; c += blockDim.x) sc[c] = curve[c];
    __syncthreads();
    const float band2 = band * band;
    const long long n = p.n_rays;
    // whole warps iterate together (the appends are warp-collective)
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const long long id = base + (threadIdx.x & 31);
        bool is_crit = false;
        if (id < n) {
            const int frame = (int)(id / p.n_pix);
            const int pix = (int)(id - (long long)frame * p.n_pix);
            const int row = p.row0 + pix / p.nx, col = pix % p.nx;
            const float alf = (float)(p.amin + (col + 0.5) * p.da), bef = (float)(p.bmin + (row + 0.5) * p.db);
            if (alf >= box.x && alf <= box.y && bef >= box.z && bef <= box.w) {
                float d2;
                bool inside;
                curve_relation(alf, bef, sc, n_curve, false, d2, inside);
                is_crit = d2 < band2;
            }
        }
        const long long sc_slot = warp_push_slot(&cnt[kCntListCrit], id < n && is_crit);
        const long long sr_slot = warp_push_slot(&cnt[kCntListRest], id < n && !is_crit);
        if (id < n) {
            if (is_crit) crit[sc_slot] = (int)id;
            else rest[sr_slot] = (int)id;
        }
    }
}

}  // namespace raptor
