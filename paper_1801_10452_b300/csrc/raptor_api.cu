// raptor_api.cu -- host implementation of the C ABI declared in include/raptor.h.
//
// Validation on the host, context-owned device buffers, launch configuration, the
// persistent kernels of raptor_kernels_fp64.cuh / raptor_kernels_mixed.cuh and the
// deterministic flux reduction.  No host-side fallback computes any part of a result.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/raptor.h"
#include "raptor_kernels_fp64.cuh"
#include "raptor_kernels_mixed.cuh"
#include "raptor_surrogate.cuh"
#include "raptor_mlp_tc.cuh"
#include "raptor_crossings.cuh"

using namespace raptor;

struct raptor_ctx {
    raptor_camera_desc cam;
    raptor_plasma_desc plasma;
    bool has_plasma = false;
    int device = 0;
    int num_sms = 0;
    float* d_grid = nullptr;      // interleaved [snap][n2][n1][8]
    float* d_x2tab = nullptr;     // MKS inversion table [kX2TabN + 1] of the loaded grid's h
    size_t grid_cap = 0;
    unsigned long long* d_counters = nullptr;  // [8] work counters
    unsigned long long* d_stats = nullptr;     // [kNumStats]
    double* d_partial = nullptr;
    unsigned long long* d_hist = nullptr;  // thin-disk spectrum (fixed point)
    size_t hist_cap = 0;
    double2* d_fwd = nullptr;              // forward-scheme transfer records
    size_t fwd_cap_elems = 0;
    size_t partial_cap = 0;
    double* d_flux = nullptr;
    size_t flux_cap = 0;
    double* d_img = nullptr;      // scratch image (host render, light curves without images)
    size_t img_cap = 0;
    double* d_tframes = nullptr;
    size_t tframes_cap = 0;
    int* d_trace_int = nullptr;   // [2]
    double* d_trace_I = nullptr;  // [64]
    double* d_rec = nullptr;
    size_t rec_cap = 0;
    MixedQueues mq;               // mixed-precision hand-off queues
    size_t mq_cap = 0;
    int* d_crit = nullptr;        // mixed path: near-critical ray ids (phase A1)
    int* d_rest = nullptr;        // mixed path: the other ray ids (phase A2)
    cudaStream_t s_long = nullptr;  // second stream of the mixed path (B-long)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_tail = nullptr, ev_net = nullptr;
    int tail_split = 0;           // after this many FP64 passes the rest moves to B-tail (0: never)
    int long_block = 0;           // threads per block of the second stream's FP64 passes (0: launch_block)
    int long_passes = 1;          // near-critical rays' FP64 passes and their step budgets
    int long_budget[8] = {1 << 30, 1 << 30, 1 << 30, 1 << 30, 1 << 30, 1 << 30, 1 << 30, 1 << 30};
    // CUDA graph of the last repeated render (raptor_graph_config)
    bool graphs = true;
    cudaStream_t s_cap = nullptr;     // capture stream
    cudaGraphExec_t g_exec = nullptr;
    std::vector<unsigned char> g_key, g_seen;
    long long g_captures = 0, g_replays = 0;
    unsigned long long epoch = 0;     // device-buffer epoch (see ensure)
    double crit_band = 0.5;       // M: near-critical band of the mixed path's B-long
    int n_passes = 8;             // FP64 passes of the other rays and their step budgets
    int pass_budget[8] = {16, 32, 48, 64, 96, 128, 256, 1 << 30};
    float2* d_curve = nullptr;    // critical curve (FP32 vertices) of the current (a, i)
    int n_curve = 0;
    float4 curve_box = make_float4(0.f, 0.f, 0.f, 0.f);  // its bounding box
    double curve_a = -1.0, curve_incl = -1.0;
    std::string err;
    cudaStream_t last_stream = nullptr;
    int launch_block = 128;       // threads per block of the persistent kernels
    int launch_bps = 0;           // blocks per SM (0 = occupancy maximum)
    int launch_bps64 = 2;         // blocks per SM of the mixed path's FP64 passes
    // learned surrogate
    bool sur_ready = false;
    float* s_P = nullptr;            // parameters (MlpLayout::SIZE)
    float* s_G = nullptr;            // gradients
    float* s_m1 = nullptr;           // Adam moments
    float* s_m2 = nullptr;
    __nv_bfloat16* s_w = nullptr;    // w2, w2t, w3, w3t, then w2, w3 in the tcgen05 operand layout (6 x 256 x 256)
    int s_kernel = RAPTOR_MLP_TCGEN05;  // inference kernel
    int* s_err = nullptr;            // device flag: a tensor-core wait ran out
    __nv_bfloat16* s_h2tc = nullptr; // tcgen05 inference: h2 tiles (64 KB each)
    size_t s_h2tc_tiles = 0;
    long long s_rows = 0;            // work-buffer rows
    float *s_x = nullptr, *s_z1 = nullptr, *s_z2 = nullptr, *s_z3 = nullptr, *s_out = nullptr, *s_dout = nullptr;
    float *s_dzf = nullptr, *s_dh = nullptr;
    __nv_bfloat16 *s_h1 = nullptr, *s_h2 = nullptr, *s_h3 = nullptr, *s_dzb = nullptr;
    double* s_y = nullptr;
    double* s_loss = nullptr;        // per-block loss partials
    float* s_in = nullptr;           // render: network inputs [rays][4]
    unsigned char* s_fb = nullptr;   // render: fallback flags
    float2* s_start = nullptr;       // render: start states [8][rays] (float pairs)
    size_t s_ray_cap = 0;
    double s_band = 0.5, s_r_exit = 50.0;
    int s_handoff = kSurrogateSteps;      // hand-off steps of the data raptor_surrogate_generate writes
    int s_handoff_net = kSurrogateSteps;  // hand-off steps of the network in use (from its parameters)
    unsigned long long s_step = 0;   // Adam step counter
    // crossing network (the surrogate's equatorial outputs); shares the work buffers above
    bool x_ready = false;
    float *x_P = nullptr, *x_G = nullptr, *x_m1 = nullptr, *x_m2 = nullptr;  // XLayout::SIZE each
    __nv_bfloat16* x_w = nullptr;    // w2, w2t, w3, w3t
    float *x_out = nullptr, *x_dout = nullptr;  // [rows][16]
    double* x_y = nullptr;           // [rows][16]
    unsigned long long x_step = 0;
    double x_band = 1.0;             // learned disk: fallback band around the critical curve (M)
    bool x_df = true;                // learned disk: fallback pixels in double-float arithmetic
    float x_norm[8] = {0.f};         // crossing network: input scale[4], shift[4] (host copy)
    double x_zmargin = 2.0;          // learned disk: presence logits within this of 0 fall back
    double x_lnr_margin = 0.01;      // learned disk: radii within this (in ln r) of r_in, r_out fall back
    __nv_bfloat16* x_h2tc = nullptr; // tcgen05 inference: h2 tiles (64 KB each)
    size_t x_h2tc_tiles = 0;
    int* x_list = nullptr;           // learned disk: fallback pixels
    unsigned int* x_nlist = nullptr;
    size_t x_list_cap = 0;
    // per-kernel CUDA-event timing (raptor_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct OpenRec {
        int slot, lane;
        cudaEvent_t a, b;
    };
    struct TimeRec {
        int slot, lane;
        double start_ms, dur_ms;
    };
    std::vector<OpenRec> ev_open;
    std::vector<TimeRec> timeline;   // per-launch records since the last clear (capped)
    cudaEvent_t ev_t0 = nullptr;     // timeline origin: recorded before the first scope
    bool t0_pending = false;
    double prof_ms[kProfSlots] = {0};
    long long prof_launches[kProfSlots] = {0};
};

namespace {

cudaEvent_t take_event(raptor_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one kernel launch (or `kernels` launches) with events on its stream when
// profiling is on; the slot's launch counter counts kernels.
struct ProfScope {
    raptor_ctx* c;
    int slot;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(raptor_ctx* c_, int slot_, cudaStream_t s_, int kernels = 1) : c(c_), slot(slot_), s(s_) {
        c->prof_launches[slot] += kernels;
        if (c->prof) {
            if (c->t0_pending) {
                if (!c->ev_t0) cudaEventCreate(&c->ev_t0);
                cudaEventRecord(c->ev_t0, s);
                c->t0_pending = false;
            }
            a = take_event(c);
            b = take_event(c);
            cudaEventRecord(a, s);
        }
    }
    ~ProfScope() {
        if (c->prof && a && b) {
            cudaEventRecord(b, s);
            c->ev_open.push_back({slot, (c->s_long && s == c->s_long) ? 1 : 0, a, b});
        }
    }
};

raptor_status fail(raptor_ctx* c, raptor_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define RCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RAPTOR_ENOMEM : RAPTOR_ECUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

// The context's device-buffer epoch (raptor_ctx::epoch) is bumped whenever the library
// frees or (re)allocates a buffer that a render's kernels reference, so that a captured
// render graph is never replayed with stale pointers.
template <typename T>
cudaError_t ensure(raptor_ctx* c, T** p, size_t* cap, size_t n) {
    if (*cap >= n && *p) return cudaSuccess;
    c->epoch += 1;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

std::string validate_camera(const raptor_camera_desc* d) {
    if (!d) return "camera descriptor is NULL";
    if (!std::isfinite(d->spin) || std::fabs(d->spin) >= 1.0) return "spin must satisfy |a| < 1";
    if (!finite_pos(d->mass_msun)) return "mass_msun must be positive";
    if (!finite_pos(d->distance_pc)) return "distance_pc must be positive";
    const double rh = 1.0 + std::sqrt(1.0 - d->spin * d->spin);
    if (!std::isfinite(d->r_cam) || d->r_cam <= 2.0 * rh || d->r_cam > 1e7) return "r_cam must lie in (2 r_h, 1e7]";
    if (!std::isfinite(d->incl_deg) || d->incl_deg <= 0.0 || d->incl_deg >= 180.0) return "incl_deg must lie in (0, 180)";
    if (d->nx < 1 || d->ny < 1 || (long long)d->nx * d->ny > (1LL << 31) - 1) return "nx, ny must be >= 1 with nx*ny < 2^31";
    if (!(d->alpha_max > d->alpha_min) || !std::isfinite(d->alpha_min) || !std::isfinite(d->alpha_max)) return "alpha range invalid";
    if (!(d->beta_max > d->beta_min) || !std::isfinite(d->beta_min) || !std::isfinite(d->beta_max)) return "beta range invalid";
    if (!(d->eps > 0.0) || !(d->eps <= 1.0)) return "eps must lie in (0, 1]";
    if (!(d->r_stop_factor >= 1.0) || !std::isfinite(d->r_stop_factor)) return "r_stop_factor must be >= 1";
    if (!std::isfinite(d->r_escape) || d->r_escape < d->r_cam) return "r_escape must be finite and >= r_cam";
    if (!(d->tau_cut > 0.0)) return "tau_cut must be > 0 (may be +inf)";
    if (d->max_steps < 1) return "max_steps must be >= 1";
    if (d->precision < RAPTOR_FP64 || d->precision > RAPTOR_MIXED_MLP) return "unknown precision";
    if (d->flags & ~(RAPTOR_FLAG_K2_EXACT | RAPTOR_FLAG_STEP_LINEAR_R | RAPTOR_FLAG_INNER_DF64 | RAPTOR_FLAG_VERLET |
                     RAPTOR_FLAG_VERLET_REEVAL | RAPTOR_FLAG_FORWARD_RT))
        return "unknown flag bits";
    if ((d->flags & (RAPTOR_FLAG_VERLET | RAPTOR_FLAG_VERLET_REEVAL)) && d->precision != RAPTOR_FP64)
        return "the Verlet integrator is built for RAPTOR_FP64 only";
    if ((d->flags & RAPTOR_FLAG_FORWARD_RT) && d->precision != RAPTOR_FP64)
        return "the forward transfer scheme is built for RAPTOR_FP64 only";
    if (!(d->r_fp64 >= 0.0) || !std::isfinite(d->r_fp64)) return "r_fp64 must be finite and >= 0";
    if (!(d->turn_kr >= 0.0) || !std::isfinite(d->turn_kr)) return "turn_kr must be finite and >= 0";
    if (!std::isfinite(d->t_delay)) return "t_delay must be finite";
    return "";
}

std::string validate_plasma(const raptor_plasma_desc* d) {
    if (!d) return "plasma descriptor is NULL";
    if (!(d->theta_e_min >= 0.0) || !std::isfinite(d->theta_e_min)) return "theta_e_min must be finite and >= 0";
    if (d->kind == RAPTOR_PLASMA_ANALYTIC) {
        const double v[6] = {d->n0, d->n_pow, d->the0, d->the_pow, d->B0_gauss, d->B_pow};
        for (double x : v)
            if (!std::isfinite(x)) return "analytic plasma constants must be finite";
        if (!(d->n0 >= 0.0) || !(d->the0 > 0.0) || !(d->B0_gauss >= 0.0)) return "need n0 >= 0, the0 > 0, B0 >= 0";
        return "";
    }
    if (d->kind != RAPTOR_PLASMA_GRID_MKS2D) return "unknown plasma kind";
    if (!d->fields) return "grid fields pointer is NULL";
    if (d->n1 < 2 || d->n2 < 2 || d->n_snap < 1) return "grid needs n1, n2 >= 2 and n_snap >= 1";
    if ((long long)d->n1 * d->n2 * d->n_snap * 8 > (1LL << 34)) return "grid too large";
    if (!(d->x1_max > d->x1_min) || !std::isfinite(d->x1_min) || !std::isfinite(d->x1_max)) return "x1 range invalid";
    if (!(d->h_mks > 0.0) || !(d->h_mks <= 1.0)) return "h_mks must lie in (0, 1]";
    if (d->n_snap > 1 && !finite_pos(d->dt_snap)) return "dt_snap must be positive";
    if (!std::isfinite(d->t0)) return "t0 must be finite";
    if (!finite_pos(d->mass_unit_g)) return "mass_unit_g must be positive";
    if (!(d->r_high > 0.0) || !(d->r_low > 0.0) || !std::isfinite(d->r_high) || !std::isfinite(d->r_low)) return "R_high, R_low must be positive";
    if (!(d->gamma_ad > 1.0) || !std::isfinite(d->gamma_ad)) return "gamma_ad must be > 1";
    return "";
}

double r_isco_prograde(double a) {
    const double z1 = 1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
    const double z2 = std::sqrt(3.0 * a * a + z1 * z1);
    const double sg = a < 0.0 ? -1.0 : 1.0;
    return 3.0 + z2 - sg * std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

// FP32 copies of the scalar parameters (frequencies are copied when they are set).
void fill_float_params(Params& p) {
    ParamsF& f = p.f;
    f.a = (float)p.a; f.eps = (float)p.eps; f.r_stop = (float)p.r_stop; f.r_esc = (float)p.r_esc;
    f.Lcm = (float)p.Lcm; f.tau_cut = (float)p.tau_cut;
    f.n0 = (float)p.n0; f.n_pow = (float)p.n_pow; f.the0 = (float)p.the0; f.the_pow = (float)p.the_pow;
    f.B0 = (float)p.B0; f.B_pow = (float)p.B_pow; f.r_isco = (float)p.r_isco; f.the_min = (float)p.the_min;
    f.x1_min = (float)p.x1_min; f.x1_max = (float)p.x1_max; f.dx1 = (float)p.dx1; f.dx2 = (float)p.dx2;
    f.h_mks = (float)p.h_mks; f.t0 = (float)p.t0; f.dt_snap = (float)p.dt_snap; f.rho0_ne = (float)p.rho0_ne;
    f.B_unit = (float)p.B_unit; f.r_high = (float)p.r_high; f.r_low = (float)p.r_low; f.gam = (float)p.gam;
    f.r_fp64 = (float)p.r_fp64; f.turn_kr = (float)p.turn_kr;
    f.r_isco_p = make_float2((float)p.r_isco, (float)(p.r_isco - (double)(float)p.r_isco));
    for (int i = 0; i < 16; ++i) f.nu[i] = (float)p.nu[i];
    auto pair = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    f.a_p = pair(p.a);
    f.sin_i_p = pair(p.sin_i);
    f.cos_i_p = pair(p.cos_i);
    f.r_cam_p = pair(p.r_cam);
    f.incl_p = pair(p.incl);
    f.cam_phi_p = pair(p.cam_phi);
    f.amin_p = pair(p.amin);
    f.da_p = pair(p.da);
    f.bmin_p = pair(p.bmin);
    f.db_p = pair(p.db);
}

// Host-side parameter block shared by every launch of a context.
Params base_params(const raptor_ctx* c) {
    Params p;
    std::memset(&p, 0, sizeof(p));
    const raptor_camera_desc& d = c->cam;
    p.a = d.spin;
    p.r_cam = d.r_cam;
    p.incl = d.incl_deg * kPi / 180.0;
    p.sin_i = std::sin(p.incl);
    p.cos_i = std::cos(p.incl);
    camera_x_terms(p.a, p.r_cam, &p.cam_logdel, &p.cam_tterm, &p.cam_phi);
    p.nx = d.nx;
    p.ny = d.ny;
    p.da = (d.alpha_max - d.alpha_min) / d.nx;
    p.db = (d.beta_max - d.beta_min) / d.ny;
    p.amin = d.alpha_min;
    p.bmin = d.beta_min;
    p.eps = d.eps;
    p.r_stop = d.r_stop_factor * (1.0 + std::sqrt(1.0 - d.spin * d.spin));
    p.r_esc = d.r_escape;
    p.tau_cut = d.tau_cut;
    p.max_steps = d.max_steps;
    p.flags = d.flags;
    p.Lcm = kG * d.mass_msun * kMsun / (kC * kC);
    const double D = d.distance_pc * kPc;
    p.pix_jy = p.da * p.db * p.Lcm * p.Lcm / (D * D) / 1e-23;
    p.r_fp64 = d.r_fp64;
    p.turn_kr = d.turn_kr;
    const raptor_plasma_desc& q = c->plasma;
    p.kind = q.kind;
    p.slow = q.slow_light;
    p.n0 = q.n0;
    p.n_pow = q.n_pow;
    p.the0 = q.the0;
    p.the_pow = q.the_pow;
    p.B0 = q.B0_gauss;
    p.B_pow = q.B_pow;
    p.r_isco = r_isco_prograde(d.spin);
    p.the_min = q.theta_e_min;
    if (q.kind == RAPTOR_PLASMA_GRID_MKS2D) {
        p.grid = c->d_grid;
        p.x2tab = c->d_x2tab;
        p.n1 = q.n1;
        p.n2 = q.n2;
        p.n_snap = q.n_snap;
        p.x1_min = q.x1_min;
        p.x1_max = q.x1_max;
        p.dx1 = (q.x1_max - q.x1_min) / q.n1;
        p.dx2 = 1.0 / q.n2;
        p.h_mks = q.h_mks;
        p.t0 = q.t0;
        p.dt_snap = q.n_snap > 1 ? q.dt_snap : 1.0;
        const double rho0 = q.mass_unit_g / (p.Lcm * p.Lcm * p.Lcm);
        p.rho0_ne = rho0 / (kMe + kMp);
        p.B_unit = kC * std::sqrt(4.0 * kPi * rho0);
        p.r_high = q.r_high;
        p.r_low = q.r_low;
        p.gam = q.gamma_ad;
    }
    fill_float_params(p);
    return p;
}

int grid_blocks(const raptor_ctx* c, int per_sm_occ) {
    const int bps = c->launch_bps > 0 ? std::min(c->launch_bps, per_sm_occ) : per_sm_occ;
    return std::max(1, bps) * c->num_sms;
}

template <int NF>
cudaError_t launch_fp64_nf(raptor_ctx* c, const Params& p, cudaStream_t s) {
    int occ = 0;
    const bool verlet = (p.flags & (kFlagVerlet | kFlagVerletReeval)) != 0;
    cudaError_t e = verlet ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_render_fp64<NF, true>, c->launch_block, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_render_fp64<NF, false>, c->launch_block, 0);
    if (e != cudaSuccess) return e;
    const long long need = (p.n_rays + c->launch_block - 1) / c->launch_block;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(grid_blocks(c, std::max(occ, 1)), need));
    Params q = p;
    if (p.flags & kFlagForwardRT) {
        // forward scheme: each thread's transfer records, [record][frequency][thread]
        q.fwd_stride = (long long)blocks * c->launch_block;
        q.fwd_cap = kForwardCap;
        e = ensure(c, &c->d_fwd, &c->fwd_cap_elems, (size_t)q.fwd_stride * kForwardCap * p.nf);
        if (e != cudaSuccess) return e;
        q.fwd = c->d_fwd;
    }
    ProfScope ps(c, kProfRenderFp64, s);
    if (verlet) k_render_fp64<NF, true><<<blocks, c->launch_block, 0, s>>>(q, c->d_counters, c->d_stats);
    else k_render_fp64<NF, false><<<blocks, c->launch_block, 0, s>>>(q, c->d_counters, c->d_stats);
    return cudaGetLastError();
}

cudaError_t launch_fp64(raptor_ctx* c, const Params& p, cudaStream_t s) {
    if (p.nf <= 1) return launch_fp64_nf<1>(c, p, s);
    if (p.nf <= 2) return launch_fp64_nf<2>(c, p, s);
    if (p.nf <= 4) return launch_fp64_nf<4>(c, p, s);
    if (p.nf <= 8) return launch_fp64_nf<8>(c, p, s);
    return launch_fp64_nf<16>(c, p, s);
}

std::vector<double> critical_curve(double a, double incl, int n);
int ew_blocks(long long n);

// The critical curve of the camera's (a, i) as kMaxCurve FP32 vertices on the device, and its
// bounding box (recomputed when a or i change).  The host vector is pageable: the copy is
// staged before cudaMemcpyAsync returns.
cudaError_t upload_curve(raptor_ctx* c, const Params& p, cudaStream_t s) {
    if (!c->d_curve) {
        c->epoch += 1;
        cudaError_t e = cudaMalloc((void**)&c->d_curve, kMaxCurve * sizeof(float2));
        if (e != cudaSuccess) return e;
    }
    if (c->curve_a == p.a && c->curve_incl == p.incl) return cudaSuccess;
    const std::vector<double> cc = critical_curve(p.a, p.incl, kMaxCurve);
    const int nc = (int)(cc.size() / 2);
    std::vector<float2> cf(nc);
    float4 box = make_float4(3e38f, -3e38f, 3e38f, -3e38f);
    for (int q = 0; q < nc; ++q) {
        cf[q] = make_float2((float)cc[2 * q], (float)cc[2 * q + 1]);
        box.x = std::min(box.x, cf[q].x);
        box.y = std::max(box.y, cf[q].x);
        box.z = std::min(box.z, cf[q].y);
        box.w = std::max(box.w, cf[q].y);
    }
    if (nc > 0) {
        cudaError_t e = cudaMemcpyAsync(c->d_curve, cf.data(), nc * sizeof(float2), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    c->n_curve = nc;
    c->curve_box = box;
    c->curve_a = p.a;
    c->curve_incl = p.incl;
    return cudaSuccess;
}

// Mixed precision (per frequency chunk): split the rays into near-critical and other
// (k_select_critical); phase A1 on the near-critical rays; snapshot of the FP64 queue; fork:
// B-long (their FP64 phase, no step budget) and phase C on its leavers on the context's
// second stream; on the caller's stream phase A2, the FP64 passes of growing step budget on
// the other queued rays, phase C on their leavers; join.
constexpr int kPassBudget[kMaxPasses] = {16, 32, 48, 64, 96, 128, 256, 1 << 30};
constexpr long long kGraphMaxRays = 1LL << 19;  // largest call replayed from a graph

template <int NF, typename S>
cudaError_t launch_fp64_phase(raptor_ctx* c, const Params& p, const PhaseIO& io, int blocks, int threads, cudaStream_t s) {
    ProfScope ps(c, io.long_lane ? kProfMixedBLong : kProfMixedB, s);
    k_mixed_fp64<NF, S><<<std::max(1, blocks), threads, 0, s>>>(p, io, c->mq.cap, c->d_counters, c->d_stats);
    return cudaGetLastError();
}

cudaError_t surrogate_prepare(raptor_ctx* ctx, const Params& p, cudaStream_t s);
cudaError_t surrogate_infer(raptor_ctx* ctx, const Params& p, cudaStream_t s);

// One frequency chunk of a mixed render.  sur_stage: run the surrogate's inference first
// (the first chunk of a learned render).
template <int NF>
cudaError_t launch_mixed_nf(raptor_ctx* c, const Params& p, cudaStream_t s, bool sur_stage) {
    cudaError_t e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * kNumCounters, s);
    if (e == cudaSuccess) e = upload_curve(c, p, s);
    if (e == cudaSuccess && !c->s_long) {
        // the near-critical rays' chain of steps bounds the frame: their stream gets the
        // highest priority, so its blocks are placed first whenever an SM frees resources
        // (kernel nodes captured into a graph keep the priority)
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->s_long, cudaStreamNonBlocking, hi);
    }
    cudaEvent_t* evs[] = {&c->ev_fork, &c->ev_join, &c->ev_tail, &c->ev_net};
    for (cudaEvent_t* ev : evs)
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    int occ32 = 0, occ64 = 0;
    const bool df = (p.flags & kFlagInnerDf64) != 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_mixed_fp32<NF>, c->launch_block, 0);
    if (e == cudaSuccess)
        e = df ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k_mixed_fp64<NF, df64>, c->launch_block, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k_mixed_fp64<NF, double>, c->launch_block, 0);
    if (e != cudaSuccess) return e;
    const int b32 = grid_blocks(c, std::max(occ32, 1));
    const int b64 = c->num_sms * std::max(1, c->launch_bps64 > 0 ? std::min(c->launch_bps64, occ64) : occ64);
    const long long need = (p.n_rays + c->launch_block - 1) / c->launch_block;
    const int bA = (int)std::max<long long>(1, std::min<long long>(b32, need));
    const MixedQueues& mq = c->mq;
    unsigned long long* cnt = c->d_counters;
    auto fp64_phase = [&](const PhaseIO& io, int blocks, int threads, cudaStream_t st) {
        return df ? launch_fp64_phase<NF, df64>(c, p, io, blocks, threads, st)
                  : launch_fp64_phase<NF, double>(c, p, io, blocks, threads, st);
    };
    // the second stream's launches keep the thread count of the first's FP64 passes; smaller
    // blocks return their registers to the SM as soon as their warps are done
    const int long_threads = c->long_block > 0 ? c->long_block : c->launch_block;
    const int b_long = (int)(((long long)b64 * c->launch_block + long_threads - 1) / long_threads);
    // the surrogate's stage (first frequency chunk of a learned render).  When every
    // near-critical ray is a fallback ray (critical band <= fallback band: the same FP32
    // predicate), those rays start at the camera and need nothing from the network: A1 runs
    // on the second stream beside the network's kernels, and B-long still waits for the
    // start states, so that it starts beside A2 as it does otherwise.
    const bool early = sur_stage && c->crit_band <= c->s_band;
    if (sur_stage) {
        e = surrogate_prepare(c, p, s);
        if (e == cudaSuccess && !early) e = surrogate_infer(c, p, s);
        if (e != cudaSuccess) return e;
    }
    // near-critical / other split
    const float grow = (float)c->crit_band + 1e-3f;
    const float4 box = make_float4(c->curve_box.x - grow, c->curve_box.y + grow, c->curve_box.z - grow, c->curve_box.w + grow);
    k_select_critical<<<ew_blocks(p.n_rays), 256, 0, s>>>(p, c->d_curve, c->n_curve, (float)c->crit_band, box, c->d_crit,
                                                          c->d_rest, cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // phase A1: near-critical rays.  Their entries fill the top of q64 (from cap - number of
    // near-critical rays up) and of the re-queue targets, the other rays' the bottom: each
    // ray has at most one entry per queue, so the ranges never meet.
    PhaseIO a1{};
    a1.fresh = c->d_crit;
    a1.push = mq.q64;
    a1.fetch = kCntFreshCrit;
    a1.total = kCntListCrit;
    a1.push_cnt = kCntPush64C;
    a1.push_top = kCntListCrit;
    a1.requeue_cnt = -1;
    if (early) {
        e = cudaEventRecord(c->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_long, c->ev_fork, 0);
        if (e != cudaSuccess) return e;
        {
            // one block per SM: every SM keeps room for a network CTA beside it (A1 has
            // time to spare until the start states are ready)
            ProfScope ps(c, kProfMixedA, c->s_long);
            k_mixed_fp32<NF><<<std::min(bA, c->num_sms), c->launch_block, 0, c->s_long>>>(p, a1, mq.cap, cnt, c->d_stats);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = surrogate_infer(c, p, s);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_net, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_long, c->ev_net, 0);
        if (e != cudaSuccess) return e;
    } else {
        {
            ProfScope ps(c, kProfMixedA, s);
            k_mixed_fp32<NF><<<bA, c->launch_block, 0, s>>>(p, a1, mq.cap, cnt, c->d_stats);
        }
        e = cudaGetLastError();
        // fork: the near-critical rays' FP64 phase on the second stream
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_long, c->ev_fork, 0);
        if (e != cudaSuccess) return e;
    }
    // the near-critical rays' FP64 phase on the second stream, in passes like the other
    // rays' (each pass re-packs the unfinished rays into full warps)
    const int LK = c->long_passes;
    for (int pass = 0; pass < LK; ++pass) {
        PhaseIO bl{};
        bl.in = pass == 0 ? mq.q64 : ((pass & 1) ? mq.q64b : mq.q64c);
        bl.in_top = kCntListCrit;
        bl.requeue = (pass & 1) ? mq.q64c : mq.q64b;
        bl.requeue_top = kCntListCrit;
        bl.push = mq.q32l;
        bl.fetch = kCntLPassFetch + pass;
        bl.total = pass == 0 ? kCntPush64C : kCntLPassOut + pass - 1;
        bl.push_cnt = kCntPush32L;
        bl.requeue_cnt = pass + 1 < LK ? kCntLPassOut + pass : -1;
        bl.budget = pass + 1 < LK ? c->long_budget[pass] : (1 << 30);
        bl.in_exact = pass > 0;
        bl.long_lane = 1;
        e = fp64_phase(bl, b_long, long_threads, c->s_long);
        if (e != cudaSuccess) return e;
    }
    // phase A2
    PhaseIO a2{};
    a2.fresh = c->d_rest;
    a2.push = mq.q64;
    a2.fetch = kCntFreshRest;
    a2.total = kCntListRest;
    a2.push_cnt = kCntPush64;
    a2.requeue_cnt = -1;
    {
        ProfScope ps(c, kProfMixedA, s);
        k_mixed_fp32<NF><<<bA, c->launch_block, 0, s>>>(p, a2, mq.cap, cnt, c->d_stats);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // phase C template (FP32 queue -> termination)
    PhaseIO cc{};
    cc.in = mq.q32;
    cc.fetch = kCntFetch32;
    cc.total = kCntPush32;
    cc.push_cnt = -1;
    cc.requeue_cnt = -1;
    // FP64 passes on the other rays: q64 [snapshot, end) -> q64b -> q64c -> q64b ...; with a
    // tail split after K passes, pass K - 1 still re-queues, and B-tail (second stream, after
    // B-long and after pass K - 1) takes those rays to the end of their FP64 phase
    const int K = (c->tail_split > 0 && c->tail_split < c->n_passes) ? c->tail_split : c->n_passes;
    const bool tail = K < c->n_passes;
    for (int pass = 0; pass < K; ++pass) {
        PhaseIO b{};
        b.in = pass == 0 ? mq.q64 : ((pass & 1) ? mq.q64b : mq.q64c);
        b.requeue = (pass & 1) ? mq.q64c : mq.q64b;
        b.push = mq.q32;
        b.fetch = kCntPassFetch + pass;
        b.total = pass == 0 ? kCntPush64 : kCntPassOut + pass - 1;
        b.push_cnt = kCntPush32;
        b.requeue_cnt = (pass + 1 < c->n_passes) ? kCntPassOut + pass : -1;
        b.budget = pass + 1 < c->n_passes ? c->pass_budget[pass] : (1 << 30);
        b.in_exact = pass > 0;
        e = fp64_phase(b, b64, c->launch_block, s);
        if (e != cudaSuccess) return e;
    }
    if (tail) {
        e = cudaEventRecord(c->ev_tail, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_long, c->ev_tail, 0);
        if (e != cudaSuccess) return e;
        PhaseIO bt{};
        bt.in = ((K - 1) & 1) ? mq.q64c : mq.q64b;
        bt.push = mq.q32l;
        bt.fetch = kCntTailFetch;
        bt.total = kCntPassOut + K - 1;
        bt.push_cnt = kCntPush32L;
        bt.requeue_cnt = -1;
        bt.budget = 1 << 30;
        bt.in_exact = 1;
        bt.long_lane = 1;
        e = fp64_phase(bt, b_long, long_threads, c->s_long);
        if (e != cudaSuccess) return e;
    }
    // phase C on B-long's (and B-tail's) leavers, on the second stream as soon as they are
    // all queued: it overlaps the first stream's phase C instead of following it
    PhaseIO cl = cc;
    cl.in = mq.q32l;
    cl.fetch = kCntFetch32L;
    cl.total = kCntPush32L;
    {
        ProfScope ps(c, kProfMixedC, c->s_long);
        k_mixed_fp32<NF><<<std::max(1, b32), c->launch_block, 0, c->s_long>>>(p, cl, mq.cap, cnt, c->d_stats);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->s_long);
    if (e != cudaSuccess) return e;
    // phase C on the passes' leavers; then the join
    {
        ProfScope ps(c, kProfMixedC, s);
        k_mixed_fp32<NF><<<std::max(1, b32), c->launch_block, 0, s>>>(p, cc, mq.cap, cnt, c->d_stats);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
    return e;
}

cudaError_t launch_mixed(raptor_ctx* c, const Params& p, cudaStream_t s, bool sur_stage) {
    if (p.nf <= 1) return launch_mixed_nf<1>(c, p, s, sur_stage);
    if (p.nf <= 2) return launch_mixed_nf<2>(c, p, s, sur_stage);
    if (p.nf <= 4) return launch_mixed_nf<4>(c, p, s, sur_stage);
    if (p.nf <= 8) return launch_mixed_nf<8>(c, p, s, sur_stage);
    return launch_mixed_nf<16>(c, p, s, sur_stage);
}

raptor_status prepare_surrogate_render(raptor_ctx* ctx, Params& p, cudaStream_t s);
raptor_status disk_learned_stage(raptor_ctx* ctx, const Params& p, DiskArgs& a, cudaStream_t s);
raptor_status check_tc_err(raptor_ctx* ctx);

// Enqueue every ray of `p` (all frequency chunks), then the flux reduction of `planes`
// image planes into c->d_flux.
raptor_status run_rays(raptor_ctx* ctx, Params p, const double* freqs, int n_freq, long long planes_per_frame,
                       int n_frames, cudaStream_t s) {
    if (ctx->cam.precision == RAPTOR_MIXED_MLP) {
        const raptor_status st = prepare_surrogate_render(ctx, p, s);
        if (st != RAPTOR_OK) return st;
    }
    p.nf_total = n_freq;
    p.i_unscale = ctx->cam.precision == RAPTOR_FP64 ? 1.0 : kIUnscale;
    for (int f0 = 0; f0 < n_freq; f0 += 16) {
        p.f_off = f0;
        p.nf = std::min(16, n_freq - f0);
        for (int f = 0; f < p.nf; ++f) p.nu[f] = freqs[f0 + f];
        for (int f = 0; f < 16; ++f) p.f.nu[f] = (float)p.nu[f];
        if (ctx->cam.precision == RAPTOR_FP64) {
            RCK(cudaMemsetAsync(ctx->d_counters, 0, sizeof(unsigned long long) * kNumCounters, s));
            RCK(launch_fp64(ctx, p, s));
        } else {
            const size_t need = (size_t)p.n_rays;
            if (p.n_rays > 0x7fffffffLL) return fail(ctx, RAPTOR_EINVAL, "the mixed path takes at most 2^31 - 1 rays per call");
            if (ctx->mq_cap < need || ctx->mq.nf_cap < p.nf) {
                ctx->epoch += 1;
                free_mixed_queues(ctx->mq);
                cudaFree(ctx->d_crit);
                cudaFree(ctx->d_rest);
                ctx->d_crit = ctx->d_rest = nullptr;
                ctx->mq_cap = 0;
                RCK(alloc_mixed_queues(ctx->mq, need, 16));
                RCK(cudaMalloc((void**)&ctx->d_crit, need * sizeof(int)));
                RCK(cudaMalloc((void**)&ctx->d_rest, need * sizeof(int)));
                ctx->mq_cap = need;
            }
            RCK(launch_mixed(ctx, p, s, ctx->cam.precision == RAPTOR_MIXED_MLP && f0 == 0));
        }
    }
    // flux: planes = n_frames * n_freq, each n_rows * nx
    const long long len = (long long)p.n_rows * p.nx;
    const int planes = n_frames * n_freq;
    const int chunks = (int)std::min<long long>(256, std::max<long long>(1, len / 4096));
    RCK(ensure(ctx, &ctx->d_partial, &ctx->partial_cap, (size_t)planes * chunks));
    RCK(ensure(ctx, &ctx->d_flux, &ctx->flux_cap, (size_t)planes));
    dim3 g1(chunks, planes);
    {
        ProfScope ps(ctx, kProfReduce, s);
        k_reduce_partial<<<g1, kRedThreads, 0, s>>>(p.image, len, chunks, ctx->d_partial);
    }
    RCK(cudaGetLastError());
    {
        ProfScope ps(ctx, kProfReduce, s);
        k_reduce_final<<<planes, kRedThreads, 0, s>>>(ctx->d_partial, chunks, ctx->d_flux);
    }
    RCK(cudaGetLastError());
    (void)planes_per_frame;
    return RAPTOR_OK;
}

// run_rays through a CUDA graph: the second identical call (same parameters, frequencies,
// context settings and device buffers) captures the whole launch sequence, both streams
// included, on the context's capture stream; later identical calls replay it with one
// cudaGraphLaunch.  Calls with profiling on, or whose capture fails, run directly.
raptor_status run_rays_graph(raptor_ctx* ctx, const Params& p, const double* freqs, int n_freq, long long planes_per_frame,
                             int n_frames, cudaStream_t s) {
    // Graph replay saves the launch latencies, which matter up to ~2^19 rays per call
    // (measured 3-5 % at 64^2 .. 512^2); beyond, the graph's own ordering of the two streams'
    // kernels overlaps them worse than direct launches do (measured 2-7 % slower at 1024^2).
    if (!ctx->graphs || ctx->prof || p.n_rays > kGraphMaxRays) return run_rays(ctx, p, freqs, n_freq, planes_per_frame, n_frames, s);
    std::vector<unsigned char> key;
    auto put = [&key](const void* v, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(v);
        key.insert(key.end(), b, b + n);
    };
    const unsigned long long epoch = ctx->epoch;
    put(&p, sizeof(p));
    put(&n_freq, sizeof(n_freq));
    put(freqs, sizeof(double) * n_freq);
    put(&planes_per_frame, sizeof(planes_per_frame));
    put(&n_frames, sizeof(n_frames));
    put(&ctx->cam, sizeof(ctx->cam));
    int cfg[] = {ctx->launch_block, ctx->launch_bps, ctx->launch_bps64, ctx->n_passes, ctx->tail_split, ctx->s_kernel,
                 ctx->sur_ready ? 1 : 0, ctx->long_block, ctx->long_passes, ctx->s_handoff_net};
    put(cfg, sizeof(cfg));
    put(ctx->pass_budget, sizeof(ctx->pass_budget));
    put(ctx->long_budget, sizeof(ctx->long_budget));
    double dcfg[] = {ctx->crit_band, ctx->s_band, ctx->s_r_exit};
    put(dcfg, sizeof(dcfg));
    put(&epoch, sizeof(epoch));
    put(&s, sizeof(s));
    if (ctx->g_exec && key == ctx->g_key) {
        RCK(cudaGraphLaunch(ctx->g_exec, s));
        ctx->g_replays += 1;
        return RAPTOR_OK;
    }
    if (key != ctx->g_seen) {
        ctx->g_seen = key;
        return run_rays(ctx, p, freqs, n_freq, planes_per_frame, n_frames, s);
    }
    // second identical call: capture
    if (!ctx->s_cap) RCK(cudaStreamCreateWithFlags(&ctx->s_cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    RCK(cudaStreamBeginCapture(ctx->s_cap, cudaStreamCaptureModeThreadLocal));
    const raptor_status st = run_rays(ctx, p, freqs, n_freq, planes_per_frame, n_frames, ctx->s_cap);
    const cudaError_t ec = cudaStreamEndCapture(ctx->s_cap, &g);
    cudaGraphExec_t ex = nullptr;
    const bool ok = st == RAPTOR_OK && ec == cudaSuccess && g && ctx->epoch == epoch &&
                    cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        if (ex) cudaGraphExecDestroy(ex);
        cudaGetLastError();  // clear a capture error; run the call directly
        ctx->g_seen.clear();
        ctx->err.clear();
        return run_rays(ctx, p, freqs, n_freq, planes_per_frame, n_frames, s);
    }
    if (ctx->g_exec) cudaGraphExecDestroy(ctx->g_exec);
    ctx->g_exec = ex;
    ctx->g_key = key;
    ctx->g_captures += 1;
    RCK(cudaGraphLaunch(ctx->g_exec, s));
    ctx->g_replays += 1;
    return RAPTOR_OK;
}

raptor_status check_freqs(raptor_ctx* ctx, const double* freqs, int n_freq) {
    if (!freqs) return fail(ctx, RAPTOR_EINVAL, "freqs_hz is NULL");
    if (n_freq < 1 || n_freq > 64) return fail(ctx, RAPTOR_EINVAL, "n_freq must lie in [1, 64]");
    for (int f = 0; f < n_freq; ++f)
        if (!finite_pos(freqs[f])) return fail(ctx, RAPTOR_EINVAL, "frequencies must be finite and positive");
    if ((ctx->cam.flags & RAPTOR_FLAG_FORWARD_RT) && n_freq > kForwardMaxFreq)
        return fail(ctx, RAPTOR_EINVAL, "the forward scheme takes at most 4 frequencies");
    return RAPTOR_OK;
}

}  // namespace

extern "C" {

int raptor_version(void) { return 10000; }

void raptor_camera_desc_default(raptor_camera_desc* d) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->spin = 0.9;
    d->mass_msun = 4.0e6;
    d->distance_pc = 7.88e3;
    d->r_cam = 1000.0;
    d->incl_deg = 60.0;
    d->nx = d->ny = 64;
    d->alpha_min = d->beta_min = -20.0;
    d->alpha_max = d->beta_max = 20.0;
    d->eps = 0.05;
    d->r_stop_factor = 1.01;
    d->r_escape = 1000.0;
    d->tau_cut = INFINITY;
    d->max_steps = 100000;
    d->precision = RAPTOR_FP64;
    d->flags = 0;
    d->r_fp64 = 6.0;
    d->turn_kr = 0.05;
    d->t_delay = 1000.0;
}

void raptor_plasma_desc_default(raptor_plasma_desc* d) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->kind = RAPTOR_PLASMA_ANALYTIC;
    d->n0 = 1.0e6;
    d->n_pow = -1.5;
    d->the0 = 10.0;
    d->the_pow = -1.0;
    d->B0_gauss = 20.0;
    d->B_pow = -1.0;
    d->h_mks = 1.0;
    d->dt_snap = 1.0;
    d->r_high = d->r_low = 1.0;
    d->gamma_ad = 4.0 / 3.0;
}

raptor_status raptor_camera_init(const raptor_camera_desc* desc, raptor_ctx** out) {
    if (!out) return RAPTOR_EINVAL;
    *out = nullptr;
    const std::string v = validate_camera(desc);
    if (!v.empty()) return RAPTOR_EINVAL;
    raptor_ctx* ctx = new (std::nothrow) raptor_ctx();
    if (!ctx) return RAPTOR_ENOMEM;
    ctx->cam = *desc;
    raptor_plasma_desc_default(&ctx->plasma);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_counters, kNumCounters * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_stats, kNumStats * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, kNumStats * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_trace_int, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_trace_I, 64 * sizeof(double));
    if (e == cudaSuccess) {
        // the sin/cos node table of this device (double-float polar-angle sin/cos)
        float4 tab[kSinTabN + 1];
        sincos_table_fill(tab);
        e = cudaMemcpyToSymbol(g_sincos_tab, tab, sizeof(tab));
    }
    if (e != cudaSuccess) {
        const raptor_status s = e == cudaErrorMemoryAllocation ? RAPTOR_ENOMEM : RAPTOR_ECUDA;
        raptor_destroy(ctx);
        return s;
    }
    *out = ctx;
    return RAPTOR_OK;
}

raptor_status raptor_camera_set(raptor_ctx* ctx, const raptor_camera_desc* desc) {
    if (!ctx) return RAPTOR_EINVAL;
    const std::string v = validate_camera(desc);
    if (!v.empty()) return fail(ctx, RAPTOR_EINVAL, v);
    ctx->cam = *desc;
    return RAPTOR_OK;
}

// Transpose [snap][8][n2][n1] planes into interleaved [snap][n2][n1][8] cells.
__global__ void k_interleave_grid(const float* __restrict__ src, float* __restrict__ dst, long long cells_per_snap, int n_snap) {
    const long long total = cells_per_snap * n_snap;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total; c += (long long)gridDim.x * blockDim.x) {
        const long long s = c / cells_per_snap, cell = c - s * cells_per_snap;
        const float* S = src + s * 8 * cells_per_snap + cell;
        float4 lo = make_float4(S[0], S[cells_per_snap], S[2 * cells_per_snap], S[3 * cells_per_snap]);
        float4 hi = make_float4(S[4 * cells_per_snap], S[5 * cells_per_snap], S[6 * cells_per_snap], S[7 * cells_per_snap]);
        reinterpret_cast<float4*>(dst)[2 * c] = lo;
        reinterpret_cast<float4*>(dst)[2 * c + 1] = hi;
    }
}

raptor_status raptor_load_plasma(raptor_ctx* ctx, const raptor_plasma_desc* desc, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    const std::string v = validate_plasma(desc);
    if (!v.empty()) return fail(ctx, RAPTOR_EINVAL, v);
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    if (desc->kind == RAPTOR_PLASMA_GRID_MKS2D) {
        const size_t cells = (size_t)desc->n1 * desc->n2;
        const size_t n = cells * desc->n_snap * 8;
        RCK(ensure(ctx, &ctx->d_grid, &ctx->grid_cap, n));
        float* staging = nullptr;
        RCK(cudaMallocAsync((void**)&staging, n * sizeof(float), s));
        cudaError_t e = cudaMemcpyAsync(staging, desc->fields, n * sizeof(float),
                                        desc->fields_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            const int blocks = (int)std::min<size_t>(4096, (cells * desc->n_snap + 255) / 256);
            ProfScope ps(ctx, kProfLoad, s);
            k_interleave_grid<<<std::max(blocks, 1), 256, 0, s>>>(staging, ctx->d_grid, (long long)cells, desc->n_snap);
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaFreeAsync(staging, s);
        if (e == cudaSuccess) e = e2;
        // x2(theta) at the table's angles for this grid's h (FP64 Newton roots)
        if (e == cudaSuccess && !ctx->d_x2tab) e = cudaMalloc((void**)&ctx->d_x2tab, (kX2TabN + 1) * sizeof(float));
        if (e == cudaSuccess) {
            std::vector<float> tab(kX2TabN + 1);
            for (int i = 0; i <= kX2TabN; ++i) tab[i] = (float)newton_x2<double>(kPi * i / kX2TabN, desc->h_mks);
            e = cudaMemcpyAsync(ctx->d_x2tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host table goes out of scope
        }
        if (e == cudaSuccess && !desc->fields_on_device) e = cudaStreamSynchronize(s);  // caller may free its host buffer
        ctx->epoch += 1;  // the kernels read the new table
        if (e != cudaSuccess) return fail(ctx, RAPTOR_ECUDA, std::string("load_plasma: ") + cudaGetErrorString(e));
    }
    ctx->plasma = *desc;
    ctx->plasma.fields = nullptr;
    ctx->has_plasma = true;
    return RAPTOR_OK;
}

raptor_status raptor_render_ex(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs, int row0, int n_rows,
                               int snap, double* image_dev, double* flux_jy_host, int* steps_dev, int* status_dev,
                               void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->has_plasma) return fail(ctx, RAPTOR_ENOPLASMA, "raptor_load_plasma has not been called");
    raptor_status st = check_freqs(ctx, freqs_hz, n_freq);
    if (st != RAPTOR_OK) return st;
    if (!image_dev) return fail(ctx, RAPTOR_EINVAL, "image_dev is NULL");
    if (row0 < 0 || n_rows < 1 || row0 + n_rows > ctx->cam.ny) return fail(ctx, RAPTOR_EINVAL, "row window outside the image");
    if (!std::isfinite(t_obs)) return fail(ctx, RAPTOR_EINVAL, "t_obs must be finite");
    if (ctx->plasma.kind == RAPTOR_PLASMA_GRID_MKS2D && (snap < 0 || snap >= ctx->plasma.n_snap))
        return fail(ctx, RAPTOR_EINVAL, "snap outside [0, n_snap)");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    Params p = base_params(ctx);
    p.row0 = row0;
    p.n_rows = n_rows;
    p.n_pix = n_rows * ctx->cam.nx;
    p.n_rays = p.n_pix;
    p.t_cam = t_obs + ctx->cam.t_delay;
    p.snap = snap;
    p.image = image_dev;
    p.steps_out = steps_dev;
    p.status_out = status_dev;
    st = run_rays_graph(ctx, p, freqs_hz, n_freq, n_freq, 1, s);
    if (st != RAPTOR_OK) return st;
    if (flux_jy_host) {
        RCK(cudaMemcpyAsync(flux_jy_host, ctx->d_flux, n_freq * sizeof(double), cudaMemcpyDeviceToHost, s));
        RCK(cudaStreamSynchronize(s));
        if (ctx->cam.precision == RAPTOR_MIXED_MLP) return check_tc_err(ctx);
    }
    return RAPTOR_OK;
}

raptor_status raptor_render(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs, double* image_dev,
                            double* flux_jy_host, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    return raptor_render_ex(ctx, freqs_hz, n_freq, t_obs, 0, ctx->cam.ny, 0, image_dev, flux_jy_host, nullptr, nullptr,
                            stream);
}

raptor_status raptor_disk_desc_default(raptor_disk_desc* d) {
    if (!d) return RAPTOR_EINVAL;
    d->r_in = 0.0;
    d->r_out = 15.0;
    d->q = 2.0;
    d->max_cross = 10;
    d->profile_order = 1;
    d->n_bins = 64;
    d->x_min = 0.2;
    d->x_max = 1.6;
    return RAPTOR_OK;
}

static raptor_status disk_render_impl(raptor_ctx* ctx, const raptor_disk_desc* d, double* ratio_dev, double* intensity_dev,
                                      int* order_dev, int* status_dev, int* steps_dev, double* profile_host, void* stream,
                                      bool learned) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!d) return fail(ctx, RAPTOR_EINVAL, "disk descriptor is NULL");
    if (!ratio_dev || !intensity_dev || !order_dev) return fail(ctx, RAPTOR_EINVAL, "ratio, intensity and order buffers are required");
    if (ctx->cam.flags & (RAPTOR_FLAG_VERLET | RAPTOR_FLAG_VERLET_REEVAL))
        return fail(ctx, RAPTOR_EUNSUPPORTED, "the thin disk is integrated with RK4 only");
    const double r_in = d->r_in > 0.0 ? d->r_in : r_isco_prograde(ctx->cam.spin);
    if (!std::isfinite(d->r_in) || !(d->r_out > r_in) || !std::isfinite(d->r_out))
        return fail(ctx, RAPTOR_EINVAL, "need finite 0 < r_in < r_out (r_in <= 0: the ISCO)");
    if (!std::isfinite(d->q) || d->max_cross < 1 || d->profile_order < 0)
        return fail(ctx, RAPTOR_EINVAL, "need finite q, max_cross >= 1, profile_order >= 0");
    if (profile_host && (d->n_bins < 1 || d->n_bins > (1 << 20) || !(d->x_max > d->x_min) || !(d->x_min >= 0.0) ||
                         !std::isfinite(d->x_max)))
        return fail(ctx, RAPTOR_EINVAL, "need 1 <= n_bins <= 2^20 and 0 <= x_min < x_max");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    Params p = base_params(ctx);
    p.row0 = 0;
    p.n_rows = ctx->cam.ny;
    p.n_pix = ctx->cam.ny * ctx->cam.nx;
    p.n_rays = p.n_pix;
    p.t_cam = 0.0;
    DiskArgs a{};
    a.r_in = r_in;
    a.r_out = d->r_out;
    a.q = d->q;
    a.max_cross = d->max_cross;
    a.ratio = ratio_dev;
    a.inten = intensity_dev;
    a.order = order_dev;
    a.status = status_dev;
    a.steps = steps_dev;
    if (learned) {
        const raptor_status ls = disk_learned_stage(ctx, p, a, s);
        if (ls != RAPTOR_OK) return ls;
    }
    RCK(cudaMemsetAsync(ctx->d_counters, 0, sizeof(unsigned long long) * kNumCounters, s));
    // the learned disk's fallback pixels in double-float arithmetic unless FP64 is asked for
    const bool df = learned && ctx->x_df;
    const int blk = df ? 128 : ctx->launch_block;
    int occ = 0;
    if (df) RCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_disk_df, blk, 0));
    else RCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_disk_fp64, blk, 0));
    const long long need = (p.n_rays + blk - 1) / blk;
    const long long blocks = std::max<long long>(1, std::min<long long>(grid_blocks(ctx, std::max(occ, 1)), need));
    {
        ProfScope ps(ctx, kProfDisk, s);
        if (df) k_disk_df<<<(int)blocks, blk, 0, s>>>(p, a, ctx->d_counters, ctx->d_stats);
        else k_disk_fp64<<<(int)blocks, blk, 0, s>>>(p, a, ctx->d_counters, ctx->d_stats);
    }
    RCK(cudaGetLastError());
    if (!profile_host) return RAPTOR_OK;
    // fixed-point scale: the largest possible total (every pixel at the top bin edge and the
    // inner radius, times the field of view) stays below 2^62
    const double pix_area = p.da * p.db;
    const double w_max = std::pow(d->x_max, 4.0) * std::pow(r_in, -d->q) * pix_area * (double)p.n_pix;
    const double scale = std::ldexp(1.0, 62 - (int)std::ceil(std::log2(std::max(w_max, 1e-290))));
    RCK(ensure(ctx, &ctx->d_hist, &ctx->hist_cap, (size_t)d->n_bins));
    RCK(cudaMemsetAsync(ctx->d_hist, 0, sizeof(unsigned long long) * d->n_bins, s));
    const double dx = (d->x_max - d->x_min) / d->n_bins;
    {
        ProfScope ps(ctx, kProfDisk, s);
        k_disk_profile<<<ew_blocks(p.n_pix), 256, 0, s>>>(ratio_dev, intensity_dev, order_dev, p.n_pix, d->profile_order,
                                                          d->x_min, dx, d->n_bins, pix_area, scale, ctx->d_hist);
    }
    RCK(cudaGetLastError());
    std::vector<unsigned long long> h(d->n_bins);
    RCK(cudaMemcpyAsync(h.data(), ctx->d_hist, sizeof(unsigned long long) * d->n_bins, cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    if (learned) {
        const raptor_status te = check_tc_err(ctx);
        if (te != RAPTOR_OK) return te;
    }
    for (int b = 0; b < d->n_bins; ++b) profile_host[b] = (double)h[b] / scale;
    return RAPTOR_OK;
}

raptor_status raptor_disk_render(raptor_ctx* ctx, const raptor_disk_desc* d, double* ratio_dev, double* intensity_dev,
                                 int* order_dev, int* status_dev, int* steps_dev, double* profile_host, void* stream) {
    return disk_render_impl(ctx, d, ratio_dev, intensity_dev, order_dev, status_dev, steps_dev, profile_host, stream, false);
}

raptor_status raptor_disk_render_learned(raptor_ctx* ctx, const raptor_disk_desc* d, double* ratio_dev,
                                         double* intensity_dev, int* order_dev, int* status_dev, int* steps_dev,
                                         double* profile_host, void* stream) {
    return disk_render_impl(ctx, d, ratio_dev, intensity_dev, order_dev, status_dev, steps_dev, profile_host, stream, true);
}

raptor_status raptor_render_host(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs, double* image_host,
                                 double* flux_jy_host, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    raptor_status st = check_freqs(ctx, freqs_hz, n_freq);
    if (st != RAPTOR_OK) return st;
    const size_t n = (size_t)n_freq * ctx->cam.nx * ctx->cam.ny;
    RCK(ensure(ctx, &ctx->d_img, &ctx->img_cap, n));
    double flux[64];
    st = raptor_render(ctx, freqs_hz, n_freq, t_obs, ctx->d_img, flux, stream);
    if (st != RAPTOR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (image_host) {
        RCK(cudaMemcpyAsync(image_host, ctx->d_img, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        RCK(cudaStreamSynchronize(s));
    }
    if (flux_jy_host) std::memcpy(flux_jy_host, flux, n_freq * sizeof(double));
    return RAPTOR_OK;
}

raptor_status raptor_lightcurve(raptor_ctx* ctx, const double* freqs_hz, int n_freq, const double* t_obs_host, int n_frames,
                                int first_frame, double* flux_jy_host, double* images_dev, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->has_plasma) return fail(ctx, RAPTOR_ENOPLASMA, "raptor_load_plasma has not been called");
    raptor_status st = check_freqs(ctx, freqs_hz, n_freq);
    if (st != RAPTOR_OK) return st;
    if (!t_obs_host || n_frames < 1) return fail(ctx, RAPTOR_EINVAL, "need t_obs_host and n_frames >= 1");
    if (!flux_jy_host) return fail(ctx, RAPTOR_EINVAL, "flux_jy_host is NULL");
    for (int f = 0; f < n_frames; ++f)
        if (!std::isfinite(t_obs_host[f])) return fail(ctx, RAPTOR_EINVAL, "frame times must be finite");
    const bool grid = ctx->plasma.kind == RAPTOR_PLASMA_GRID_MKS2D;
    const bool fast = grid && !ctx->plasma.slow_light;
    if (fast && (first_frame < 0 || first_frame + n_frames > ctx->plasma.n_snap))
        return fail(ctx, RAPTOR_EINVAL, "fast-light frames need snapshots first_frame .. first_frame + n_frames - 1");
    const long long npix = (long long)ctx->cam.nx * ctx->cam.ny;
    if (npix * n_frames > (1LL << 40)) return fail(ctx, RAPTOR_EINVAL, "too many rays");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(ensure(ctx, &ctx->d_tframes, &ctx->tframes_cap, (size_t)n_frames));
    std::vector<double> tf(n_frames);
    for (int f = 0; f < n_frames; ++f) tf[f] = t_obs_host[f] + ctx->cam.t_delay;
    RCK(cudaMemcpyAsync(ctx->d_tframes, tf.data(), n_frames * sizeof(double), cudaMemcpyHostToDevice, s));
    double* img = images_dev;
    if (!img) {
        RCK(ensure(ctx, &ctx->d_img, &ctx->img_cap, (size_t)npix * n_freq * n_frames));
        img = ctx->d_img;
    }
    Params p = base_params(ctx);
    p.row0 = 0;
    p.n_rows = ctx->cam.ny;
    p.n_pix = (int)npix;
    p.n_rays = npix * n_frames;
    p.t_frames = ctx->d_tframes;
    p.lc_fast = fast ? 1 : 0;
    p.frame_snap0 = first_frame;
    p.image = img;
    st = run_rays_graph(ctx, p, freqs_hz, n_freq, n_freq, n_frames, s);
    if (st != RAPTOR_OK) return st;
    RCK(cudaMemcpyAsync(flux_jy_host, ctx->d_flux, (size_t)n_frames * n_freq * sizeof(double), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    return RAPTOR_OK;
}

raptor_status raptor_trace_ray(raptor_ctx* ctx, double alpha, double beta, double t_obs, const double* freqs_hz, int n_freq,
                               int max_rec, double* rec_host, int* n_steps, int* ray_status, double* intensity_host,
                               void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->has_plasma) return fail(ctx, RAPTOR_ENOPLASMA, "raptor_load_plasma has not been called");
    raptor_status st = check_freqs(ctx, freqs_hz, n_freq);
    if (st != RAPTOR_OK) return st;
    if (n_freq > 16) return fail(ctx, RAPTOR_EINVAL, "trace supports at most 16 frequencies");
    if (max_rec < 0 || (max_rec > 0 && !rec_host)) return fail(ctx, RAPTOR_EINVAL, "rec_host needed for max_rec > 0");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(t_obs)) return fail(ctx, RAPTOR_EINVAL, "non-finite ray");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(ensure(ctx, &ctx->d_rec, &ctx->rec_cap, (size_t)std::max(max_rec, 1) * 12));
    Params p = base_params(ctx);
    p.i_unscale = 1.0;
    p.nf = n_freq;
    p.nf_total = n_freq;
    for (int f = 0; f < n_freq; ++f) p.nu[f] = freqs_hz[f];
    p.snap = 0;
    const double tc = t_obs + ctx->cam.t_delay;
    ProfScope ps(ctx, kProfTrace, s);
    if (p.flags & kFlagForwardRT) {
        if (n_freq > kForwardMaxFreq) return fail(ctx, RAPTOR_EINVAL, "the forward scheme takes at most 4 frequencies");
        RCK(ensure(ctx, &ctx->d_fwd, &ctx->fwd_cap_elems, (size_t)kForwardCap * n_freq));
        p.fwd = ctx->d_fwd;
        p.fwd_cap = kForwardCap;
        p.fwd_stride = 1;
    }
    const bool verlet = (p.flags & (kFlagVerlet | kFlagVerletReeval)) != 0;
    int* ti = ctx->d_trace_int;
    if (n_freq <= 1 && !verlet)
        k_trace_fp64<1, false><<<1, 32, 0, s>>>(p, alpha, beta, tc, max_rec, ctx->d_rec, ti, ti + 1, ctx->d_trace_I);
    else if (n_freq <= 1)
        k_trace_fp64<1, true><<<1, 32, 0, s>>>(p, alpha, beta, tc, max_rec, ctx->d_rec, ti, ti + 1, ctx->d_trace_I);
    else if (!verlet)
        k_trace_fp64<16, false><<<1, 32, 0, s>>>(p, alpha, beta, tc, max_rec, ctx->d_rec, ti, ti + 1, ctx->d_trace_I);
    else
        k_trace_fp64<16, true><<<1, 32, 0, s>>>(p, alpha, beta, tc, max_rec, ctx->d_rec, ti, ti + 1, ctx->d_trace_I);
    RCK(cudaGetLastError());
    int hi[2] = {0, 0};
    RCK(cudaMemcpyAsync(hi, ctx->d_trace_int, sizeof(hi), cudaMemcpyDeviceToHost, s));
    double Ih[16];
    RCK(cudaMemcpyAsync(Ih, ctx->d_trace_I, n_freq * sizeof(double), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    const int nrec = std::min(hi[0], max_rec);
    if (nrec > 0) {
        RCK(cudaMemcpyAsync(rec_host, ctx->d_rec, (size_t)nrec * 12 * sizeof(double), cudaMemcpyDeviceToHost, s));
        RCK(cudaStreamSynchronize(s));
    }
    if (n_steps) *n_steps = hi[0];
    if (ray_status) *ray_status = hi[1];
    if (intensity_host) std::memcpy(intensity_host, Ih, n_freq * sizeof(double));
    return RAPTOR_OK;
}

raptor_status raptor_stats(raptor_ctx* ctx, unsigned long long* rays, unsigned long long* steps,
                           unsigned long long* fp64_steps, unsigned long long* truncated, unsigned long long* errors,
                           unsigned long long* fallback) {
    if (!ctx) return RAPTOR_EINVAL;
    unsigned long long h[8];
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
    if (rays) *rays = h[kStatRays];
    if (steps) *steps = h[kStatSteps];
    if (fp64_steps) *fp64_steps = h[kStatFp64Steps];
    if (truncated) *truncated = h[kStatTrunc];
    if (errors) *errors = h[kStatErr];
    if (fallback) *fallback = h[kStatFallback];
    return RAPTOR_OK;
}

raptor_status raptor_stats_reset(raptor_ctx* ctx) {
    if (!ctx) return RAPTOR_EINVAL;
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemset(ctx->d_stats, 0, kNumStats * sizeof(unsigned long long)));
    return RAPTOR_OK;
}

raptor_status raptor_stats_ex(raptor_ctx* ctx, unsigned long long* values, int count) {
    if (!ctx || !values || count < 1 || count > kNumStats) return RAPTOR_EINVAL;
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(values, ctx->d_stats, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return RAPTOR_OK;
}

const char* raptor_last_error(const raptor_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void raptor_destroy(raptor_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    cudaFree(ctx->d_grid);
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_stats);
    cudaFree(ctx->d_partial);
    cudaFree(ctx->d_flux);
    cudaFree(ctx->d_img);
    cudaFree(ctx->d_tframes);
    cudaFree(ctx->d_trace_int);
    cudaFree(ctx->d_trace_I);
    cudaFree(ctx->d_rec);
    free_mixed_queues(ctx->mq);
    cudaEvent_t evs[] = {ctx->ev_fork, ctx->ev_join, ctx->ev_tail, ctx->ev_net};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (ctx->g_exec) cudaGraphExecDestroy(ctx->g_exec);
    if (ctx->s_cap) cudaStreamDestroy(ctx->s_cap);
    if (ctx->s_long) cudaStreamDestroy(ctx->s_long);
    void* sp[] = {ctx->s_P, ctx->s_G, ctx->s_m1, ctx->s_m2, ctx->s_w, ctx->s_x, ctx->s_z1, ctx->s_z2, ctx->s_z3,
                  ctx->s_out, ctx->s_dout, ctx->s_dzf, ctx->s_dh, ctx->s_h1, ctx->s_h2, ctx->s_h3, ctx->s_dzb, ctx->s_y,
                  ctx->s_loss, ctx->s_in, ctx->s_fb, ctx->s_start, ctx->d_curve, ctx->s_err, ctx->s_h2tc,
                  ctx->d_crit, ctx->d_rest, ctx->d_hist, ctx->d_fwd, ctx->d_x2tab, ctx->x_P, ctx->x_G, ctx->x_m1,
                  ctx->x_m2, ctx->x_w, ctx->x_out, ctx->x_dout, ctx->x_y, ctx->x_list, ctx->x_nlist,
                  ctx->x_h2tc};
    for (void* q : sp) cudaFree(q);
    for (auto& e : ctx->ev_open) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->ev_t0) cudaEventDestroy(ctx->ev_t0);
    delete ctx;
}

// Launch-shape control used by the autotuner (threads per block, blocks per SM; 0 = max).

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Learned surrogate (host orchestration of raptor_surrogate.cuh)
// ---------------------------------------------------------------------------------------
namespace {

constexpr long long kSurRows = 4096;  // rows per training batch / inference chunk (multiple of 128)

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

cudaError_t sur_alloc(raptor_ctx* c) {
    cudaError_t e = cudaSuccess;
    if (!c->s_P || c->s_rows < kSurRows) c->epoch += 1;
    if (!c->s_P) {
        const size_t n = MlpLayout::SIZE;
        e = cudaMalloc((void**)&c->s_P, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_G, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_m1, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_m2, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_w, 6 * kHid * kHid * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_err, sizeof(int));
        // the tcgen05 kernels' shared-memory plans (set once, outside any stream capture)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_tc12<kOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc12Smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_tc34_state, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc34Smem);
        if (e == cudaSuccess) e = cudaMemset(c->s_err, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(c->s_G, 0, n * sizeof(float));
        if (e != cudaSuccess) return e;
    }
    if (c->s_rows < kSurRows) {
        const long long R = kSurRows;
        float** f32[] = {&c->s_z1, &c->s_z2, &c->s_z3, &c->s_dzf, &c->s_dh};
        for (float** q : f32) {
            if (e == cudaSuccess) e = cudaMalloc((void**)q, R * kHid * sizeof(float));
        }
        __nv_bfloat16** b16[] = {&c->s_h1, &c->s_h2, &c->s_h3, &c->s_dzb};
        for (__nv_bfloat16** q : b16) {
            if (e == cudaSuccess) e = cudaMalloc((void**)q, R * kHid * sizeof(__nv_bfloat16));
        }
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_x, R * kIn * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_out, R * kOut * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_dout, R * kOut * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_y, R * kOutUsed * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_loss, 1024 * sizeof(double));
        if (e == cudaSuccess) c->s_rows = R;
    }
    return e;
}

int ew_blocks(long long n) { return (int)std::min<long long>(8192, std::max<long long>(1, (n + 255) / 256)); }

__nv_bfloat16* w2b(raptor_ctx* c) { return c->s_w; }
__nv_bfloat16* w2t(raptor_ctx* c) { return c->s_w + kHid * kHid; }
__nv_bfloat16* w3b(raptor_ctx* c) { return c->s_w + 2 * kHid * kHid; }
__nv_bfloat16* w3t(raptor_ctx* c) { return c->s_w + 3 * kHid * kHid; }
__nv_bfloat16* wtc(raptor_ctx* c) { return c->s_w + 4 * kHid * kHid; }  // [2][256 x 256], operand layout

// BF16 copies of the hidden weights (GEMM layouts and the tcgen05 operand layout) from the
// FP32 master parameters.
cudaError_t refresh_weights(raptor_ctx* c, cudaStream_t s) {
    k_refresh_bf16<<<256, 256, 0, s>>>(c->s_P, w2b(c), w2t(c), w3b(c), w3t(c));
    k_tc_pack<<<256, 256, 0, s>>>(c->s_P, wtc(c));
    return cudaGetLastError();
}

// Forward pass on `rows` rows already in c->s_x (rows_valid of them real).
cudaError_t sur_forward(raptor_ctx* c, long long rows, long long rows_valid, cudaStream_t s) {
    k_mlp_layer1<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_P, c->s_x, rows, rows_valid, c->s_z1, c->s_h1);
    dim3 g(kHid / kGBN, (unsigned)(rows / kGBM));
    k_gemm_bf16<true, true><<<g, 256, 0, s>>>(c->s_h1, kHid, w2b(c), kHid, c->s_z2, kHid, rows, kHid, kHid);
    k_bias_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_z2, c->s_P + MlpLayout::B2, rows, c->s_h2);
    k_gemm_bf16<true, true><<<g, 256, 0, s>>>(c->s_h2, kHid, w3b(c), kHid, c->s_z3, kHid, rows, kHid, kHid);
    k_bias_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_z3, c->s_P + MlpLayout::B3, rows, c->s_h3);
    k_mlp_layer4<<<ew_blocks(rows * 32), 256, 0, s>>>(c->s_P, c->s_h3, rows, c->s_out);
    return cudaGetLastError();
}

// Loss and gradient of the batch in (s_x, s_y) into s_G; loss partials in s_loss[0..nb).
cudaError_t sur_backward(raptor_ctx* c, long long rows, int* nb_out, cudaStream_t s) {
    const int nb = 64;
    *nb_out = nb;
    float* G = c->s_G;
    k_mse_grad<<<nb, 256, 0, s>>>(c->s_P, c->s_out, c->s_y, rows, c->s_dout, c->s_loss);
    k_colred<float, __nv_bfloat16><<<kOut * kHid, 256, 0, s>>>(c->s_dout, kOut, c->s_h3, kHid, rows, kOut, kHid,
                                                                 G + MlpLayout::W4);
    k_colred<float, float><<<kOut, 256, 0, s>>>(nullptr, 0, c->s_dout, kOut, rows, 1, kOut, G + MlpLayout::B4);
    k_back_layer4<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_P, c->s_dout, c->s_z3, rows, c->s_dzf, c->s_dzb);
    // layer 3: dW3 = dz3^T h2, db3, dh2 = dz3 W3
    dim3 gw(kHid / kGBN, kHid / kGBM), ga(kHid / kGBN, (unsigned)(rows / kGBM));
    k_gemm_bf16<false, false><<<gw, 256, 0, s>>>(c->s_dzb, kHid, c->s_h2, kHid, G + MlpLayout::W3, kHid, kHid, kHid, rows);
    k_colred<float, float><<<kHid, 256, 0, s>>>(nullptr, 0, c->s_dzf, kHid, rows, 1, kHid, G + MlpLayout::B3);
    k_gemm_bf16<true, true><<<ga, 256, 0, s>>>(c->s_dzb, kHid, w3t(c), kHid, c->s_dh, kHid, rows, kHid, kHid);
    k_back_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_dh, c->s_z2, rows * kHid, c->s_dzf, c->s_dzb);
    // layer 2
    k_gemm_bf16<false, false><<<gw, 256, 0, s>>>(c->s_dzb, kHid, c->s_h1, kHid, G + MlpLayout::W2, kHid, kHid, kHid, rows);
    k_colred<float, float><<<kHid, 256, 0, s>>>(nullptr, 0, c->s_dzf, kHid, rows, 1, kHid, G + MlpLayout::B2);
    k_gemm_bf16<true, true><<<ga, 256, 0, s>>>(c->s_dzb, kHid, w2t(c), kHid, c->s_dh, kHid, rows, kHid, kHid);
    k_back_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_dh, c->s_z1, rows * kHid, c->s_dzf, nullptr);
    // layer 1
    k_grad_w1<<<kHid * kIn, 256, 0, s>>>(c->s_P, c->s_dzf, c->s_x, rows, G);
    k_colred<float, float><<<kHid, 256, 0, s>>>(nullptr, 0, c->s_dzf, kHid, rows, 1, kHid, G + MlpLayout::B1);
    return cudaGetLastError();
}

// Evaluate n rows of raw inputs into normalised outputs out_dev [n][kOut]: two persistent
// tcgen05 kernels (one CTA per SM, each hidden layer's weights resident in shared memory)
// or the fused mma.sync kernel.
cudaError_t sur_eval_rows(raptor_ctx* c, const float* inputs, long long n, float* out_dev, cudaStream_t s) {
    if (c->s_kernel == RAPTOR_MLP_MMA_SYNC) {
        const long long blocks = (n + kFRows - 1) / kFRows;
        k_mlp_fused<<<(unsigned)blocks, 256, 0, s>>>(c->s_P, w2b(c), w3b(c), inputs, n, out_dev);
        return cudaGetLastError();
    }
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    cudaError_t e = cudaSuccess;
    if ((size_t)tiles > c->s_h2tc_tiles) {
        c->epoch += 1;
        e = cudaFree(c->s_h2tc);
        c->s_h2tc = nullptr;
        c->s_h2tc_tiles = 0;
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->s_h2tc, (size_t)tiles * kTcTileBytes);
        if (e != cudaSuccess) return e;
        c->s_h2tc_tiles = (size_t)tiles;
    }
    const unsigned grid = (unsigned)std::min<long long>(tiles, c->num_sms);
    k_mlp_tc12<<<grid, kTcThreads, kTc12Smem, s>>>(c->s_P, wtc(c), inputs, n, c->s_h2tc, c->s_err);
    k_mlp_tc34_state<<<grid, kTcThreads, kTc34Smem, s>>>(c->s_P, wtc(c) + kHid * kHid, c->s_h2tc, n, out_dev, c->s_err);
    return cudaGetLastError();
}

// After a synchronisation: report (and clear) a tensor-core wait that ran out.
raptor_status check_tc_err(raptor_ctx* ctx) {
    if (!ctx->s_err) return RAPTOR_OK;
    int flag = 0;
    RCK(cudaMemcpy(&flag, ctx->s_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return RAPTOR_OK;
    RCK(cudaMemset(ctx->s_err, 0, sizeof(int)));
    return fail(ctx, RAPTOR_ETIMEOUT, "surrogate inference: a tensor-core wait exceeded its time limit");
}

// Critical curve on the image plane (Bardeen 1973): photon-orbit radius r gives
// xi = L/E, eta = Q/E^2; alpha = -xi / sin i, beta = +-sqrt(eta + a^2 cos^2 i - xi^2 cot^2 i).
std::vector<double> critical_curve(double a, double incl, int n) {
    std::vector<double> pts;
    const double ci = std::cos(incl), si = std::sin(incl);
    if (std::fabs(a) < 1e-6) {
        const double b = 3.0 * std::sqrt(3.0);
        for (int k = 0; k < n; ++k) {
            const double t = 2.0 * kPi * k / n;
            pts.push_back(b * std::cos(t));
            pts.push_back(b * std::sin(t));
        }
        return pts;
    }
    const double aa = std::fabs(a);
    const double rp = 2.0 * (1.0 + std::cos(2.0 / 3.0 * std::acos(-aa))), rm = 2.0 * (1.0 + std::cos(2.0 / 3.0 * std::acos(aa)));
    const int half = n / 2;
    const int fine = 16 * half;
    std::vector<double> all;
    for (int k = 0; k < fine; ++k) {
        const double r = rp + (rm - rp) * k / (fine - 1.0);
        const double xi = -(r * r * r - 3.0 * r * r + a * a * r + a * a) / (a * (r - 1.0));
        const double eta = r * r * r * (4.0 * a * a - r * (r - 3.0) * (r - 3.0)) / (a * a * (r - 1.0) * (r - 1.0));
        const double b2 = eta + a * a * ci * ci - xi * xi * ci * ci / (si * si);
        if (b2 >= 0.0) {
            all.push_back(-xi / si);
            all.push_back(std::sqrt(b2));
        }
    }
    // keep `half` evenly spaced points of the visible arc (beta >= 0), mirror to beta < 0
    const size_t na = all.size() / 2;
    std::vector<double> up;
    for (int q = 0; q < half && na > 0; ++q) {
        const size_t k = na == 1 ? 0 : (size_t)((double)q * (na - 1) / (half - 1));
        up.push_back(all[2 * k]);
        up.push_back(all[2 * k + 1]);
    }
    const size_t m = up.size() / 2;
    // closed polygon: upper arc forwards, lower arc backwards
    for (size_t q = 0; q < m; ++q) { pts.push_back(up[2 * q]); pts.push_back(up[2 * q + 1]); }
    for (size_t q = m; q-- > 0;) { pts.push_back(up[2 * q]); pts.push_back(-up[2 * q + 1]); }
    return pts;
}

}  // namespace

extern "C" {

int raptor_surrogate_param_count(void) { return MlpLayout::SIZE; }

raptor_status raptor_surrogate_generate(raptor_ctx* ctx, long long n, unsigned long long seed, double spin_min,
                                        double spin_max, double incl_min_deg, double incl_max_deg, float* inputs_dev,
                                        double* targets_dev, double* states_dev, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    if (n < 1 || !inputs_dev || !targets_dev) return fail(ctx, RAPTOR_EINVAL, "need n >= 1 and output buffers");
    if (!(spin_min >= 0.0 && spin_max >= spin_min && spin_max < 1.0)) return fail(ctx, RAPTOR_EINVAL, "spin range invalid");
    if (!(incl_min_deg > 0.0 && incl_max_deg >= incl_min_deg && incl_max_deg < 180.0))
        return fail(ctx, RAPTOR_EINVAL, "inclination range invalid");
    SurrogateRange R{ctx->cam.alpha_min, ctx->cam.alpha_max, ctx->cam.beta_min, ctx->cam.beta_max, spin_min, spin_max,
                     incl_min_deg, incl_max_deg, ctx->cam.r_cam, ctx->cam.eps, ctx->s_handoff};
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    {
        ProfScope ps(ctx, kProfTrain, s);
        k_surrogate_data<<<ctx->num_sms * 8, 128, 0, s>>>(R, seed, n, inputs_dev, targets_dev, states_dev);
    }
    RCK(cudaGetLastError());
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_init(raptor_ctx* ctx, const double* targets_dev, long long n, unsigned long long seed,
                                    void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!targets_dev || n < 2) return fail(ctx, RAPTOR_EINVAL, "need targets and n >= 2");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(sur_alloc(ctx));
    const long long m = std::min<long long>(n, 65536);
    std::vector<double> y((size_t)m * kOutUsed);
    RCK(cudaMemcpyAsync(y.data(), targets_dev, y.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    std::vector<float> P(MlpLayout::SIZE, 0.f);
    uint64_t st = seed ^ 0x5EEDull;
    auto uni = [&](double lim) { return (float)(lim * (2.0 * ((splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0)); };
    for (int i = 0; i < kHid * kIn; ++i) P[MlpLayout::W1 + i] = uni(std::sqrt(6.0 / kIn));
    for (int i = 0; i < kHid * kHid; ++i) P[MlpLayout::W2 + i] = uni(std::sqrt(6.0 / kHid));
    for (int i = 0; i < kHid * kHid; ++i) P[MlpLayout::W3 + i] = uni(std::sqrt(6.0 / kHid));
    for (int i = 0; i < kOut * kHid; ++i) P[MlpLayout::W4 + i] = uni(std::sqrt(3.0 / kHid));
    // input normalisation (scale, shift): alpha, beta over the camera; a in [0, 1]; i in degrees
    const double ha = 0.5 * (ctx->cam.alpha_max - ctx->cam.alpha_min), hb = 0.5 * (ctx->cam.beta_max - ctx->cam.beta_min);
    const float scale[4] = {(float)(1.0 / ha), (float)(1.0 / hb), 2.0f, 1.0f / 40.0f};
    const float shift[4] = {(float)(0.5 * (ctx->cam.alpha_max + ctx->cam.alpha_min)),
                            (float)(0.5 * (ctx->cam.beta_max + ctx->cam.beta_min)), 0.5f, 45.0f};
    for (int c = 0; c < 4; ++c) {
        P[MlpLayout::NORM + c] = scale[c];
        P[MlpLayout::NORM + 4 + c] = shift[c];
    }
    for (int q = 0; q < kOut; ++q) {
        double mu = 0.0, var = 0.0;
        if (q < kOutUsed) {
            for (long long i = 0; i < m; ++i) mu += y[i * kOutUsed + q];
            mu /= m;
            for (long long i = 0; i < m; ++i) var += (y[i * kOutUsed + q] - mu) * (y[i * kOutUsed + q] - mu);
            var /= (m - 1);
        }
        P[MlpLayout::NORM + 8 + q] = (float)mu;
        P[MlpLayout::NORM + 16 + q] = (float)std::max(std::sqrt(var), 1e-6);
    }
    P[MlpLayout::HANDOFF] = (float)ctx->s_handoff;  // the network carries its hand-off step count
    ctx->s_handoff_net = ctx->s_handoff;
    RCK(cudaMemcpyAsync(ctx->s_P, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RCK(cudaMemsetAsync(ctx->s_m1, 0, MlpLayout::SIZE * sizeof(float), s));
    RCK(cudaMemsetAsync(ctx->s_m2, 0, MlpLayout::SIZE * sizeof(float), s));
    RCK(refresh_weights(ctx, s));
    RCK(cudaGetLastError());
    RCK(cudaStreamSynchronize(s));
    ctx->s_step = 0;
    ctx->sur_ready = true;
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_train(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                     int steps, double lr, double lr_final, unsigned long long seed, double* loss_host,
                                     void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!ctx->sur_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "surrogate not initialised");
    if (!inputs_dev || !targets_dev || n < 1 || steps < 1 || !(lr > 0.0) || !(lr_final > 0.0))
        return fail(ctx, RAPTOR_EINVAL, "invalid training arguments");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(sur_alloc(ctx));
    const float b1 = 0.9f, b2 = 0.999f;
    ProfScope ps(ctx, kProfTrain, s);
    for (int it = 0; it < steps; ++it) {
        k_gather_batch<<<ew_blocks(kSurRows), 256, 0, s>>>(inputs_dev, targets_dev, n, kSurRows, seed, (long long)ctx->s_step,
                                                          ctx->s_x, ctx->s_y);
        RCK(sur_forward(ctx, kSurRows, kSurRows, s));
        int nb = 0;
        RCK(sur_backward(ctx, kSurRows, &nb, s));
        ctx->s_step += 1;
        // cosine decay from lr to lr_final; Adam bias corrections folded into the step size
        const double frac = steps > 1 ? (double)it / (steps - 1) : 1.0;
        const double lr_it = lr_final + 0.5 * (lr - lr_final) * (1.0 + std::cos(kPi * frac));
        const double t = (double)ctx->s_step;
        const float lr_t = (float)(lr_it * std::sqrt(1.0 - std::pow(b2, t)) / (1.0 - std::pow(b1, t)));
        k_adam<<<ew_blocks(MlpLayout::NORM), 256, 0, s>>>(ctx->s_P, ctx->s_G, ctx->s_m1, ctx->s_m2, MlpLayout::NORM, lr_t, b1,
                                                         b2, 1e-8f);
        RCK(refresh_weights(ctx, s));
        RCK(cudaGetLastError());
        if (loss_host) {
            double parts[64];
            RCK(cudaMemcpyAsync(parts, ctx->s_loss, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
            RCK(cudaStreamSynchronize(s));
            double L = 0.0;
            for (int q = 0; q < nb; ++q) L += parts[q];
            loss_host[it] = L / (double)(kSurRows * kOutUsed);
        }
    }
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_grad(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                    float* grad_host, double* loss_host, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!ctx->sur_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "surrogate not initialised");
    if (!inputs_dev || !targets_dev || n < 1 || n > kSurRows || n % kGBM != 0)
        return fail(ctx, RAPTOR_EINVAL, "n must be a multiple of 128 and at most 4096");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(cudaMemcpyAsync(ctx->s_x, inputs_dev, n * kIn * sizeof(float), cudaMemcpyDeviceToDevice, s));
    RCK(cudaMemcpyAsync(ctx->s_y, targets_dev, n * kOutUsed * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RCK(sur_forward(ctx, n, n, s));
    int nb = 0;
    RCK(sur_backward(ctx, n, &nb, s));
    if (grad_host) RCK(cudaMemcpyAsync(grad_host, ctx->s_G, MlpLayout::NORM * sizeof(float), cudaMemcpyDeviceToHost, s));
    double parts[64];
    RCK(cudaMemcpyAsync(parts, ctx->s_loss, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    if (loss_host) {
        double L = 0.0;
        for (int q = 0; q < nb; ++q) L += parts[q];
        *loss_host = L / (double)(n * kOutUsed);
    }
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_eval(raptor_ctx* ctx, const float* inputs_dev, long long n, double* pred_dev, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!ctx->sur_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "surrogate not initialised");
    if (!inputs_dev || !pred_dev || n < 1) return fail(ctx, RAPTOR_EINVAL, "invalid arguments");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    float* out = nullptr;
    RCK(cudaMallocAsync((void**)&out, n * kOut * sizeof(float), s));
    cudaError_t e = sur_eval_rows(ctx, inputs_dev, n, out, s);
    std::vector<float> Pn(24);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Pn.data(), ctx->s_P + MlpLayout::NORM, 24 * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<float> o;
    if (e == cudaSuccess) {
        o.resize((size_t)n * kOut);
        e = cudaMemcpyAsync(o.data(), out, o.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFreeAsync(out, s);
    if (e != cudaSuccess) return fail(ctx, RAPTOR_ECUDA, cudaGetErrorString(e));
    const raptor_status te = check_tc_err(ctx);
    if (te != RAPTOR_OK) return te;
    std::vector<double> pr((size_t)n * kOutUsed);
    for (long long i = 0; i < n; ++i)
        for (int q = 0; q < kOutUsed; ++q)
            pr[i * kOutUsed + q] = (double)o[i * kOut + q] * (double)Pn[16 + q] + (double)Pn[8 + q];
    RCK(cudaMemcpyAsync(pred_dev, pr.data(), pr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    RCK(cudaStreamSynchronize(s));
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_get(raptor_ctx* ctx, float* params_host, int n) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!ctx->sur_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "surrogate not initialised");
    if (!params_host || n != MlpLayout::SIZE) return fail(ctx, RAPTOR_EINVAL, "n must equal raptor_surrogate_param_count()");
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(params_host, ctx->s_P, n * sizeof(float), cudaMemcpyDeviceToHost));
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_set(raptor_ctx* ctx, const float* params_host, int n) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!params_host || n != MlpLayout::SIZE) return fail(ctx, RAPTOR_EINVAL, "n must equal raptor_surrogate_param_count()");
    // hand-off step count stored with the parameters (0: a network written before the count
    // was stored, trained for the default)
    const float hf = params_host[MlpLayout::HANDOFF];
    if (!(hf == 0.f || (hf >= 1.f && hf <= (float)kMaxHandoffSteps && hf == std::floor(hf))))
        return fail(ctx, RAPTOR_EINVAL, "the parameters' hand-off step count is not an integer in [1, 1000]");
    ctx->s_handoff_net = hf == 0.f ? kSurrogateSteps : (int)hf;
    RCK(sur_alloc(ctx));
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(ctx->s_P, params_host, n * sizeof(float), cudaMemcpyHostToDevice));
    RCK(cudaMemset(ctx->s_m1, 0, n * sizeof(float)));
    RCK(cudaMemset(ctx->s_m2, 0, n * sizeof(float)));
    RCK(refresh_weights(ctx, nullptr));
    RCK(cudaGetLastError());
    RCK(cudaDeviceSynchronize());
    ctx->sur_ready = true;
    ctx->s_step = 0;
    return RAPTOR_OK;
}

// File format of a saved surrogate: 8-byte magic, u32 format version, u32 parameter count,
// the FP32 parameters (little-endian, MlpLayout order), u64 FNV-1a hash of those bytes.
constexpr char kSurMagic[8] = {'R', 'A', 'P', 'T', 'M', 'L', 'P', '1'};
constexpr uint32_t kSurVersion = 1;

static uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
    return h;
}

raptor_status raptor_surrogate_save(raptor_ctx* ctx, const char* path) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!path) return fail(ctx, RAPTOR_EINVAL, "path is NULL");
    std::vector<float> P(MlpLayout::SIZE);
    raptor_status st = raptor_surrogate_get(ctx, P.data(), MlpLayout::SIZE);
    if (st != RAPTOR_OK) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ctx, RAPTOR_EINVAL, std::string("cannot open for writing: ") + path);
    const uint32_t hdr[2] = {kSurVersion, (uint32_t)MlpLayout::SIZE};
    const uint64_t h = fnv1a(reinterpret_cast<const unsigned char*>(P.data()), P.size() * sizeof(float));
    bool ok = std::fwrite(kSurMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(P.data(), sizeof(float), P.size(), f) == P.size() && std::fwrite(&h, sizeof(h), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? RAPTOR_OK : fail(ctx, RAPTOR_EINVAL, std::string("write failed: ") + path);
}

raptor_status raptor_surrogate_load(raptor_ctx* ctx, const char* path) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!path) return fail(ctx, RAPTOR_EINVAL, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, RAPTOR_EINVAL, std::string("cannot open: ") + path);
    char magic[8];
    uint32_t hdr[2] = {0, 0};
    std::vector<float> P(MlpLayout::SIZE);
    uint64_t h = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kSurMagic, 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kSurVersion && hdr[1] == (uint32_t)MlpLayout::SIZE &&
              std::fread(P.data(), sizeof(float), P.size(), f) == P.size() && std::fread(&h, sizeof(h), 1, f) == 1;
    char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the hash
    std::fclose(f);
    if (!ok || h != fnv1a(reinterpret_cast<const unsigned char*>(P.data()), P.size() * sizeof(float)))
        return fail(ctx, RAPTOR_EINVAL, std::string("not a surrogate file of this version, or damaged: ") + path);
    return raptor_surrogate_set(ctx, P.data(), MlpLayout::SIZE);
}

raptor_status raptor_mixed_config(raptor_ctx* ctx, double crit_band, int n_passes, const int* budgets, int tail_split) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!(crit_band >= 0.0) || !std::isfinite(crit_band)) return fail(ctx, RAPTOR_EINVAL, "crit_band must be finite and >= 0");
    if (n_passes < 1 || n_passes > kMaxPasses) return fail(ctx, RAPTOR_EINVAL, "n_passes must lie in [1, 8]");
    if (budgets)
        for (int k = 0; k + 1 < n_passes; ++k)
            if (budgets[k] < 1) return fail(ctx, RAPTOR_EINVAL, "pass budgets must be >= 1");
    if (tail_split < 0) return fail(ctx, RAPTOR_EINVAL, "tail_split must be >= 0");
    ctx->crit_band = crit_band;
    ctx->tail_split = tail_split;
    ctx->n_passes = budgets ? n_passes : kMaxPasses;
    for (int k = 0; k < kMaxPasses; ++k) ctx->pass_budget[k] = budgets ? (k + 1 < n_passes ? budgets[k] : (1 << 30)) : kPassBudget[k];
    return RAPTOR_OK;
}

raptor_status raptor_long_config(raptor_ctx* ctx, int threads_per_block, int n_passes, const int* budgets) {
    if (!ctx) return RAPTOR_EINVAL;
    if (threads_per_block < 0 || threads_per_block > 128 || threads_per_block % 32)
        return fail(ctx, RAPTOR_EINVAL, "threads_per_block must be 0, 32, 64, 96 or 128");
    if (n_passes < 1 || n_passes > kMaxPasses) return fail(ctx, RAPTOR_EINVAL, "n_passes must lie in [1, 8]");
    if (n_passes > 1 && !budgets) return fail(ctx, RAPTOR_EINVAL, "budgets must be given for n_passes > 1");
    for (int k = 0; k + 1 < n_passes; ++k)
        if (budgets[k] < 1) return fail(ctx, RAPTOR_EINVAL, "pass budgets must be >= 1");
    ctx->long_block = threads_per_block;
    ctx->long_passes = n_passes;
    for (int k = 0; k < kMaxPasses; ++k) ctx->long_budget[k] = k + 1 < n_passes ? budgets[k] : (1 << 30);
    return RAPTOR_OK;
}

raptor_status raptor_graph_config(raptor_ctx* ctx, int enable) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->graphs = enable != 0;
    if (!ctx->graphs && ctx->g_exec) {
        cudaGraphExecDestroy(ctx->g_exec);
        ctx->g_exec = nullptr;
        ctx->g_key.clear();
    }
    ctx->g_seen.clear();
    return RAPTOR_OK;
}

raptor_status raptor_graph_stats(raptor_ctx* ctx, long long* captures, long long* replays) {
    if (!ctx) return RAPTOR_EINVAL;
    if (captures) *captures = ctx->g_captures;
    if (replays) *replays = ctx->g_replays;
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_kernel(raptor_ctx* ctx, int kind) {
    if (!ctx) return RAPTOR_EINVAL;
    if (kind != RAPTOR_MLP_TCGEN05 && kind != RAPTOR_MLP_MMA_SYNC) return fail(ctx, RAPTOR_EINVAL, "unknown surrogate kernel");
    ctx->s_kernel = kind;
    return RAPTOR_OK;
}

raptor_status raptor_inject_fault(raptor_ctx* ctx, int kind) {
    if (!ctx) return RAPTOR_EINVAL;
    if (kind != RAPTOR_FAULT_TC_WAIT) return fail(ctx, RAPTOR_EINVAL, "unknown fault kind");
    if (!ctx->s_err) return fail(ctx, RAPTOR_EUNSUPPORTED, "no surrogate network: nothing waits on the tensor cores");
    // the value a bounded wait of the tensor-core kernels leaves when it runs out
    const int flag = 1;
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(ctx->s_err, &flag, sizeof(int), cudaMemcpyHostToDevice));
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_handoff(raptor_ctx* ctx, int n_steps) {
    if (!ctx) return RAPTOR_EINVAL;
    if (n_steps < 1 || n_steps > kMaxHandoffSteps) return fail(ctx, RAPTOR_EINVAL, "n_steps must lie in [1, 1000]");
    ctx->s_handoff = n_steps;
    return RAPTOR_OK;
}

raptor_status raptor_surrogate_config(raptor_ctx* ctx, double fallback_band, double r_exit) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!(fallback_band >= 0.0) || !std::isfinite(fallback_band) || !(r_exit >= 0.0) || !std::isfinite(r_exit))
        return fail(ctx, RAPTOR_EINVAL, "fallback_band and r_exit must be finite and >= 0");
    ctx->s_band = fallback_band;
    ctx->s_r_exit = r_exit;
    return RAPTOR_OK;
}

}  // extern "C"

namespace {

// RAPTOR_MIXED_MLP: predicted start states for every non-fallback ray, then the mixed path.
// Buffers and launch parameters of a learned render (the kernels run in surrogate_prepare and
// surrogate_infer).
raptor_status prepare_surrogate_render(raptor_ctx* ctx, Params& p, cudaStream_t s) {
    if (!ctx->sur_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "RAPTOR_MIXED_MLP needs a trained or loaded surrogate");
    RCK(sur_alloc(ctx));
    const size_t rays = (size_t)p.n_rays;
    if (ctx->s_ray_cap < rays) {
        ctx->epoch += 1;
        cudaFree(ctx->s_in);
        cudaFree(ctx->s_fb);
        cudaFree(ctx->s_start);
        ctx->s_in = nullptr;
        ctx->s_fb = nullptr;
        ctx->s_start = nullptr;
        ctx->s_ray_cap = 0;
        RCK(cudaMalloc((void**)&ctx->s_in, rays * kIn * sizeof(float)));
        RCK(cudaMalloc((void**)&ctx->s_fb, rays));
        RCK(cudaMalloc((void**)&ctx->s_start, rays * 8 * sizeof(float2)));
        ctx->s_ray_cap = rays;
    }
    RCK(upload_curve(ctx, p, s));
    p.start_xk = ctx->s_start;
    p.fallback = ctx->s_fb;
    p.start_n = ctx->s_handoff_net;
    p.r_exit = ctx->s_r_exit;
    p.r_exit_f = (float)ctx->s_r_exit;
    return RAPTOR_OK;
}

// The surrogate's part of a learned render on stream s, as two launch sequences:
// surrogate_prepare writes the network inputs and the fallback flags; surrogate_infer runs
// the network and rebuilds the start states.
cudaError_t surrogate_prepare(raptor_ctx* ctx, const Params& p, cudaStream_t s) {
    const size_t rays = (size_t)p.n_rays;
    const float grow = (float)ctx->s_band + 1e-3f;
    const float4 box = make_float4(ctx->curve_box.x - grow, ctx->curve_box.y + grow, ctx->curve_box.z - grow,
                                   ctx->curve_box.w + grow);
    ProfScope ps(ctx, kProfSurrogate, s);
    k_surrogate_prepare<<<ew_blocks((long long)rays), 256, 0, s>>>(p, ctx->d_curve, ctx->n_curve, (float)ctx->s_band, box,
                                                                   ctx->s_in, ctx->s_fb, ctx->d_stats + kStatFallback);
    return cudaGetLastError();
}

cudaError_t surrogate_infer(raptor_ctx* ctx, const Params& p, cudaStream_t s) {
    const size_t rays = (size_t)p.n_rays;
    float* out = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&out, rays * kOut * sizeof(float), s);
    if (e != cudaSuccess) return e;
    {
        ProfScope pm(ctx, kProfSurrogateMlp, s, ctx->s_kernel == RAPTOR_MLP_MMA_SYNC ? 1 : 2);
        e = sur_eval_rows(ctx, ctx->s_in, (long long)rays, out, s);
    }
    if (e == cudaSuccess) {
        ProfScope ps(ctx, kProfSurrogate, s);
        k_surrogate_states<<<ew_blocks((long long)rays), 256, 0, s>>>(p, ctx->s_P, out, ctx->s_start);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(out, s);
    return e != cudaSuccess ? e : ef;
}

}  // namespace

extern "C" {

raptor_status raptor_set_launch(raptor_ctx* ctx, int threads_per_block, int blocks_per_sm, int blocks_per_sm_fp64) {
    if (!ctx) return RAPTOR_EINVAL;
    if (threads_per_block < 32 || threads_per_block > 128 || threads_per_block % 32)
        return fail(ctx, RAPTOR_EINVAL, "threads_per_block must be 32, 64, 96 or 128");
    if (blocks_per_sm < 0 || blocks_per_sm > 64 || blocks_per_sm_fp64 < 0 || blocks_per_sm_fp64 > 64)
        return fail(ctx, RAPTOR_EINVAL, "blocks per SM must lie in [0, 64]");
    ctx->launch_block = threads_per_block;
    ctx->launch_bps = blocks_per_sm;
    ctx->launch_bps64 = blocks_per_sm_fp64;
    return RAPTOR_OK;
}

// ---------------------------------------------------------------------------------------
// Allocation-free rendering (raptor_render_noalloc).
//
// For callers that cannot allocate device memory (a host program whose pool already owns
// the GPU's memory, or a path that must not call cudaMalloc/cudaFree after start-up since
// those calls can synchronise the device).  The FP64 persistent kernel and the flux
// reduction need scratch beyond their inputs and outputs: the ray counter, the stats
// counters and the partial flux sums.  Here they live in one file-scope device array,
// g_noalloc_scratch, of RAPTOR_NOALLOC_SCRATCH_BYTES per device, held until the process
// exits and shared by every call.  In host code the symbol is only a stand-in: its device
// address is looked up once per device, with that device current, on the first call.
// ---------------------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocCounterOff = 0;    // 8 x u64 ray/phase counters
constexpr size_t kNoAllocStatsOff = 256;    // 8 x u64 stats
constexpr size_t kNoAllocPartialOff = 512;  // [RAPTOR_NOALLOC_MAX_FREQ][256] partial flux sums
constexpr int kNoAllocChunks = 256;
constexpr size_t kNoAllocBytes = kNoAllocPartialOff + sizeof(double) * RAPTOR_NOALLOC_MAX_FREQ * kNoAllocChunks;
static_assert(kNoAllocBytes == RAPTOR_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Every kernel the allocation-free path may launch.  With lazy module loading a kernel's
// code is loaded onto the device on its first use, which can allocate device memory in the
// driver; querying its attributes loads it too, so the first call per device loads them all.
static cudaError_t noalloc_load_kernels() {
    const void* fns[] = {(const void*)k_render_fp64<1, false>, (const void*)k_render_fp64<2, false>,
                         (const void*)k_render_fp64<4, false>, (const void*)k_render_fp64<8, false>,
                         (const void*)k_render_fp64<16, false>, (const void*)k_render_fp64<1, true>,
                         (const void*)k_render_fp64<2, true>, (const void*)k_render_fp64<4, true>,
                         (const void*)k_render_fp64<8, true>, (const void*)k_render_fp64<16, true>,
                         (const void*)k_reduce_partial, (const void*)k_reduce_final};
    for (const void* f : fns) {
        cudaFuncAttributes attr;
        const cudaError_t e = cudaFuncGetAttributes(&attr, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Device address of the scratch array on device `dev` (which must be current); the first
// call per device also loads the kernels this path launches.
static cudaError_t noalloc_scratch(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = noalloc_load_kernels();
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

raptor_status raptor_render_noalloc(const raptor_camera_desc* cam, const raptor_plasma_desc* plasma, const double* freqs_hz,
                                    int n_freq, double t_obs, double* image_dev, double* flux_dev, void* stream) {
    if (!validate_camera(cam).empty() || !validate_plasma(plasma).empty()) return RAPTOR_EINVAL;
    if (cam->precision != RAPTOR_FP64) return RAPTOR_EINVAL;
    if (cam->flags & RAPTOR_FLAG_FORWARD_RT) return RAPTOR_EUNSUPPORTED;  // needs a record buffer
    if (plasma->kind != RAPTOR_PLASMA_ANALYTIC) return RAPTOR_EUNSUPPORTED;
    if (!freqs_hz || n_freq < 1 || n_freq > RAPTOR_NOALLOC_MAX_FREQ || !image_dev || !std::isfinite(t_obs))
        return RAPTOR_EINVAL;
    for (int f = 0; f < n_freq; ++f)
        if (!finite_pos(freqs_hz[f])) return RAPTOR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RAPTOR_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return RAPTOR_EINVAL;
    void* scratch = nullptr;
    if (noalloc_scratch(dev, &scratch) != cudaSuccess) return RAPTOR_ECUDA;
    unsigned char* base = static_cast<unsigned char*>(scratch);
    // A stack context that only borrows the scratch: no device memory is allocated.
    raptor_ctx tmp;
    tmp.cam = *cam;
    tmp.plasma = *plasma;
    tmp.plasma.fields = nullptr;
    tmp.has_plasma = true;
    tmp.device = dev;
    if (cudaDeviceGetAttribute(&tmp.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RAPTOR_ECUDA;
    tmp.d_counters = reinterpret_cast<unsigned long long*>(base + kNoAllocCounterOff);
    tmp.d_stats = reinterpret_cast<unsigned long long*>(base + kNoAllocStatsOff);
    double* partial = reinterpret_cast<double*>(base + kNoAllocPartialOff);
    cudaStream_t s = (cudaStream_t)stream;
    Params p = base_params(&tmp);
    p.row0 = 0;
    p.n_rows = cam->ny;
    p.n_pix = cam->nx * cam->ny;
    p.n_rays = p.n_pix;
    p.t_cam = t_obs + cam->t_delay;
    p.snap = 0;
    p.image = image_dev;
    p.i_unscale = 1.0;
    p.nf_total = n_freq;
    cudaError_t e = cudaMemsetAsync(tmp.d_stats, 0, 8 * sizeof(unsigned long long), s);
    for (int f0 = 0; f0 < n_freq && e == cudaSuccess; f0 += 16) {
        p.f_off = f0;
        p.nf = std::min(16, n_freq - f0);
        for (int f = 0; f < p.nf; ++f) p.nu[f] = freqs_hz[f0 + f];
        e = cudaMemsetAsync(tmp.d_counters, 0, 8 * sizeof(unsigned long long), s);  // ray counter starts at zero
        if (e == cudaSuccess) e = launch_fp64(&tmp, p, s);
    }
    if (e == cudaSuccess) {
        const long long len = (long long)p.n_rows * p.nx;
        const int chunks = (int)std::min<long long>(kNoAllocChunks, std::max<long long>(1, len / 4096));
        k_reduce_partial<<<dim3(chunks, n_freq), kRedThreads, 0, s>>>(image_dev, len, chunks, partial);
        e = cudaGetLastError();
        if (e == cudaSuccess && flux_dev) {
            k_reduce_final<<<n_freq, kRedThreads, 0, s>>>(partial, chunks, flux_dev);
            e = cudaGetLastError();
        }
    }
    tmp.d_counters = nullptr;
    tmp.d_stats = nullptr;
    return e == cudaSuccess ? RAPTOR_OK : RAPTOR_ECUDA;
}

raptor_status raptor_autotune(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs, int* best_block,
                              int* best_bps, int* best_bps64, double* best_ms, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    if (!ctx->has_plasma) return fail(ctx, RAPTOR_ENOPLASMA, "raptor_load_plasma has not been called");
    raptor_status st = check_freqs(ctx, freqs_hz, n_freq);
    if (st != RAPTOR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)n_freq * ctx->cam.nx * ctx->cam.ny;
    RCK(ensure(ctx, &ctx->d_img, &ctx->img_cap, n));
    const bool mixed = ctx->cam.precision == RAPTOR_MIXED;
    const int blocks[2] = {64, 128};
    const int bpss[4] = {0, 2, 3, 4};
    const int bps64s[4] = {1, 2, 3, 4};
    const int n64 = mixed ? 4 : 1;
    cudaEvent_t a = nullptr, b = nullptr;
    RCK(cudaEventCreate(&a));
    RCK(cudaEventCreate(&b));
    double best = 1e300;
    int bb = ctx->launch_block, bp = ctx->launch_bps, b64 = ctx->launch_bps64;
    const bool prof = ctx->prof;
    ctx->prof = false;
    for (int tb : blocks) {
        for (int bps : bpss) {
            if (tb == 64 && bps > 0) continue;  // 64-thread blocks only at occupancy maximum
            for (int k = 0; k < n64; ++k) {
                ctx->launch_block = tb;
                ctx->launch_bps = tb == 64 ? 2 * bps : bps;
                ctx->launch_bps64 = mixed ? (tb == 64 ? 2 * bps64s[k] : bps64s[k]) : ctx->launch_bps64;
                float t_best = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(a, s);
                    st = raptor_render(ctx, freqs_hz, n_freq, t_obs, ctx->d_img, nullptr, stream);
                    cudaEventRecord(b, s);
                    if (st != RAPTOR_OK) break;
                    if (cudaEventSynchronize(b) != cudaSuccess) { st = RAPTOR_ECUDA; break; }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, a, b);
                    t_best = std::min(t_best, t);
                }
                if (st != RAPTOR_OK) break;
                if (t_best < best) {
                    best = t_best;
                    bb = ctx->launch_block;
                    bp = ctx->launch_bps;
                    b64 = ctx->launch_bps64;
                }
            }
            if (st != RAPTOR_OK) break;
        }
        if (st != RAPTOR_OK) break;
    }
    ctx->prof = prof;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launch_block = bb;
    ctx->launch_bps = bp;
    ctx->launch_bps64 = b64;
    if (st != RAPTOR_OK) return st;
    if (best_block) *best_block = bb;
    if (best_bps) *best_bps = bp;
    if (best_bps64) *best_bps64 = b64;
    if (best_ms) *best_ms = best;
    return RAPTOR_OK;
}

raptor_status raptor_profile(raptor_ctx* ctx, int enable) {
    if (!ctx) return RAPTOR_EINVAL;
    if (enable) {
        RCK(cudaStreamSynchronize(ctx->last_stream));
        for (auto& e : ctx->ev_open) {
            ctx->ev_pool.push_back(e.a);
            ctx->ev_pool.push_back(e.b);
        }
        ctx->ev_open.clear();
        ctx->timeline.clear();
        ctx->t0_pending = true;
        for (int i = 0; i < kProfSlots; ++i) {
            ctx->prof_ms[i] = 0.0;
            ctx->prof_launches[i] = 0;
        }
    }
    ctx->prof = enable != 0;
    return RAPTOR_OK;
}

// Wait for the recorded scopes, add their durations to the slots and append them to the
// timeline (start relative to the origin event).
static raptor_status drain_profile(raptor_ctx* ctx) {
    constexpr size_t kTimelineCap = 1 << 16;
    for (auto& e : ctx->ev_open) {
        RCK(cudaEventSynchronize(e.b));
        float t = 0.f, t0 = 0.f;
        RCK(cudaEventElapsedTime(&t, e.a, e.b));
        if (ctx->ev_t0) RCK(cudaEventElapsedTime(&t0, ctx->ev_t0, e.a));
        ctx->prof_ms[e.slot] += t;
        if (ctx->timeline.size() < kTimelineCap) ctx->timeline.push_back({e.slot, e.lane, (double)t0, (double)t});
        ctx->ev_pool.push_back(e.a);
        ctx->ev_pool.push_back(e.b);
    }
    ctx->ev_open.clear();
    return RAPTOR_OK;
}

raptor_status raptor_profile_timeline(raptor_ctx* ctx, int cap, int* slot, int* lane, double* start_ms, double* dur_ms,
                                      int* count) {
    if (!ctx || cap < 0 || !count || (cap > 0 && (!slot || !lane || !start_ms || !dur_ms))) return RAPTOR_EINVAL;
    raptor_status st = drain_profile(ctx);
    if (st != RAPTOR_OK) return st;
    const int n = (int)ctx->timeline.size();
    for (int i = 0; i < n && i < cap; ++i) {
        slot[i] = ctx->timeline[i].slot;
        lane[i] = ctx->timeline[i].lane;
        start_ms[i] = ctx->timeline[i].start_ms;
        dur_ms[i] = ctx->timeline[i].dur_ms;
    }
    *count = n;
    return RAPTOR_OK;
}

raptor_status raptor_profile_read(raptor_ctx* ctx, double* ms, long long* launches) {
    if (!ctx) return RAPTOR_EINVAL;
    raptor_status st = drain_profile(ctx);
    if (st != RAPTOR_OK) return st;
    for (int i = 0; i < kProfSlots; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (launches) launches[i] = ctx->prof_launches[i];
    }
    return RAPTOR_OK;
}

raptor_status raptor_check_fp32_math(long long n, unsigned int* max_ulp) {
    if (n < 1 || !max_ulp) return RAPTOR_EINVAL;
    unsigned int* d = nullptr;
    if (cudaMalloc(&d, 5 * sizeof(unsigned int)) != cudaSuccess) return RAPTOR_ENOMEM;
    cudaError_t e = cudaMemset(d, 0, 5 * sizeof(unsigned int));
    if (e == cudaSuccess) {
        k_check_fp32_math<<<256, 256>>>(n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(max_ulp, d, 5 * sizeof(unsigned int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? RAPTOR_OK : RAPTOR_ECUDA;
}

raptor_status raptor_measure_fma_peak(int fp64, double* tflops) {
    if (!tflops) return RAPTOR_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RAPTOR_ECUDA;
    const int threads = 256, blocks = sms * 8;
    const int iters = fp64 ? 2048 : 65536;
    void* out = nullptr;
    if (cudaMalloc(&out, (size_t)threads * blocks * sizeof(double)) != cudaSuccess) return RAPTOR_ENOMEM;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        if (fp64) k_fma_peak<double><<<blocks, threads>>>((double*)out, iters, 1.0);
        else k_fma_peak<float><<<blocks, threads>>>((float*)out, iters, 1.0f);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        if (rep > 0) best = std::min(best, t);
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return RAPTOR_ECUDA;
    *tflops = 2.0 * 16.0 * iters * (double)threads * blocks / (best * 1e-3) / 1e12;
    return RAPTOR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Crossing network: the learned surrogate's equatorial outputs (raptor_crossings.cuh).  The
// same hidden layers and kernels as the state network with a 16-wide output layer; it uses
// the state network's work buffers (sur_alloc) and its own parameters and output buffers.
// ---------------------------------------------------------------------------------------
namespace {

cudaError_t x_alloc(raptor_ctx* c) {
    cudaError_t e = sur_alloc(c);
    if (e != cudaSuccess) return e;
    if (!c->x_P) {
        const size_t n = XLayout::SIZE;
        float** f[] = {&c->x_P, &c->x_G, &c->x_m1, &c->x_m2};
        for (float** q : f)
            if (e == cudaSuccess) e = cudaMalloc((void**)q, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->x_w, 6 * kHid * kHid * sizeof(__nv_bfloat16));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_tc12<kXOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc12Smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_tc34<kXOut>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc34_smem<kXOut>());
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->x_out, kSurRows * kXOut * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->x_dout, kSurRows * kXOut * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->x_y, kSurRows * kXOut * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(c->x_G, 0, n * sizeof(float));
    }
    return e;
}

// w2, w2t, w3, w3t, then w2, w3 in the tcgen05 operand layout
__nv_bfloat16* xw(raptor_ctx* c, int i) { return c->x_w + (size_t)i * kHid * kHid; }

cudaError_t x_refresh(raptor_ctx* c, cudaStream_t s) {
    k_refresh_bf16<<<256, 256, 0, s>>>(c->x_P, xw(c, 0), xw(c, 1), xw(c, 2), xw(c, 3));
    k_tc_pack<<<256, 256, 0, s>>>(c->x_P, xw(c, 4));
    return cudaGetLastError();
}

// Forward pass of the crossing network on `rows` rows in c->s_x.
cudaError_t x_forward(raptor_ctx* c, long long rows, cudaStream_t s) {
    k_mlp_layer1<kXOut><<<ew_blocks(rows * kHid), 256, 0, s>>>(c->x_P, c->s_x, rows, rows, c->s_z1, c->s_h1);
    dim3 g(kHid / kGBN, (unsigned)(rows / kGBM));
    k_gemm_bf16<true, true><<<g, 256, 0, s>>>(c->s_h1, kHid, xw(c, 0), kHid, c->s_z2, kHid, rows, kHid, kHid);
    k_bias_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_z2, c->x_P + XLayout::B2, rows, c->s_h2);
    k_gemm_bf16<true, true><<<g, 256, 0, s>>>(c->s_h2, kHid, xw(c, 2), kHid, c->s_z3, kHid, rows, kHid, kHid);
    k_bias_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_z3, c->x_P + XLayout::B3, rows, c->s_h3);
    k_mlp_layer4<kXOut><<<ew_blocks(rows * 32), 256, 0, s>>>(c->x_P, c->s_h3, rows, c->x_out);
    return cudaGetLastError();
}

// Loss and gradient of the batch in (s_x, x_y) into x_G; loss partials in s_loss[0..nb).
cudaError_t x_backward(raptor_ctx* c, long long rows, int* nb_out, cudaStream_t s) {
    const int nb = 64;
    *nb_out = nb;
    float* G = c->x_G;
    k_cross_grad<<<nb, 256, 0, s>>>(c->x_P, c->x_out, c->x_y, rows, c->x_dout, c->s_loss);
    k_colred<float, __nv_bfloat16><<<kXOut * kHid, 256, 0, s>>>(c->x_dout, kXOut, c->s_h3, kHid, rows, kXOut, kHid,
                                                                  G + XLayout::W4);
    k_colred<float, float><<<kXOut, 256, 0, s>>>(nullptr, 0, c->x_dout, kXOut, rows, 1, kXOut, G + XLayout::B4);
    k_back_layer4<kXOut><<<ew_blocks(rows * kHid), 256, 0, s>>>(c->x_P, c->x_dout, c->s_z3, rows, c->s_dzf, c->s_dzb);
    dim3 gw(kHid / kGBN, kHid / kGBM), ga(kHid / kGBN, (unsigned)(rows / kGBM));
    k_gemm_bf16<false, false><<<gw, 256, 0, s>>>(c->s_dzb, kHid, c->s_h2, kHid, G + XLayout::W3, kHid, kHid, kHid, rows);
    k_colred<float, float><<<kHid, 256, 0, s>>>(nullptr, 0, c->s_dzf, kHid, rows, 1, kHid, G + XLayout::B3);
    k_gemm_bf16<true, true><<<ga, 256, 0, s>>>(c->s_dzb, kHid, xw(c, 3), kHid, c->s_dh, kHid, rows, kHid, kHid);
    k_back_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_dh, c->s_z2, rows * kHid, c->s_dzf, c->s_dzb);
    k_gemm_bf16<false, false><<<gw, 256, 0, s>>>(c->s_dzb, kHid, c->s_h1, kHid, G + XLayout::W2, kHid, kHid, kHid, rows);
    k_colred<float, float><<<kHid, 256, 0, s>>>(nullptr, 0, c->s_dzf, kHid, rows, 1, kHid, G + XLayout::B2);
    k_gemm_bf16<true, true><<<ga, 256, 0, s>>>(c->s_dzb, kHid, xw(c, 1), kHid, c->s_dh, kHid, rows, kHid, kHid);
    k_back_silu<<<ew_blocks(rows * kHid), 256, 0, s>>>(c->s_dh, c->s_z1, rows * kHid, c->s_dzf, nullptr);
    k_grad_w1<kXOut><<<kHid * kIn, 256, 0, s>>>(c->x_P, c->s_dzf, c->s_x, rows, G);
    k_colred<float, float><<<kHid, 256, 0, s>>>(nullptr, 0, c->s_dzf, kHid, rows, 1, kHid, G + XLayout::B1);
    return cudaGetLastError();
}

// Network outputs [n][16] (normalised) of n raw input rows: the two persistent tcgen05
// kernels (the output layer's 16 sums reduced in two rounds of 8), or the fused mma.sync
// kernel (raptor_surrogate_kernel chooses for both networks).
cudaError_t x_eval_rows(raptor_ctx* c, const float* inputs, long long n, float* out, cudaStream_t s) {
    if (c->s_kernel == RAPTOR_MLP_MMA_SYNC) {
        const long long blocks = (n + kFRows - 1) / kFRows;
        k_mlp_fused<kXOut><<<(unsigned)blocks, 256, 0, s>>>(c->x_P, xw(c, 0), xw(c, 2), inputs, n, out);
        return cudaGetLastError();
    }
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    cudaError_t e = cudaSuccess;
    if ((size_t)tiles > c->x_h2tc_tiles) {
        e = cudaFree(c->x_h2tc);
        c->x_h2tc = nullptr;
        c->x_h2tc_tiles = 0;
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->x_h2tc, (size_t)tiles * kTcTileBytes);
        if (e != cudaSuccess) return e;
        c->x_h2tc_tiles = (size_t)tiles;
    }
    const unsigned grid = (unsigned)std::min<long long>(tiles, c->num_sms);
    k_mlp_tc12<kXOut><<<grid, kTcThreads, kTc12Smem, s>>>(c->x_P, xw(c, 4), inputs, n, c->x_h2tc, c->s_err);
    k_mlp_tc34<kXOut><<<grid, kTcThreads, tc34_smem<kXOut>(), s>>>(c->x_P, xw(c, 5), c->x_h2tc, n, out, c->s_err);
    return cudaGetLastError();
}

double sum_parts(raptor_ctx* c, int nb, cudaStream_t s, cudaError_t* e) {
    double parts[64];
    *e = cudaMemcpyAsync(parts, c->s_loss, nb * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (*e == cudaSuccess) *e = cudaStreamSynchronize(s);
    double L = 0.0;
    for (int q = 0; q < nb; ++q) L += parts[q];
    return L;
}

}  // namespace

namespace {

// The learned part of a thin-disk image (raptor_disk_render_learned): network inputs and
// fallback flags per pixel (k_surrogate_prepare, the critical curve of the camera's spin and
// inclination), the crossing network, the decoded hits of the pixels outside the fallback
// set, and the list of the others, which k_disk_fp64 then integrates (a.list).
raptor_status disk_learned_stage(raptor_ctx* ctx, const Params& p, DiskArgs& a, cudaStream_t s) {
    if (!ctx->x_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "the learned disk needs a trained crossing network");
    if (a.r_in < r_isco_prograde(ctx->cam.spin) * (1.0 - 1e-12))
        return fail(ctx, RAPTOR_EUNSUPPORTED, "the learned disk starts at or outside the ISCO (its ratios are trained there)");
    // the network maps its training range of spin and inclination to [-1, 1]; outside it
    // (beyond a small margin) its outputs are extrapolations
    const double na = (ctx->cam.spin - ctx->x_norm[4 + 2]) * ctx->x_norm[2];
    const double ni = (ctx->cam.incl_deg - ctx->x_norm[4 + 3]) * ctx->x_norm[3];
    if (!(std::fabs(na) <= 1.02) || !(std::fabs(ni) <= 1.02))
        return fail(ctx, RAPTOR_EUNSUPPORTED, "camera spin or inclination outside the crossing network's training range");
    const size_t n = (size_t)p.n_rays;
    if (ctx->s_ray_cap < n) {
        ctx->epoch += 1;
        cudaFree(ctx->s_in);
        cudaFree(ctx->s_fb);
        cudaFree(ctx->s_start);
        ctx->s_in = nullptr;
        ctx->s_fb = nullptr;
        ctx->s_start = nullptr;
        ctx->s_ray_cap = 0;
        RCK(cudaMalloc((void**)&ctx->s_in, n * kIn * sizeof(float)));
        RCK(cudaMalloc((void**)&ctx->s_fb, n));
        RCK(cudaMalloc((void**)&ctx->s_start, n * 8 * sizeof(float2)));
        ctx->s_ray_cap = n;
    }
    if (ctx->x_list_cap < n) {
        cudaFree(ctx->x_list);
        ctx->x_list = nullptr;
        ctx->x_list_cap = 0;
        RCK(cudaMalloc((void**)&ctx->x_list, n * sizeof(int)));
        ctx->x_list_cap = n;
    }
    if (!ctx->x_nlist) RCK(cudaMalloc((void**)&ctx->x_nlist, sizeof(unsigned int)));
    RCK(upload_curve(ctx, p, s));
    const float grow = (float)ctx->x_band + 1e-3f;
    const float4 box = make_float4(ctx->curve_box.x - grow, ctx->curve_box.y + grow, ctx->curve_box.z - grow,
                                   ctx->curve_box.w + grow);
    float* out = nullptr;
    RCK(cudaMallocAsync((void**)&out, n * kXOut * sizeof(float), s));
    cudaError_t e = cudaSuccess;
    {
        ProfScope ps(ctx, kProfSurrogate, s, 2);
        k_surrogate_prepare<<<ew_blocks((long long)n), 256, 0, s>>>(p, ctx->d_curve, ctx->n_curve, (float)ctx->x_band, box,
                                                                    ctx->s_in, ctx->s_fb, ctx->d_stats + kStatFallback);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            ProfScope pm(ctx, kProfSurrogateMlp, s, ctx->s_kernel == RAPTOR_MLP_MMA_SYNC ? 1 : 2);
            e = x_eval_rows(ctx, ctx->s_in, (long long)n, out, s);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->x_list, 0xFF, n * sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->x_nlist, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) {
            k_disk_learned<<<ew_blocks((long long)n), 256, 0, s>>>(p, a, ctx->x_P, out, ctx->s_fb, ctx->x_list, ctx->x_nlist,
                                                                   (float)ctx->x_zmargin, (float)ctx->x_lnr_margin);
            e = cudaGetLastError();
        }
    }
    const cudaError_t ef = cudaFreeAsync(out, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return fail(ctx, RAPTOR_ECUDA, cudaGetErrorString(e));
    a.list = ctx->x_list;
    return RAPTOR_OK;
}

}  // namespace

extern "C" {

int raptor_crossings_param_count(void) { return XLayout::SIZE; }

raptor_status raptor_crossings_generate(raptor_ctx* ctx, long long n, unsigned long long seed, double spin_min,
                                        double spin_max, double incl_min_deg, double incl_max_deg, float* inputs_dev,
                                        double* targets_dev, double* raw_dev, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (n < 1 || !inputs_dev || !targets_dev) return fail(ctx, RAPTOR_EINVAL, "need n >= 1 and output buffers");
    if (!(spin_min > -1.0 && spin_max >= spin_min && spin_max < 1.0)) return fail(ctx, RAPTOR_EINVAL, "spin range invalid");
    if (!(incl_min_deg > 0.0 && incl_max_deg >= incl_min_deg && incl_max_deg < 90.0))
        return fail(ctx, RAPTOR_EINVAL, "inclination range invalid (0 < i < 90 deg: the camera above the plane)");
    SurrogateRange R{ctx->cam.alpha_min, ctx->cam.alpha_max, ctx->cam.beta_min, ctx->cam.beta_max, spin_min, spin_max,
                     incl_min_deg, incl_max_deg, ctx->cam.r_cam, ctx->cam.eps};
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    {
        ProfScope ps(ctx, kProfTrain, s);
        k_crossing_data<<<ctx->num_sms * 8, 128, 0, s>>>(R, ctx->cam.r_stop_factor, ctx->cam.r_escape, ctx->cam.max_steps,
                                                          seed, n, inputs_dev, targets_dev, raw_dev);
    }
    RCK(cudaGetLastError());
    return RAPTOR_OK;
}

raptor_status raptor_crossings_init(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                    unsigned long long seed, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!targets_dev || n < 2) return fail(ctx, RAPTOR_EINVAL, "need targets and n >= 2");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(x_alloc(ctx));
    const long long m = std::min<long long>(n, 65536);
    std::vector<double> y((size_t)m * kXOut);
    RCK(cudaMemcpyAsync(y.data(), targets_dev, y.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    std::vector<float> P(XLayout::SIZE, 0.f);
    uint64_t st = seed ^ 0xC505ull;
    auto uni = [&](double lim) { return (float)(lim * (2.0 * ((splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0)); };
    for (int i = 0; i < kHid * kIn; ++i) P[XLayout::W1 + i] = uni(std::sqrt(6.0 / kIn));
    for (int i = 0; i < kHid * kHid; ++i) P[XLayout::W2 + i] = uni(std::sqrt(6.0 / kHid));
    for (int i = 0; i < kHid * kHid; ++i) P[XLayout::W3 + i] = uni(std::sqrt(6.0 / kHid));
    for (int i = 0; i < kXOut * kHid; ++i) P[XLayout::W4 + i] = uni(std::sqrt(3.0 / kHid));
    const double ha = 0.5 * (ctx->cam.alpha_max - ctx->cam.alpha_min), hb = 0.5 * (ctx->cam.beta_max - ctx->cam.beta_min);
    float scale[4] = {(float)(1.0 / ha), (float)(1.0 / hb), 2.0f, 1.0f / 40.0f};
    float shift[4] = {(float)(0.5 * (ctx->cam.alpha_max + ctx->cam.alpha_min)),
                      (float)(0.5 * (ctx->cam.beta_max + ctx->cam.beta_min)), 0.5f, 45.0f};
    if (inputs_dev) {
        // spin and inclination mapped to [-1, 1] over the range of all n given inputs
        unsigned* mm = nullptr;
        RCK(cudaMallocAsync((void**)&mm, 4 * sizeof(unsigned), s));
        const unsigned init[4] = {0xFFFFFFFFu, 0u, 0xFFFFFFFFu, 0u};
        cudaError_t e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            k_input_range<<<ew_blocks(n), 256, 0, s>>>(inputs_dev, n, mm);
            e = cudaGetLastError();
        }
        unsigned h[4] = {0u, 0u, 0u, 0u};
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        const cudaError_t ef = cudaFreeAsync(mm, s);
        if (e == cudaSuccess) e = ef;
        if (e != cudaSuccess) return fail(ctx, RAPTOR_ECUDA, cudaGetErrorString(e));
        for (int c = 2; c < 4; ++c) {
            const float lo = ordered_to_float(h[2 * (c - 2)]), hi = ordered_to_float(h[2 * (c - 2) + 1]);
            if (!std::isfinite(lo) || !std::isfinite(hi)) return fail(ctx, RAPTOR_EINVAL, "non-finite spin or inclination input");
            shift[c] = 0.5f * (lo + hi);
            scale[c] = hi > lo ? 2.0f / (hi - lo) : 1.0f;
        }
    }
    for (int c = 0; c < 4; ++c) {
        P[XLayout::NORM + c] = scale[c];
        P[XLayout::NORM + 4 + c] = shift[c];
        ctx->x_norm[c] = scale[c];
        ctx->x_norm[4 + c] = shift[c];
    }
    // output normalisation over the targets present (presence logits: none)
    for (int q = 0; q < kXOut; ++q) {
        double mu = 0.0, var = 0.0;
        long long cnt = 0;
        if (q % 4 != 0) {
            for (long long i = 0; i < m; ++i) {
                const double v = y[i * kXOut + q];
                if (std::isnan(v)) continue;
                mu += v;
                cnt += 1;
            }
            mu = cnt ? mu / cnt : 0.0;
            for (long long i = 0; i < m; ++i) {
                const double v = y[i * kXOut + q];
                if (!std::isnan(v)) var += (v - mu) * (v - mu);
            }
            var = cnt > 1 ? var / (cnt - 1) : 1.0;
        } else {
            var = 1.0;
        }
        P[XLayout::MU + q] = (float)mu;
        P[XLayout::SD + q] = (float)std::max(std::sqrt(var), 1e-6);
    }
    RCK(cudaMemcpyAsync(ctx->x_P, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RCK(cudaMemsetAsync(ctx->x_m1, 0, XLayout::SIZE * sizeof(float), s));
    RCK(cudaMemsetAsync(ctx->x_m2, 0, XLayout::SIZE * sizeof(float), s));
    RCK(x_refresh(ctx, s));
    RCK(cudaStreamSynchronize(s));
    ctx->x_step = 0;
    ctx->x_ready = true;
    return RAPTOR_OK;
}

raptor_status raptor_crossings_train(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                     int steps, double lr, double lr_final, unsigned long long seed, double* loss_host,
                                     void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->x_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "crossing network not initialised");
    if (!inputs_dev || !targets_dev || n < 1 || steps < 1 || !(lr > 0.0) || !(lr_final > 0.0))
        return fail(ctx, RAPTOR_EINVAL, "invalid training arguments");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(x_alloc(ctx));
    const float b1 = 0.9f, b2 = 0.999f;
    ProfScope ps(ctx, kProfTrain, s);
    for (int it = 0; it < steps; ++it) {
        k_gather_batch<kXOut><<<ew_blocks(kSurRows), 256, 0, s>>>(inputs_dev, targets_dev, n, kSurRows, seed,
                                                                  (long long)ctx->x_step, ctx->s_x, ctx->x_y);
        RCK(x_forward(ctx, kSurRows, s));
        int nb = 0;
        RCK(x_backward(ctx, kSurRows, &nb, s));
        ctx->x_step += 1;
        const double frac = steps > 1 ? (double)it / (steps - 1) : 1.0;
        const double lr_it = lr_final + 0.5 * (lr - lr_final) * (1.0 + std::cos(kPi * frac));
        const double t = (double)ctx->x_step;
        const float lr_t = (float)(lr_it * std::sqrt(1.0 - std::pow(b2, t)) / (1.0 - std::pow(b1, t)));
        k_adam<<<ew_blocks(XLayout::NORM), 256, 0, s>>>(ctx->x_P, ctx->x_G, ctx->x_m1, ctx->x_m2, XLayout::NORM, lr_t, b1, b2,
                                                       1e-8f);
        RCK(x_refresh(ctx, s));
        if (loss_host) {
            cudaError_t e = cudaSuccess;
            const double L = sum_parts(ctx, nb, s, &e);
            RCK(e);
            loss_host[it] = L / (double)(kSurRows * kXOut);
        }
    }
    return RAPTOR_OK;
}

raptor_status raptor_crossings_grad(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                    float* grad_host, double* loss_host, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->x_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "crossing network not initialised");
    if (!inputs_dev || !targets_dev || n < 1 || n > kSurRows || n % kGBM != 0)
        return fail(ctx, RAPTOR_EINVAL, "n must be a multiple of 128 and at most 4096");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    RCK(cudaMemcpyAsync(ctx->s_x, inputs_dev, n * kIn * sizeof(float), cudaMemcpyDeviceToDevice, s));
    RCK(cudaMemcpyAsync(ctx->x_y, targets_dev, n * kXOut * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RCK(x_forward(ctx, n, s));
    int nb = 0;
    RCK(x_backward(ctx, n, &nb, s));
    if (grad_host) RCK(cudaMemcpyAsync(grad_host, ctx->x_G, XLayout::NORM * sizeof(float), cudaMemcpyDeviceToHost, s));
    cudaError_t e = cudaSuccess;
    const double L = sum_parts(ctx, nb, s, &e);
    RCK(e);
    if (loss_host) *loss_host = L / (double)(n * kXOut);
    return RAPTOR_OK;
}

raptor_status raptor_crossings_eval(raptor_ctx* ctx, const float* inputs_dev, long long n, double* pred_dev, void* stream) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->x_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "crossing network not initialised");
    if (!inputs_dev || !pred_dev || n < 1) return fail(ctx, RAPTOR_EINVAL, "invalid arguments");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    float* out = nullptr;
    RCK(cudaMallocAsync((void**)&out, n * kXOut * sizeof(float), s));
    cudaError_t e = x_eval_rows(ctx, inputs_dev, n, out, s);
    if (e == cudaSuccess) {
        k_crossings_decode<<<ew_blocks(n), 256, 0, s>>>(ctx->x_P, inputs_dev, out, n, (float)ctx->cam.r_cam, pred_dev);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(out, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return fail(ctx, RAPTOR_ECUDA, cudaGetErrorString(e));
    return RAPTOR_OK;
}

raptor_status raptor_crossings_config(raptor_ctx* ctx, double fallback_band, int fallback_df64) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!(fallback_band >= 0.0) || !std::isfinite(fallback_band))
        return fail(ctx, RAPTOR_EINVAL, "fallback_band must be finite and >= 0");
    if (fallback_df64 != 0 && fallback_df64 != 1) return fail(ctx, RAPTOR_EINVAL, "fallback_df64 must be 0 or 1");
    ctx->x_band = fallback_band;
    ctx->x_df = fallback_df64 != 0;
    return RAPTOR_OK;
}

raptor_status raptor_crossings_confidence(raptor_ctx* ctx, double presence_margin, double radius_margin) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!(presence_margin >= 0.0) || !std::isfinite(presence_margin) || !(radius_margin >= 0.0) ||
        !std::isfinite(radius_margin))
        return fail(ctx, RAPTOR_EINVAL, "presence_margin and radius_margin must be finite and >= 0");
    ctx->x_zmargin = presence_margin;
    ctx->x_lnr_margin = radius_margin;
    return RAPTOR_OK;
}

raptor_status raptor_crossings_get(raptor_ctx* ctx, float* params_host, int n) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!ctx->x_ready) return fail(ctx, RAPTOR_EUNSUPPORTED, "crossing network not initialised");
    if (!params_host || n != XLayout::SIZE) return fail(ctx, RAPTOR_EINVAL, "n must equal raptor_crossings_param_count()");
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(params_host, ctx->x_P, n * sizeof(float), cudaMemcpyDeviceToHost));
    return RAPTOR_OK;
}

raptor_status raptor_crossings_set(raptor_ctx* ctx, const float* params_host, int n) {
    if (!ctx) return RAPTOR_EINVAL;
    ctx->err.clear();
    if (!params_host || n != XLayout::SIZE) return fail(ctx, RAPTOR_EINVAL, "n must equal raptor_crossings_param_count()");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(params_host[i])) return fail(ctx, RAPTOR_EINVAL, "parameters must be finite");
    for (int q = 0; q < kXOut; ++q)
        if (!(params_host[XLayout::SD + q] > 0.f)) return fail(ctx, RAPTOR_EINVAL, "output scales must be positive");
    RCK(x_alloc(ctx));
    RCK(cudaStreamSynchronize(ctx->last_stream));
    RCK(cudaMemcpy(ctx->x_P, params_host, n * sizeof(float), cudaMemcpyHostToDevice));
    for (int c = 0; c < 8; ++c) ctx->x_norm[c] = params_host[XLayout::NORM + c];
    RCK(cudaMemset(ctx->x_m1, 0, n * sizeof(float)));
    RCK(cudaMemset(ctx->x_m2, 0, n * sizeof(float)));
    RCK(x_refresh(ctx, nullptr));
    RCK(cudaDeviceSynchronize());
    ctx->x_step = 0;
    ctx->x_ready = true;
    return RAPTOR_OK;
}

}  // extern "C"
