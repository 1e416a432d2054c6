// raptor_surrogate.cuh -- learned far-field surrogate: training data from the integrator,
// a 4-layer MLP trained and evaluated with hand-written kernels, and the reconstruction of
// an integrator state from its prediction.
//
// What is learned: the FP64 integrator's state after exactly n_steps adaptive RK4 steps from
// the camera (the hand-off step count, raptor_surrogate_handoff; stored with the network's
// parameters), as a function of (alpha, beta, a, i).  For a fixed step count the state is a
// smooth function of the inputs (no quantisation of the step sequence), and the rays of a
// +-20 M camera are still far outside the emitting region there (r >~ 40 M after 60 steps).
// The network's angular error at the hand-off carries over to the path inside the emitting
// region, and the residual it learns (the deflection accumulated since the camera) falls
// like r^-2 with the hand-off radius: an earlier hand-off gives a more accurate path.  The exact integrator continues from the predicted state, so the transfer is
// sampled on the same step sequence as the full integration.  E, L and Q follow exactly from
// the inputs; the network predicts the position (t - t_cam, ln r, theta, phi) and the signs
// of k^theta and k^r, and the wave vector is rebuilt from the constants of motion.
//
// Network: in(4, FP32) -> 256 -> 256 -> 256 -> out(8), SiLU activations.  The two
// 256 x 256 layers run on tensor cores (BF16 operands, FP32 accumulation, mma.sync
// m16n8k16); the thin input and output layers run in FP32 so that alpha and beta are not
// rounded to BF16's 8-bit mantissa.  FP32 master weights, Adam.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "raptor_physics.cuh"

namespace raptor {

constexpr int kSurrogateSteps = 60;   // default hand-off step count (raptor_surrogate_handoff)
constexpr int kMaxHandoffSteps = 1000;
constexpr int kHid = 256;
constexpr int kIn = 4;
constexpr int kOut = 8;      // 6 used: dt, ln r, theta, phi, k^theta, k^r
constexpr int kOutUsed = 6;

// ---------------------------------------------------------------------------------------
// Training data: counter-based samples (SplitMix64 of seed and index) -> inputs
// (alpha, beta, a, i in degrees) and the integrator's state after kSurrogateSteps steps.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double u01(uint64_t seed, uint64_t idx, int stream) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (idx * 4 + (uint64_t)stream + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

struct SurrogateRange {
    double amin, amax, bmin, bmax;   // image plane
    double smin, smax;               // spin
    double imin, imax;               // inclination, degrees
    double r_cam, eps;
    int n_steps = kSurrogateSteps;   // state after this many steps (the hand-off)
};

// Flat-space baseline: the camera ray's initial state (KS at r_cam) continued as a straight
// line (r, theta, phi read as spherical coordinates, M -> 0), advanced by the same step rule
// for n_steps steps (the hand-off step count), all in FP32.  It is a fixed, smooth function of the inputs; the
// network learns only the difference between the integrator and this baseline (the
// gravitational deflection and delay, a few per cent), which BF16 layers resolve far better
// than the state itself.  Output as the targets: dt, ln r, theta, phi, k^theta, k^r.
RAPTOR_HD void surrogate_baseline(const float x0[4], const float k0[4], float eps, int n_steps, float out[kOutUsed]) {
    const float r = x0[1], th = x0[2], ph = x0[3];
    const float st = sinf(th), ct = cosf(th), sp = sinf(ph), cp = cosf(ph);
    // position and velocity in Cartesian components
    float px = r * st * cp, py = r * st * sp, pz = r * ct;
    const float kr = k0[1], kh = k0[2], kp = k0[3];
    const float vx = kr * st * cp + r * kh * ct * cp - r * st * kp * sp;
    const float vy = kr * st * sp + r * kh * ct * sp + r * st * kp * cp;
    const float vz = kr * ct - r * kh * st;
    const float kt = k0[0];
    float lam = 0.f, rr = r, thn = th, vr = kr, vth = kh;
    for (int n = 0; n <= n_steps; ++n) {
        // spherical components: r, theta and the rates dr, dtheta, dphi per unit lambda
        const float rho2 = px * px + py * py;
        rr = sqrtf(rho2 + pz * pz);
        const float rho = sqrtf(rho2), irr = 1.f / rr;
        thn = atan2f(rho, pz);
        const float vp = vx * px + vy * py;
        vr = (vp + vz * pz) * irr;
        vth = (pz * vp / fmaxf(rho, 1e-30f) - vz * rho) * irr * irr;
        if (n == n_steps) break;
        const float vph = (vy * px - vx * py) / fmaxf(rho2, 1e-30f);
        const float xs[4] = {0.f, rr, thn, 0.f}, ks[4] = {kt, vr, vth, vph};
        const float dl = step_size<float>(eps, false, xs, ks);
        px += vx * dl;
        py += vy * dl;
        pz += vz * dl;
        lam += dl;
    }
    out[0] = kt * lam;
    out[1] = logf(rr);
    out[2] = thn;
    out[3] = atan2f(py, px);
    out[4] = vth;
    out[5] = vr;
}

// The baseline of the ray through (alpha, beta) from the camera parameters: the camera wave
// vector in FP32 (phi0: the camera's KS azimuth).  Training and rendering both use this.
RAPTOR_HD void surrogate_base(float a, float sn_i, float cs_i, float incl, float r_cam, float phi0, float alpha, float beta,
                              float eps, int n_steps, float out[kOutUsed]) {
    float k0[4];
    camera_k_t<float>(a, sn_i, cs_i, r_cam, alpha, beta, k0);
    const float x0[4] = {0.f, r_cam, incl, phi0};
    surrogate_baseline(x0, k0, eps, n_steps, out);
}

// Integrator state after n_steps steps (FP64) minus the baseline: the targets (raw,
// optional: the state itself in the same six components).
RAPTOR_HD void surrogate_targets(double a, double incl_deg, double r_cam, double eps, double alpha, double beta,
                                 int n_steps, double out[kOutUsed], double* raw = nullptr) {
    const double inc = incl_deg * (kPi / 180.0);
    const double sn = sin(inc), cs = cos(inc);
    double x[4], k[4];
    camera_ray_ai(a, sn, cs, inc, r_cam, alpha, beta, 0.0, x, k);
    float base[kOutUsed];
    surrogate_base((float)a, (float)sn, (float)cs, (float)inc, (float)r_cam, (float)x[3], (float)alpha, (float)beta,
                   (float)eps, n_steps, base);
    const double t0 = x[0];
    for (int n = 0; n < n_steps; ++n) rk4_step<double>(a, x, k, step_size<double>(eps, false, x, k));
    out[0] = x[0] - t0 - base[0];
    out[1] = log(x[1]) - base[1];
    out[2] = x[2] - base[2];
    out[3] = x[3] - base[3];
    out[4] = k[2] - base[4];
    out[5] = k[1] - base[5];
    if (raw) {
        raw[0] = x[0] - t0;
        raw[1] = log(x[1]);
        raw[2] = x[2];
        raw[3] = x[3];
        raw[4] = k[2];
        raw[5] = k[1];
    }
}

__global__ void k_surrogate_data(SurrogateRange R, uint64_t seed, long long n, float* __restrict__ inputs,
                                 double* __restrict__ targets, double* __restrict__ raw) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        // inputs are stored (and later evaluated) in FP32: the targets use the same values
        const double al = (double)(float)(R.amin + (R.amax - R.amin) * u01(seed, i, 0));
        const double be = (double)(float)(R.bmin + (R.bmax - R.bmin) * u01(seed, i, 1));
        const double a = (double)(float)(R.smin + (R.smax - R.smin) * u01(seed, i, 2));
        const double inc = (double)(float)(R.imin + (R.imax - R.imin) * u01(seed, i, 3));
        inputs[i * kIn + 0] = (float)al;
        inputs[i * kIn + 1] = (float)be;
        inputs[i * kIn + 2] = (float)a;
        inputs[i * kIn + 3] = (float)inc;
        double t[kOutUsed], rw[kOutUsed];
        surrogate_targets(a, inc, R.r_cam, R.eps, al, be, R.n_steps, t, rw);
        for (int q = 0; q < kOutUsed; ++q) targets[i * kOutUsed + q] = t[q];
        if (raw)
            for (int q = 0; q < kOutUsed; ++q) raw[i * kOutUsed + q] = rw[q];
    }
}

// ---------------------------------------------------------------------------------------
// Parameters: one FP32 buffer holding every tensor, plus BF16 copies of the two hidden
// weight matrices ([out][in] and transposed [in][out]) for the tensor-core GEMMs.
// ---------------------------------------------------------------------------------------
template <int NOUT>
struct MlpLayoutT {
    static constexpr int W1 = 0;                         // [256][4]
    static constexpr int B1 = W1 + kHid * kIn;           // [256]
    static constexpr int W2 = B1 + kHid;                 // [256][256]
    static constexpr int B2 = W2 + kHid * kHid;
    static constexpr int W3 = B2 + kHid;
    static constexpr int B3 = W3 + kHid * kHid;
    static constexpr int W4 = B3 + kHid;                 // [NOUT][256]
    static constexpr int B4 = W4 + NOUT * kHid;          // [NOUT]
    static constexpr int NORM = B4 + NOUT;               // input scale[4], shift[4], output mean[NOUT], std[NOUT]
    static constexpr int MU = NORM + 8;
    static constexpr int SD = MU + NOUT;
    static constexpr int HANDOFF = MU + NOUT - 1;        // unused output's mean slot: the hand-off step count
    static constexpr int SIZE = SD + NOUT;
};
using MlpLayout = MlpLayoutT<kOut>;

// SiLU with the hardware exponential and reciprocal (the argument of exp is capped at 80 so
// that 1 + e^-z stays inside the approximate division's range; below z = -80, silu is ~0).
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(fminf(-z, 80.f))); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Layer 1 (FP32): z1 = W1 x_n + b1, h1 = silu(z1) (BF16), x_n = (x - shift) * scale.
template <int NOUT = kOut>
__global__ void k_mlp_layer1(const float* __restrict__ P, const float* __restrict__ x, long long rows, long long rows_valid,
                             float* __restrict__ z1, __nv_bfloat16* __restrict__ h1) {
    const long long total = rows * kHid;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / kHid;
        const int j = (int)(e - m * kHid);
        float acc = P[MlpLayoutT<NOUT>::B1 + j];
        if (m < rows_valid) {
#pragma unroll
            for (int c = 0; c < kIn; ++c) {
                const float xn = (x[m * kIn + c] - P[MlpLayoutT<NOUT>::NORM + 4 + c]) * P[MlpLayoutT<NOUT>::NORM + c];
                acc += P[MlpLayoutT<NOUT>::W1 + j * kIn + c] * xn;
            }
        }
        if (z1) z1[e] = acc;
        h1[e] = __float2bfloat16(silu(acc));
    }
}

// z += bias (optional); h = silu(z) in BF16.
__global__ void k_bias_silu(float* __restrict__ z, const float* __restrict__ bias, long long rows, __nv_bfloat16* __restrict__ h) {
    const long long total = rows * kHid;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const float v = z[e] + bias[e % kHid];
        z[e] = v;
        h[e] = __float2bfloat16(silu(v));
    }
}

// Output layer (FP32 weights, BF16 activations): out[m][o] = W4[o] . h3[m] + b4[o].
// One warp per row.
template <int NOUT = kOut>
__global__ void k_mlp_layer4(const float* __restrict__ P, const __nv_bfloat16* __restrict__ h3, long long rows,
                             float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long m = warp; m < rows; m += nw) {
        float acc[NOUT];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) acc[o] = 0.f;
        for (int j = lane; j < kHid; j += 32) {
            const float h = __bfloat162float(h3[m * kHid + j]);
#pragma unroll
            for (int o = 0; o < NOUT; ++o) acc[o] += P[MlpLayoutT<NOUT>::W4 + o * kHid + j] * h;
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            float v = acc[o];
            for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
            if (lane == 0) out[m * NOUT + o] = v + P[MlpLayoutT<NOUT>::B4 + o];
        }
    }
}

// ---------------------------------------------------------------------------------------
// BF16 tensor-core GEMM: C[M][N] (FP32) = sum_k A(m, k) B(n, k), with
//   A(m, k) = A[m * lda + k] (A_KMAJ) or A[k * lda + m];  B(n, k) likewise.
// Tiles 128 x 128 x 32, 256 threads (8 warps as 2 x 4, each 64 x 32), mma.sync m16n8k16
// BF16 -> FP32.  M, N multiples of 128 and K a multiple of 32 (the host pads).
// ---------------------------------------------------------------------------------------
constexpr int kGBM = 128, kGBN = 128, kGBK = 32, kGPad = 8;

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Load a 128 x 32 tile (rows r0.., k0..) of op(X) into smem S[128][32 + pad] ([row][k]).
template <bool KMAJ>
__device__ __forceinline__ void gemm_load_tile(const __nv_bfloat16* __restrict__ X, long long ld, long long r0, long long k0,
                                               __nv_bfloat16 (*S)[kGBK + kGPad]) {
    const int t = threadIdx.x;
    if (KMAJ) {
        // 128 rows x 32 k = 128 x 4 uint4; each thread loads 2
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = t + q * 256;
            const int row = idx >> 2, c = (idx & 3) * 8;
            const uint4 v = *reinterpret_cast<const uint4*>(X + (r0 + row) * ld + k0 + c);
            *reinterpret_cast<uint4*>(&S[row][c]) = v;
        }
    } else {
        // 32 k-rows x 128 (contiguous) = 32 x 16 uint4; each thread loads 2, stores transposed
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = t + q * 256;
            const int kk = idx >> 4, c = (idx & 15) * 8;
            const uint4 v = *reinterpret_cast<const uint4*>(X + (k0 + kk) * ld + r0 + c);
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int u = 0; u < 8; ++u) S[c + u][kk] = e[u];
        }
    }
}

template <bool A_KMAJ, bool B_KMAJ>
__global__ void __launch_bounds__(256) k_gemm_bf16(const __nv_bfloat16* __restrict__ A, long long lda,
                                                   const __nv_bfloat16* __restrict__ B, long long ldb, float* __restrict__ C,
                                                   long long ldc, long long M, long long N, long long K) {
    __shared__ __align__(16) __nv_bfloat16 As[kGBM][kGBK + kGPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[kGBN][kGBK + kGPad];
    const long long m0 = (long long)blockIdx.y * kGBM, n0 = (long long)blockIdx.x * kGBN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const int gr = lane >> 2, gc = (lane & 3) * 2;
    for (long long k0 = 0; k0 < K; k0 += kGBK) {
        gemm_load_tile<A_KMAJ>(A, lda, m0, k0, As);
        gemm_load_tile<B_KMAJ>(B, ldb, n0, k0, Bs);
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kGBK; ks += 16) {
            uint32_t af[4][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = wm + i * 16 + gr;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + gc]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + gc]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + gc + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + gc + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + gr;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + gc]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + gc + 8]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long r = m0 + wm + i * 16 + gr, c = n0 + wn + j * 8 + gc;
            C[r * ldc + c] = acc[i][j][0];
            C[r * ldc + c + 1] = acc[i][j][1];
            C[(r + 8) * ldc + c] = acc[i][j][2];
            C[(r + 8) * ldc + c + 1] = acc[i][j][3];
        }
}

// ---------------------------------------------------------------------------------------
// Fused inference: one CTA runs 64 rows through all four layers.  Activations stay in
// shared memory (BF16, 64 x 256); the hidden weights stream through shared memory in
// 256 x 32 K-chunks (they are shared by every CTA and stay in L2); the 8 warps (2 x 4) each
// own a 32 x 64 block of a layer's output, computed with mma.sync m16n8k16 BF16 -> FP32.
// ---------------------------------------------------------------------------------------
constexpr int kFRows = 64, kFPadH = 8, kFChunk = 32, kFPadW = 8;

__device__ __forceinline__ void fused_hidden_layer(const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                                                   __nv_bfloat16 (*H)[kHid + kFPadH],
                                                   __nv_bfloat16 (*Wc)[kFChunk + kFPadW]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 2) * 32, wn = (warp & 3) * 64;
    const int gr = lane >> 2, gc = (lane & 3) * 2;
    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = 0; k0 < kHid; k0 += kFChunk) {
        // W[:, k0:k0+32] -> Wc ([out][k])
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = threadIdx.x + q * 256;
            const int row = idx >> 2, c = (idx & 3) * 8;
            *reinterpret_cast<uint4*>(&Wc[row][c]) = *reinterpret_cast<const uint4*>(W + (long long)row * kHid + k0 + c);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kFChunk; ks += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gr;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&H[r][k0 + ks + gc]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&H[r + 8][k0 + ks + gc]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&H[r][k0 + ks + gc + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&H[r + 8][k0 + ks + gc + 8]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = wn + j * 8 + gr;
                uint32_t bfr[2];
                bfr[0] = *reinterpret_cast<const uint32_t*>(&Wc[c][ks + gc]);
                bfr[1] = *reinterpret_cast<const uint32_t*>(&Wc[c][ks + gc + 8]);
#pragma unroll
                for (int i = 0; i < 2; ++i) mma_bf16_16816(acc[i][j], af[i], bfr);
            }
        }
        __syncthreads();
    }
    // epilogue: bias + SiLU -> BF16, written over the input activations (all reads are done)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = wm + i * 16 + gr, c = wn + j * 8 + gc;
            const float b0 = bias[c], b1 = bias[c + 1];
            H[r][c] = __float2bfloat16(silu(acc[i][j][0] + b0));
            H[r][c + 1] = __float2bfloat16(silu(acc[i][j][1] + b1));
            H[r + 8][c] = __float2bfloat16(silu(acc[i][j][2] + b0));
            H[r + 8][c + 1] = __float2bfloat16(silu(acc[i][j][3] + b1));
        }
    __syncthreads();
}

template <int NOUT = kOut>
__global__ void __launch_bounds__(256) k_mlp_fused(const float* __restrict__ P, const __nv_bfloat16* __restrict__ w2,
                                                   const __nv_bfloat16* __restrict__ w3, const float* __restrict__ x,
                                                   long long n, float* __restrict__ out) {
    __shared__ __align__(16) __nv_bfloat16 H[kFRows][kHid + kFPadH];
    __shared__ __align__(16) __nv_bfloat16 Wc[kHid][kFChunk + kFPadW];
    const long long m0 = (long long)blockIdx.x * kFRows;
    // layer 1 (FP32): 64 x 256 outputs, 64 per thread
    for (int e = threadIdx.x; e < kFRows * kHid; e += 256) {
        const int m = e / kHid, j = e - m * kHid;
        float acc = P[MlpLayoutT<NOUT>::B1 + j];
        if (m0 + m < n) {
#pragma unroll
            for (int c = 0; c < kIn; ++c) {
                const float xn = (x[(m0 + m) * kIn + c] - P[MlpLayoutT<NOUT>::NORM + 4 + c]) * P[MlpLayoutT<NOUT>::NORM + c];
                acc += P[MlpLayoutT<NOUT>::W1 + j * kIn + c] * xn;
            }
        }
        H[m][j] = __float2bfloat16(silu(acc));
    }
    __syncthreads();
    fused_hidden_layer(w2, P + MlpLayoutT<NOUT>::B2, H, Wc);
    fused_hidden_layer(w3, P + MlpLayoutT<NOUT>::B3, H, Wc);
    // layer 4 (FP32 weights): thread -> (row, NOUT / 4 consecutive outputs)
    constexpr int PER = NOUT / 4;
    static_assert(NOUT % 4 == 0, "four threads per row");
    const int m = threadIdx.x >> 2, o = (threadIdx.x & 3) * PER;
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = P[MlpLayoutT<NOUT>::B4 + o + q];
    for (int j = 0; j < kHid; ++j) {
        const float h = __bfloat162float(H[m][j]);
#pragma unroll
        for (int q = 0; q < PER; ++q) acc[q] += P[MlpLayoutT<NOUT>::W4 + (o + q) * kHid + j] * h;
    }
    if (m0 + m < n) {
#pragma unroll
        for (int q = 0; q < PER; ++q) out[(m0 + m) * NOUT + o + q] = acc[q];
    }
}

// ---------------------------------------------------------------------------------------
// Backward pieces.
// ---------------------------------------------------------------------------------------
// Loss: mean over rows and the kOutUsed outputs of (out - y)^2 (y normalised on the fly);
// dout = d loss / d out.  loss_acc gets the per-block partial sums (deterministic order).
__global__ void k_mse_grad(const float* __restrict__ P, const float* __restrict__ out, const double* __restrict__ y,
                           long long rows, float* __restrict__ dout, double* __restrict__ loss_acc) {
    __shared__ double sh[256];
    double part = 0.0;
    const float inv = 1.f / (float)(rows * kOutUsed);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * kOut; e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / kOut;
        const int o = (int)(e - m * kOut);
        float g = 0.f;
        if (o < kOutUsed) {
            const float yn = (float)((y[m * kOutUsed + o] - P[MlpLayout::NORM + 8 + o]) / P[MlpLayout::NORM + 16 + o]);
            const float d = out[e] - yn;
            part += (double)d * d;
            g = 2.f * d * inv;
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

// dh3 = dout W4 (FP32), then dz3 = dh3 * silu'(z3) stored BF16 (the operand of the next GEMMs)
// and FP32 for the bias gradient.
template <int NOUT = kOut>
__global__ void k_back_layer4(const float* __restrict__ P, const float* __restrict__ dout, const float* __restrict__ z3,
                              long long rows, float* __restrict__ dz3f, __nv_bfloat16* __restrict__ dz3) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * kHid; e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / kHid;
        const int j = (int)(e - m * kHid);
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < NOUT; ++o) acc += dout[m * NOUT + o] * P[MlpLayoutT<NOUT>::W4 + o * kHid + j];
        const float g = acc * dsilu(z3[e]);
        dz3f[e] = g;
        dz3[e] = __float2bfloat16(g);
    }
}

// dz = dh * silu'(z) (dh from a GEMM, FP32); BF16 and FP32 copies.
__global__ void k_back_silu(const float* __restrict__ dh, const float* __restrict__ z, long long n, float* __restrict__ dzf,
                            __nv_bfloat16* __restrict__ dz) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float g = dh[e] * dsilu(z[e]);
        dzf[e] = g;
        if (dz) dz[e] = __float2bfloat16(g);
    }
}

// Column reductions over the batch (fixed order, one block per output element):
//   G[p][q] = sum_m X[m][p] * Y[m][q]   (X: FP32 or 1 for bias), p < P, q < Q.
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) k_colred(const TX* __restrict__ X, int ldx, const TY* __restrict__ Y, int ldy,
                                                long long rows, int P, int Q, float* __restrict__ G) {
    __shared__ float sh[256];
    const int e = blockIdx.x;
    const int p = e / Q, q = e - p * Q;
    float acc = 0.f;
    for (long long m = threadIdx.x; m < rows; m += 256) {
        const float xv = X ? (float)X[m * ldx + p] : 1.f;
        acc += xv * (float)Y[m * ldy + q];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[e] = sh[0];
}

// Input-layer weight gradient: dW1[j][c] = sum_m dz1[m][j] * x_n[m][c].
template <int NOUT = kOut>
__global__ void __launch_bounds__(256) k_grad_w1(const float* __restrict__ P, const float* __restrict__ dz1,
                                                 const float* __restrict__ x, long long rows, float* __restrict__ G) {
    __shared__ float sh[256];
    const int e = blockIdx.x;  // j * 4 + c
    const int j = e / kIn, c = e - j * kIn;
    float acc = 0.f;
    for (long long m = threadIdx.x; m < rows; m += 256) {
        const float xn = (x[m * kIn + c] - P[MlpLayoutT<NOUT>::NORM + 4 + c]) * P[MlpLayoutT<NOUT>::NORM + c];
        acc += dz1[m * kHid + j] * xn;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[MlpLayoutT<NOUT>::W1 + e] = sh[0];
}

// Adam (decoupled bias correction folded into the step size) over the first n parameters.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1, float* __restrict__ m2,
                       int n, float lr_t, float b1, float b2, float eps) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float b = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = b;
        P[i] -= lr_t * a / (sqrtf(b) + eps);
    }
}

// BF16 copies of W2, W3: [out][in] and transposed [in][out].
__global__ void k_refresh_bf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ w2, __nv_bfloat16* __restrict__ w2t,
                               __nv_bfloat16* __restrict__ w3, __nv_bfloat16* __restrict__ w3t) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kHid * kHid; e += gridDim.x * blockDim.x) {
        const int o = e / kHid, i = e - o * kHid;
        const __nv_bfloat16 a = __float2bfloat16(P[MlpLayout::W2 + e]);
        const __nv_bfloat16 b = __float2bfloat16(P[MlpLayout::W3 + e]);
        w2[e] = a;
        w2t[i * kHid + o] = a;
        w3[e] = b;
        w3t[i * kHid + o] = b;
    }
}

// Gather a training batch: rows idx = hash(seed, step, r) mod n (NY targets per row).
template <int NY = kOutUsed>
__global__ void k_gather_batch(const float* __restrict__ x, const double* __restrict__ y, long long n, long long rows,
                               uint64_t seed, long long step, float* __restrict__ xb, double* __restrict__ yb) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
        const long long i = (long long)(u01(seed, (uint64_t)step * (uint64_t)rows + r, 7) * (double)n) % n;
        for (int c = 0; c < kIn; ++c) xb[r * kIn + c] = x[i * kIn + c];
        for (int q = 0; q < NY; ++q) yb[r * NY + q] = y[i * NY + q];
    }
}

// ---------------------------------------------------------------------------------------
// Reconstruction of the integrator state from a prediction (FP32: the prediction's own
// error, ~1e-5 of the state, is far above FP32 rounding): position from the network
// (x[0] the offset from the camera's KS time); k_t = 1 and k_phi = -L of the backward ray;
// |k_theta| from the Carter constant with the predicted sign of k^theta; k^r from the null
// condition with the predicted sign.
// ---------------------------------------------------------------------------------------
RAPTOR_HD void surrogate_state(float a, float sn_i, float cs_i, float alpha, float beta, const float pred[kOutUsed],
                               float x[4], float k[4]) {
    const float a2 = a * a;
    const float L = -alpha * sn_i;                              // physical photon, E = 1
    const float Q = beta * beta + cs_i * cs_i * (alpha * alpha - a2);
    const float r = expf(pred[1]), th = pred[2];
    x[0] = pred[0];
    x[1] = r;
    x[2] = th;
    x[3] = pred[3];
    float sn, cs;
    sc(th, &sn, &cs);
    const float s2 = sn * sn;
    const float Sig = r * r + a2 * cs * cs, iS = 1.f / Sig, z = 2.f * r * iS;
    const float Del = r * r - 2.f * r + a2;
    float Th = Q + a2 * cs * cs - L * L * cs * cs / s2;
    if (Th < 0.f) Th = 0.f;
    const float kct = 1.f, kcp = -L;                            // backward-ray covariant components
    const float kch = (pred[4] >= 0.f ? 1.f : -1.f) * sqrtf(Th);  // sign(k_theta) = sign(k^theta)
    // KS inverse metric
    const float gtt = -(1.f + z), gtr = z, grr = Del * iS, grp = a * iS, ghh = iS, gpp = iS / s2;
    const float Bq = gtr * kct + grp * kcp;
    const float Cq = gtt * kct * kct + ghh * kch * kch + gpp * kcp * kcp;
    float D = Bq * Bq - grr * Cq;
    if (D < 0.f) D = 0.f;
    const float kr_up = (pred[5] >= 0.f ? 1.f : -1.f) * sqrtf(D);  // k^r = Bq + grr k_r
    const float kcr = (kr_up - Bq) / grr;
    k[0] = gtt * kct + gtr * kcr;
    k[1] = kr_up;
    k[2] = ghh * kch;
    k[3] = grp * kcr + gpp * kcp;
}

// Squared distance from a pixel centre to the nearest vertex of the critical-curve polygon
// (sc[n], in order around the closed curve) and, with `want_inside`, the even-odd test for
// the centre lying inside it.  FP32 with every rounding explicit (no contraction), so that
// the kernels taking decisions on the same pixel (fallback flag, near-critical list) take
// them identically.
__device__ __forceinline__ void curve_relation(float alf, float bef, const float2* sc, int n, bool want_inside,
                                               float& d2, bool& inside) {
    d2 = 3.0e38f;
    inside = false;
    for (int c = 0; c < n; ++c) {
        const float2 v1 = sc[c];
        const float dx = __fsub_rn(alf, v1.x), dy = __fsub_rn(bef, v1.y);
        d2 = fminf(d2, __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
        if (want_inside) {
            const float2 v2 = sc[c + 1 < n ? c + 1 : 0];
            if ((v1.y > bef) != (v2.y > bef) &&
                alf < __fadd_rn(v1.x, __fdiv_rn(__fmul_rn(dy, __fsub_rn(v2.x, v1.x)), __fsub_rn(v2.y, v1.y))))
                inside = !inside;
        }
    }
}

// Per ray of a render: network inputs (alpha, beta, a, i in degrees) and the fallback flag:
// pixel centre within `band` M of the critical curve (n_curve <= kMaxCurve points in order
// around the closed curve, FP32) or inside it (captured rays, whose near-horizon emission is
// too sensitive to the hand-off state for the surrogate's accuracy), or within kAxisBand M
// of alpha = 0: rays of (nearly) zero angular momentum pass the polar axis, where the step
// rule's min(theta, pi - theta) factor makes the transfer's samples follow tiny changes of
// L, such as the network's error.  Pixels outside the curve's bounding box grown by the
// band (`box` = alpha_min, alpha_max, beta_min, beta_max) are not near the curve, and skip
// the polygon loop.
constexpr int kMaxCurve = 512;
constexpr float kAxisBand = 0.01f;
__global__ void __launch_bounds__(256) k_surrogate_prepare(const Params p, const float2* __restrict__ curve, int n_curve,
                                                           float band, float4 box, float* __restrict__ inputs,
                                                           unsigned char* __restrict__ fallback,
                                                           unsigned long long* __restrict__ n_fallback) {
    __shared__ float2 sc[kMaxCurve];
    __shared__ unsigned int block_fb;
    if (threadIdx.x == 0) block_fb = 0;
    for (int c = threadIdx.x; c < n_curve; c += blockDim.x) sc[c] = curve[c];
    __syncthreads();
    unsigned int my_fb = 0;
    const float a_f = p.f.a, inc_deg = (float)(p.incl * (180.0 / kPi));
    const float band2 = band * band;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < p.n_rays;
         id += (long long)gridDim.x * blockDim.x) {
        const int frame = (int)(id / p.n_pix);
        const int pix = (int)(id - (long long)frame * p.n_pix);
        const int row = p.row0 + pix / p.nx, col = pix % p.nx;
        const float alf = (float)(p.amin + (col + 0.5) * p.da), bef = (float)(p.bmin + (row + 0.5) * p.db);
        reinterpret_cast<float4*>(inputs)[id] = make_float4(alf, bef, a_f, inc_deg);
        unsigned char fb = fabsf(alf) < kAxisBand ? 1 : 0;
        if (!fb && alf >= box.x && alf <= box.y && bef >= box.z && bef <= box.w) {
            // FP32 suffices: the band edge needs no more precision
            float d2;
            bool inside;
            curve_relation(alf, bef, sc, n_curve, true, d2, inside);
            fb = (inside || d2 < band2) ? 1 : 0;
        }
        fallback[id] = fb;
        my_fb += fb;
    }
    // rays that start at the camera (counted in the context's statistics)
    if (my_fb) atomicAdd(&block_fb, my_fb);
    __syncthreads();
    if (threadIdx.x == 0 && block_fb && n_fallback) atomicAdd(n_fallback, (unsigned long long)block_fb);
}

// Denormalise the network outputs and rebuild the start states [8][n_rays] (FP32 except the
// camera time and the pixel centres).
__global__ void k_surrogate_states(const Params p, const float* __restrict__ P, const float* __restrict__ out,
                                   float2* __restrict__ start_xk) {
    // the camera's KS time at t_cam = 0 and azimuth, the same for every pixel: the render's
    // terms of camera_x_ai, computed once on the host (per thread they would cost two FP64
    // logarithms and square roots each)
    const double xc0 = p.cam_logdel + p.cam_tterm;
    const float af = p.f.a, sif = (float)p.sin_i, cif = (float)p.cos_i, incf = (float)p.incl, rcf = (float)p.r_cam;
    const float ph0 = (float)p.cam_phi;
    float mu[kOutUsed], sd[kOutUsed];
#pragma unroll
    for (int q = 0; q < kOutUsed; ++q) {
        mu[q] = P[MlpLayout::NORM + 8 + q];
        sd[q] = P[MlpLayout::NORM + 16 + q];
    }
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < p.n_rays;
         id += (long long)gridDim.x * blockDim.x) {
        const int frame = (int)(id / p.n_pix);
        const int pix = (int)(id - (long long)frame * p.n_pix);
        const int row = p.row0 + pix / p.nx, col = pix % p.nx;
        const float al = (float)(p.amin + (col + 0.5) * p.da), be = (float)(p.bmin + (row + 0.5) * p.db);
        float base[kOutUsed];
        surrogate_base(af, sif, cif, incf, rcf, ph0, al, be, p.f.eps, p.start_n, base);
        const float4 o0 = reinterpret_cast<const float4*>(out)[2 * id];
        const float4 o1 = reinterpret_cast<const float4*>(out)[2 * id + 1];
        const float o[kOutUsed] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y};
        float pred[kOutUsed];
#pragma unroll
        for (int q = 0; q < kOutUsed; ++q) pred[q] = base[q] + (o[q] * sd[q] + mu[q]);
        float x[4], k[4];
        surrogate_state(af, sif, cif, al, be, pred, x, k);
        const double tc = p.t_frames ? p.t_frames[frame] : p.t_cam;
        const double t = tc + xc0 + (double)x[0];
        const float th = (float)t;
        start_xk[id] = make_float2(th, (float)(t - (double)th));
#pragma unroll
        for (int i = 1; i < 4; ++i) start_xk[(long long)i * p.n_rays + id] = make_float2(x[i], 0.f);
#pragma unroll
        for (int i = 0; i < 4; ++i) start_xk[(long long)(4 + i) * p.n_rays + id] = make_float2(k[i], 0.f);
    }
}

}  // namespace raptor
