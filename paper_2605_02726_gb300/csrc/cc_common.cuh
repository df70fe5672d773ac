// Shared device-side definitions of the encoder-step kernels: geometry, parameter layout,
// counter noise, Laplace mass, block reductions.  Included by every .cu of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cc {

constexpr int kL = 7;        // latent grids (Sec. III-A1, Eq. 1; Table II 1/1..1/64)
constexpr int kNH = 3;       // hyperlatent grids when enabled (Sec. III-A3, Eq. 6; Table II 1/16..1/64)
constexpr int kHB = 4;       // the largest hyperlatent grid is 1/2^kHB of the image
constexpr int kG = kL + kNH; // grid slots: latent grids 0..6, then hyperlatent grids 7..9
constexpr int kNCtx = 16;    // spatial context values
constexpr int kF = 4;        // IFCE output width
constexpr int kNIfce = 3;    // grids 0..2 carry an IFCE (Table II)
constexpr int kAIn = kNCtx + kF;
constexpr int kAH = 16;      // ARM hidden width
constexpr int kC = 3;        // image channels
constexpr int kSH = 40;      // synthesis hidden width
constexpr float kLogbMin = -5.f, kLogbMax = 5.f;
constexpr float kPMin = 1.f / 65536.f;

// Flat parameter vector (row-major [out][in] matrices); the interface documented in coolchic.h.
namespace po {
constexpr int arm_w1 = 0, arm_b1 = 320, arm_w2 = 336, arm_b2 = 592, arm_w3 = 608, arm_b3 = 640,
              arm_ws = 642, arm_bs = 682;
constexpr int if_w0 = 684, if_b0 = 708, if_w1 = 712, if_b1 = 732, if_w2 = 736, if_b2 = 752;
constexpr int up = 756;
constexpr int syn_w1 = 780, syn_b1 = 1060, syn_w2 = 1100, syn_b2 = 1220, syn_ws = 1223, syn_bs = 1244;
constexpr int cv1_w = 1247, cv1_b = 1328, cv2_w = 1331, cv2_b = 1412;
constexpr int total = 1415;
constexpr int arm_block = up;                 // ARM + IFCE parameters: [0, 756)
constexpr int syn_block = cv1_w - syn_w1;     // 467
constexpr int conv_block = total - cv1_w;     // 168
// with hyperlatents: the IFCE weights of the hyperlatent inputs [grid k][output o][grid q] follow
constexpr int ifce_h = total, ifce_h_n = kNIfce * kF * kNH, total_h = total + ifce_h_n;  // 1451
constexpr int arm_block_h = arm_block + ifce_h_n;  // per-CTA ARM partials with hyperlatents: 792
}  // namespace po

__host__ __device__ constexpr int ifce_w_off(int k) { return k == 0 ? po::if_w0 : (k == 1 ? po::if_w1 : po::if_w2); }
__host__ __device__ constexpr int ifce_b_off(int k) { return k == 0 ? po::if_b0 : (k == 1 ? po::if_b1 : po::if_b2); }
__host__ __device__ constexpr int ifce_nin(int k) { return k < kNIfce ? kL - k - 1 : 0; }

// Causal context offsets (dy, dx), nearest first; 3 rows up, 3 columns either side.
// (written as selects so that no lookup table is ever materialised in local memory)
//   n : 0  1  2  3  4  5  6  7  8  9 10 11 12 13 14 15
//   dy: 0 -1 -1 -1  0 -2 -1 -1 -2 -2 -2 -2  0 -3 -1 -1
//   dx:-1  0 -1  1 -2  0 -2  2 -1  1 -2  2 -3  0 -3  3
__host__ __device__ constexpr int ctx_dy(int n) {
    return (n == 0 || n == 4 || n == 12) ? 0 : (n == 5 || (n >= 8 && n <= 11)) ? -2 : (n == 13) ? -3 : -1;
}
__host__ __device__ constexpr int ctx_dx(int n) {
    return n == 0 ? -1 : n == 1 ? 0 : n == 2 ? -1 : n == 3 ? 1 : n == 4 ? -2 : n == 5 ? 0 : n == 6 ? -2
         : n == 7 ? 2 : n == 8 ? -1 : n == 9 ? 1 : n == 10 ? -2 : n == 11 ? 2 : n == 12 ? -3 : n == 13 ? 0
         : n == 14 ? -3 : 3;
}

// Grid slots k = 0..kL-1 are the latent grids (ceil(H/2^k) x ceil(W/2^k)); with hyperlatents
// (nh = kNH) slots kL..kL+kNH-1 are the hyperlatent grids, slot kL + q with the shape of latent
// grid kHB + q.  Unused slots are empty and start at the end of the latents, off[kG] = N.
struct Geom {
    int H, W, nh, pad_;
    int h[kG], w[kG];
    int64_t off[kG + 1];
};

inline Geom make_geom(int H, int W, int hyper = 0) {
    Geom g;
    g.H = H;
    g.W = W;
    g.nh = hyper ? kNH : 0;
    g.pad_ = 0;
    g.off[0] = 0;
    for (int k = 0; k < kG; ++k) {
        const int s = k < kL ? k : kHB + (k - kL);
        const bool used = k < kL + g.nh;
        g.h[k] = used ? (H + (1 << s) - 1) >> s : 0;
        g.w[k] = used ? (W + (1 << s) - 1) >> s : 0;
        g.off[k + 1] = g.off[k] + (int64_t)g.h[k] * g.w[k];
    }
    return g;
}

__device__ __forceinline__ int grid_of(const Geom& g, int64_t i) {
    int k = 0;
#pragma unroll
    for (int j = 1; j < kG; ++j) k += (i >= g.off[j]) ? 1 : 0;
    return k;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------------------------------------
// Counter noise: SplitMix64 output function (Steele, Lea, Flood 2014) of
// seed ^ ((step << 32) + i) * 0x9E3779B97F4A7C15; top 24 bits -> u in [-1/2, 1/2), exact in FP32.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t counter_hash(uint64_t seed, int64_t step, int64_t i) {
    uint64_t z = seed ^ ((((uint64_t)step << 32) + (uint64_t)i) * 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float counter_uniform(uint64_t seed, int64_t step, int64_t i) {
    return (float)(uint32_t)(counter_hash(seed, step, i) >> 40) * (1.f / 16777216.f) - 0.5f;
}
// Standard normal from the same hash by the Box-Muller transform (Box and Muller, 1958):
// u1 = (bits 40..63 + 1/2) / 2^24 in (0, 1), u2 = bits 16..39 / 2^24, n = sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ float counter_gauss(uint64_t seed, int64_t step, int64_t i) {
    const uint64_t z = counter_hash(seed, step, i);
    const float u1 = ((float)(uint32_t)(z >> 40) + 0.5f) * (1.f / 16777216.f);
    const float u2 = (float)(uint32_t)((z >> 16) & 0xFFFFFFull) * (1.f / 16777216.f);
    return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}
// Soft rounding, Eq. 14 (after Agustsson and Theis): s_T(x) = floor(x) + 1/2 + tanh(D / T) /
// (2 tanh(1 / (2T))), D = x - floor(x) - 1/2; d = s_T'(x) = (1 - tanh^2(D / T)) / (2 T tanh(1 / (2T))).
__device__ __forceinline__ float softround(float x, float T, float& d) {
    const float fl = floorf(x), D = x - fl - 0.5f, th = tanhf(D / T), den = 2.f * tanhf(0.5f / T);
    d = (1.f - th * th) / (T * den);
    return fl + 0.5f + th / den;
}

// ---------------------------------------------------------------------------------------------
// Laplace mass of [y - 1/2, y + 1/2] (Eq. 3), location mu, scale b = exp(logb), evaluated on the
// side of mu where it does not cancel; derivatives with respect to y and log b.
//   dP/dy = f(hi) - f(lo),  dP/dlogb = -(hi f(hi) - lo f(lo)),  f(z) = exp(-|z|/b) / (2b).
// ---------------------------------------------------------------------------------------------
struct LapOut {
    float p, dp_dy, dp_dlogb;
};

__device__ __forceinline__ LapOut laplace_mass(float y, float mu, float logb) {
    float b = expf(logb);
    float inv_b = __frcp_rn(b);
    float lo = y - 0.5f - mu, hi = y + 0.5f - mu;
    float el = expf(-fabsf(lo) * inv_b), eh = expf(-fabsf(hi) * inv_b);
    float p;
    if (lo >= 0.f)
        p = -0.5f * el * expm1f(-inv_b);
    else if (hi <= 0.f)
        p = -0.5f * eh * expm1f(-inv_b);
    else
        p = 1.f - 0.5f * el - 0.5f * eh;
    float fh = 0.5f * inv_b * eh, fl = 0.5f * inv_b * el;
    LapOut o;
    o.p = p;
    o.dp_dy = fh - fl;
    o.dp_dlogb = -(hi * fh - lo * fl);
    return o;
}

// Adam bias corrections 1 - beta^t (Sec. IV-B) as -expm1(t log(beta)) with log(beta) =
// log1p(beta - 1): FP32 with a relative error of a few 1e-7 at every t, where 1 - powf(beta, t)
// would lose most digits to cancellation at small t.
__device__ __forceinline__ void adam_bias_corrections(int64_t t, float beta1, float beta2, float& bc1, float& bc2) {
    const float tf = (float)t;
    bc1 = -expm1f(tf * log1pf(beta1 - 1.f));
    bc2 = -expm1f(tf * log1pf(beta2 - 1.f));
}

// ---------------------------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV values per thread, fixed order; result valid in thread 0.  `scratch`
// holds NV * (blockDim.x / 32) floats.
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) scratch[j * nw + wid] = v[j];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float s = 0.f;
            for (int q = 0; q < nw; ++q) s += scratch[j * nw + q];
            v[j] = s;
        }
    __syncthreads();
}

// Asynchronous 4-byte global -> shared copy (no register staging, latencies overlap);
// cp_async_wait_all() waits for all of this thread's copies.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// GELU, exact erf form, and its derivative.
// GELU with the exact (erf) Gaussian CDF, Phi(a) = (1 + erf(a / sqrt 2)) / 2, through the rational
// approximation of Abramowitz & Stegun formula 7.1.26 (Hastings):
//   erfc(x) = (a1 s + a2 s^2 + a3 s^3 + a4 s^4 + a5 s^5) exp(-x^2),  s = 1 / (1 + p x),  x >= 0,
// absolute error <= 1.5e-7 over the whole line.  Phi(-|a|) = erfc(|a| / sqrt 2) / 2 is taken
// straight from the product (no cancellation in the lower tail), Phi(|a|) = 1 - Phi(-|a|), and
// exp(-a^2 / 2) is shared with the derivative gelu'(a) = Phi(a) + a exp(-a^2 / 2) / sqrt(2 pi).
__device__ __forceinline__ float gelu_lower_tail(float a, float& ex) {  // Phi(-|a|); ex = exp(-a^2/2)
    const float x = fabsf(a) * 0.70710678118654752f;
    const float s = __fdividef(1.f, fmaf(0.3275911f, x, 1.f));
    float q = fmaf(1.061405429f, s, -1.453152027f);
    q = fmaf(q, s, 1.421413741f);
    q = fmaf(q, s, -0.284496736f);
    q = fmaf(q, s, 0.254829592f);
    ex = __expf(-x * x);
    return 0.5f * (q * s) * ex;
}
__device__ __forceinline__ float gelu_f(float a) {
    float ex;
    const float lt = gelu_lower_tail(a, ex);
    return a * (a < 0.f ? lt : 1.f - lt);
}
// gelu_f of two values in packed two-wide FP32 instructions: each component goes through exactly
// the operations of gelu_f (the packed multiply and fused multiply-add round like the scalar
// ones; the reciprocal and the exponential stay scalar calls), so the results are the same bits.
__device__ __forceinline__ float2 gelu2_f(float2 a) {
    const float2 x = __fmul2_rn(make_float2(fabsf(a.x), fabsf(a.y)), make_float2(0.70710678118654752f, 0.70710678118654752f));
    const float2 d = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), x, make_float2(1.f, 1.f));
    const float2 s = make_float2(__fdividef(1.f, d.x), __fdividef(1.f, d.y));
    float2 q = __ffma2_rn(make_float2(1.061405429f, 1.061405429f), s, make_float2(-1.453152027f, -1.453152027f));
    q = __ffma2_rn(q, s, make_float2(1.421413741f, 1.421413741f));
    q = __ffma2_rn(q, s, make_float2(-0.284496736f, -0.284496736f));
    q = __ffma2_rn(q, s, make_float2(0.254829592f, 0.254829592f));
    const float2 e = __fmul2_rn(make_float2(-x.x, -x.y), x);
    const float2 ex = make_float2(__expf(e.x), __expf(e.y));
    const float2 lt = __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), __fmul2_rn(q, s)), ex);
    return __fmul2_rn(a, make_float2(a.x < 0.f ? lt.x : 1.f - lt.x, a.y < 0.f ? lt.y : 1.f - lt.y));
}
// gelu(a) and gelu'(a) together
__device__ __forceinline__ void gelu_fg(float a, float& g, float& dg) {
    float ex;
    const float lt = gelu_lower_tail(a, ex);
    const float phi = a < 0.f ? lt : 1.f - lt;
    g = a * phi;
    dg = fmaf(a * 0.39894228040143268f, ex, phi);
}

// Polyphase taps of the x2 upsampler (Sec. III-B): output position o reads 4 inputs at
// p-2..p+1 (even o) or p-1..p+2 (odd o), p = o >> 1, with tap order
//   even: a c d b      odd: b d c a       (a, b, c, d = taps[0..3])
// Written with selects on constant indices so that nothing is indexed dynamically.
__device__ __forceinline__ int poly_first(int o) { return (o >> 1) - 2 + (o & 1); }
__device__ __forceinline__ int poly_tap(int o, int q) {  // tap index (0..3) of the q-th input
    const bool odd = o & 1;
    return q == 0 ? (odd ? 1 : 0) : q == 1 ? (odd ? 3 : 2) : q == 2 ? (odd ? 2 : 3) : (odd ? 0 : 1);
}
__device__ __forceinline__ void poly_w(int o, const float (&tp)[4], float (&w)[4]) {
    const bool odd = o & 1;
    w[0] = odd ? tp[1] : tp[0];
    w[1] = odd ? tp[3] : tp[2];
    w[2] = odd ? tp[2] : tp[3];
    w[3] = odd ? tp[0] : tp[1];
}

}  // namespace cc
