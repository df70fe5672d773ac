// Decoder-side integer entropy model (Sec. III-A; integer, platform-independent arithmetic as
// motivated in Sec. III-A2) and helpers of coolchic_decode_image.
//
// Fixed point with 8 fractional bits: w_q = rint(256 w) for every ARM and IFCE weight and bias;
// the spatial context enters as 256 q; each layer accumulates in 64-bit integers, adds its bias
// shifted to the product scale, shifts right by 8 (floor) and applies ReLU.  mu_q and logb_q are
// on a 1/256 grid, logb_q clamped to [-1280, 1280].  The CDF has 16-bit total mass:
//   C(t) = 65536 - E(s, t) (t >= 0),  E(s, -t) (t < 0),
//   E(s, u) = ((T_HI[hi] * T_LO[lo]) >> 15) >> n  with  v = u * K[s], n = v >> 28,
//   hi = (v >> 18) & 1023, lo = (v >> 8) & 1023, E = 0 once n >= 16,
//   K[s] = rint(2^20 log2(e) exp(-s/256)), T_HI[j] = rint(2^15 2^(-j/1024)), T_LO[j] = rint(2^15 2^(-j/2^20)),
// i.e. E ~ 2^15 exp(-u / (256 b)).  The tables are built here on the host in FP64 and copied
// to each device once; everything after them is integer arithmetic, hence bit-exact.  With
// hyperlatent grids (Sec. III-A3) their latents are decoded by the same model, and the IFCEs of
// grids 0..2 add the co-located hyperlatents times their 2^-8-grid weights.
#include <cmath>
#include <mutex>
#include <vector>

#include "cc_kernels.h"

namespace cc {
namespace {

constexpr int kSMin = -1280, kSMax = 1280;
__device__ long long d_K[kSMax - kSMin + 1];
__device__ int d_THI[1024];
__device__ int d_TLO[1024];

__device__ __forceinline__ long long q8(float w) { return (long long)rintf(w * 256.f); }

__device__ __forceinline__ long long cdf_q16(int s, long long t) {
    const long long u = t >= 0 ? t : -t;
    const long long v = u * d_K[s - kSMin];
    const long long n = v >> 28;
    long long e = 0;
    if (n < 16) e = (((long long)d_THI[(v >> 18) & 1023] * (long long)d_TLO[(v >> 8) & 1023]) >> 15) >> n;
    return t >= 0 ? 65536 - e : e;
}

__global__ void k_decode_arm(Geom gp, const int32_t* __restrict__ q, const float* __restrict__ P, float* yq,
                             uint32_t* prob, int32_t* mu_out, int32_t* logb_out) {
    __shared__ long long sW[po::arm_block];
    __shared__ long long sWh[po::ifce_h_n];  // hyperlatent IFCE weights [k][o][q]
    __shared__ Geom g;  // shared copy: the grid tables are indexed with a runtime grid number
    for (int j = threadIdx.x; j < po::arm_block; j += blockDim.x) sW[j] = q8(P[j]);
    for (int j = threadIdx.x; j < po::ifce_h_n; j += blockDim.x) sWh[j] = gp.nh ? q8(P[po::ifce_h + j]) : 0ll;
    if (threadIdx.x == 0) g = gp;
    __syncthreads();
    const int64_t N = g.off[kG];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = grid_of(g, i);
        const int wk = g.w[k];
        const int li = (int)(i - g.off[k]);
        const int r = li / wk, c = li - r * wk;
        const int32_t* qk = q + g.off[k];
        long long x[kAIn];
#pragma unroll
        for (int n = 0; n < kNCtx; ++n) {
            const int rr = r + ctx_dy(n), cc = c + ctx_dx(n);
            x[n] = (rr >= 0 && cc >= 0 && cc < wk) ? 256ll * qk[rr * wk + cc] : 0ll;
        }
        const int nin = ifce_nin(k);
        long long rv[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            rv[j] = 0;
            if (j < nin) {
                const int gj = k + 1 + j;
                const int rr = min(r >> (j + 1), g.h[gj] - 1), cc = min(c >> (j + 1), g.w[gj] - 1);
                rv[j] = q[g.off[gj] + rr * g.w[gj] + cc];
            }
        }
#pragma unroll
        for (int o = 0; o < kF; ++o) {
            long long acc = 0;
            if (nin > 0) {
                acc = sW[ifce_b_off(k) + o];
#pragma unroll
                for (int j = 0; j < 6; ++j)
                    if (j < nin) acc += sW[ifce_w_off(k) + o * nin + j] * rv[j];
                for (int hq = 0; hq < g.nh; ++hq) {
                    const int gq = kL + hq, sh = kHB + hq - k;
                    const int rr = min(r >> sh, g.h[gq] - 1), cc = min(c >> sh, g.w[gq] - 1);
                    acc += sWh[(k * kF + o) * kNH + hq] * (long long)q[g.off[gq] + rr * g.w[gq] + cc];
                }
            }
            x[kNCtx + o] = acc;
        }
        long long h1[kAH], h2[kAH];
#pragma unroll
        for (int o = 0; o < kAH; ++o) {
            long long acc = sW[po::arm_b1 + o] * 256;
#pragma unroll
            for (int n = 0; n < kAIn; ++n) acc += sW[po::arm_w1 + o * kAIn + n] * x[n];
            acc >>= 8;
            h1[o] = acc > 0 ? acc : 0;
        }
#pragma unroll
        for (int o = 0; o < kAH; ++o) {
            long long acc = sW[po::arm_b2 + o] * 256;
#pragma unroll
            for (int n = 0; n < kAH; ++n) acc += sW[po::arm_w2 + o * kAH + n] * h1[n];
            acc >>= 8;
            h2[o] = acc > 0 ? acc : 0;
        }
        long long out[2];
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            long long acc = (sW[po::arm_b3 + o] + sW[po::arm_bs + o]) * 256;
#pragma unroll
            for (int n = 0; n < kAH; ++n) acc += sW[po::arm_w3 + o * kAH + n] * h2[n];
#pragma unroll
            for (int n = 0; n < kAIn; ++n) acc += sW[po::arm_ws + o * kAIn + n] * x[n];
            out[o] = acc >> 8;
        }
        const long long mu = out[0];
        const int s = (int)(out[1] < kSMin ? kSMin : (out[1] > kSMax ? kSMax : out[1]));
        const long long yq256 = 256ll * q[i];
        const long long pq = cdf_q16(s, yq256 + 128 - mu) - cdf_q16(s, yq256 - 128 - mu);
        if (prob) prob[i] = (uint32_t)(pq < 1 ? 1 : pq);
        if (mu_out) mu_out[i] = (int32_t)mu;
        if (logb_out) logb_out[i] = s;
        if (yq) yq[i] = (float)q[i];
    }
}

__global__ void k_clamp01(float* x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fminf(fmaxf(x[i], 0.f), 1.f);
}

std::mutex g_tab_mu;
std::vector<int> g_tab_ready;  // per device

}  // namespace

void decode_init_tables() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if ((int)g_tab_ready.size() <= dev) g_tab_ready.resize(dev + 1, 0);
    if (g_tab_ready[dev]) return;
    std::vector<long long> K(kSMax - kSMin + 1);
    std::vector<int> thi(1024), tlo(1024);
    const double log2e = 1.0 / std::log(2.0);
    for (int s = kSMin; s <= kSMax; ++s) K[s - kSMin] = (long long)std::rint(1048576.0 * log2e * std::exp(-(double)s / 256.0));
    for (int j = 0; j < 1024; ++j) {
        thi[j] = (int)std::rint(32768.0 * std::exp2(-(double)j / 1024.0));
        tlo[j] = (int)std::rint(32768.0 * std::exp2(-(double)j / 1048576.0));
    }
    cudaMemcpyToSymbol(d_K, K.data(), K.size() * sizeof(long long));
    cudaMemcpyToSymbol(d_THI, thi.data(), thi.size() * sizeof(int));
    cudaMemcpyToSymbol(d_TLO, tlo.data(), tlo.size() * sizeof(int));
    g_tab_ready[dev] = 1;
}

void launch_decode(const Geom& g, const int32_t* q, const float* params, float* yq, uint32_t* prob, int32_t* mu_q,
                   int32_t* logb_q, cudaStream_t s) {
    const int64_t N = g.off[kG];
    int64_t blocks = (N + 127) / 128;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    k_decode_arm<<<(int)blocks, 128, 0, s>>>(g, q, params, yq, prob, mu_q, logb_q);
}

void launch_clamp01(float* x, int64_t n, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    k_clamp01<<<(int)blocks, 256, 0, s>>>(x, n);
}

}  // namespace cc
