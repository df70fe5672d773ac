// Relaxation of the latents, assembly of the latent gradient (gather form), Adam (Sec. IV-B),
// fixed-order reduction of the per-CTA parameter gradients and the FP64 loss record (Eq. 10).
#include "cc_kernels.h"

namespace cc {
namespace {

__global__ void k_relax(const float* __restrict__ y, float* __restrict__ yt, int64_t N, uint64_t seed,
                        const int64_t* step_dev, int64_t step_host, int relax) {
    const int64_t step = step_dev ? *step_dev : step_host;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = y[i];
        yt[i] = relax == kRelaxNoise ? v + counter_uniform(seed, step, i) : (relax == kRelaxHard ? rintf(v) : v);
    }
}

// IFCE gradient reaching the coarse grids g >= 3, first stage.  A latent of grid g is read by
// the IFCE of grid k' (k' = 0..2) at every position of the 2^(g-k') x 2^(g-k') block under it,
// through channel g - k' - 1 of dR_k'.  Every such block is a union of the blocks under the
// grid-3 cells, so per grid-3 cell and per g: Q[g-3][cell] = sum_k' (block of 2^(3-k') x 2^(3-k')
// under the cell of dR_k' channel g - k' - 1).  One thread per (g, cell); fixed-size unrolled
// loads.  The gather kernel adds Q over the 2^(g-3) x 2^(g-3) cells under each grid-g latent.
template <int B>
__device__ __forceinline__ float block_sum_clipped(const float* __restrict__ plane, int h, int w, int r0, int c0) {
    float acc = 0.f;
#pragma unroll
    for (int rr = 0; rr < B; ++rr)
#pragma unroll
        for (int cc = 0; cc < B; ++cc)
            if (r0 + rr < h && c0 + cc < w) acc += __ldg(plane + (int64_t)(r0 + rr) * w + c0 + cc);
    return acc;
}

__global__ void k_ifce_cells(Geom g, const float* __restrict__ dR0, const float* __restrict__ dR1,
                             const float* __restrict__ dR2, float* Q) {
    const int n3 = g.h[3] * g.w[3];
    const int64_t n0 = (int64_t)g.h[0] * g.w[0], n1 = (int64_t)g.h[1] * g.w[1], n2 = (int64_t)g.h[2] * g.w[2];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 4 * (int64_t)n3;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int gg = 3 + (int)(e / n3), cell = (int)(e % n3);
        const int r3 = cell / g.w[3], c3 = cell - r3 * g.w[3];
        float acc = block_sum_clipped<8>(dR0 + (gg - 1) * n0, g.h[0], g.w[0], 8 * r3, 8 * c3);
        acc += block_sum_clipped<4>(dR1 + (gg - 2) * n1, g.h[1], g.w[1], 4 * r3, 4 * c3);
        acc += block_sum_clipped<2>(dR2 + (gg - 3) * n2, g.h[2], g.w[2], 2 * r3, 2 * c3);
        Q[e] = acc;
    }
}

// Latent gradient: direct rate term + the 16 context users + IFCE users + upsampling/synthesis,
// then Adam on (y, m, v) or a copy to grad_out.
__global__ void k_gather(Geom gp, const float* __restrict__ dYd, const float* __restrict__ dS,
                         const float* __restrict__ dR0, const float* __restrict__ dR1,
                         const float* __restrict__ dIf, const float* __restrict__ dYsyn, int zero_grad,
                         float* grad_out, float* y, float* m, float* v, Hp hp, const int64_t* step_dev) {
    __shared__ float s_bc[2];
    __shared__ Geom g;  // shared copy: the grid tables are indexed with a runtime grid number
    if (threadIdx.x == 0) {
        g = gp;
        if (!grad_out) {
            const double t = (double)(*step_dev + 1);
            s_bc[0] = (float)(1.0 - pow((double)hp.beta1, t));
            s_bc[1] = (float)(1.0 - pow((double)hp.beta2, t));
        }
    }
    __syncthreads();
    const int64_t N = g.off[kL];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = grid_of(g, i);
        const int hk = g.h[k], wk = g.w[k];
        const int li = (int)(i - g.off[k]);
        const int r = li / wk, c = li - r * wk;
        float acc = dYd[i] + dYsyn[i];
        const float* dSk = dS + g.off[k];
#pragma unroll
        for (int n = 0; n < kNCtx; ++n) {
            const int rr = r - ctx_dy(n), cc = c - ctx_dx(n);  // the latent that reads i via slot n
            if (rr < hk && cc >= 0 && cc < wk) acc += __ldg(dSk + (int64_t)n * N + rr * wk + cc);
        }
        if (k == 1 || k == 2) {
            // grid 1: 2x2 block of dR0 channel 0; grid 2: 4x4 block of dR0 channel 1, 2x2 of dR1 channel 0
            for (int kp = 0; kp < k; ++kp) {
                const float* dR = kp == 0 ? dR0 : dR1;
                const int sh = k - kp, ch = k - kp - 1;
                const int hkp = g.h[kp], wp = g.w[kp];
                const int r0 = r << sh, c0 = c << sh;
                const int bh = min(1 << sh, hkp - r0), bw = min(1 << sh, wp - c0);
                const float* plane = dR + (int64_t)ch * hkp * wp;
                for (int rr = 0; rr < bh; ++rr)
                    for (int cc = 0; cc < bw; ++cc) acc += __ldg(plane + (int64_t)(r0 + rr) * wp + c0 + cc);
            }
        } else if (k == kNIfce) {
            acc += dIf[li];
        } else if (k > kNIfce) {
            // grid k >= 4: the 2^(k-3) x 2^(k-3) grid-3 cells under (r, c), plane k-3 of Q
            const int sh = k - kNIfce, h3 = g.h[kNIfce], w3 = g.w[kNIfce];
            const float* plane = dIf + (int64_t)sh * h3 * w3;
            const int r0 = r << sh, c0 = c << sh;
            const int bh = min(1 << sh, h3 - r0), bw = min(1 << sh, w3 - c0);
            for (int rr = 0; rr < bh; ++rr)
                for (int cc = 0; cc < bw; ++cc) acc += plane[(int64_t)(r0 + rr) * w3 + c0 + cc];
        }
        if (zero_grad) acc = 0.f;
        if (grad_out) {
            grad_out[i] = acc;
        } else {
            const float mi = hp.beta1 * m[i] + (1.f - hp.beta1) * acc;
            const float vi = hp.beta2 * v[i] + (1.f - hp.beta2) * acc * acc;
            m[i] = mi;
            v[i] = vi;
            y[i] -= hp.lr * (mi / s_bc[0]) / (sqrtf(vi / s_bc[1]) + hp.eps);
        }
    }
}

// Fixed-order sum of the per-CTA partial parameter gradients, then Adam or a scaled copy.
// A CTA owns 32 consecutive parameters (one per lane); its 8 warps take interleaved slices of the
// partial rows (coalesced across lanes) and their sums are added in warp order.
struct UpCounts {
    int n[kL - 1];
};

__global__ void __launch_bounds__(256) k_param_reduce(const float* __restrict__ garm, int n_arm,
                                                      const float* __restrict__ gup, UpCounts nup,
                                                      const float* __restrict__ gsyn, int n_syn,
                                                      const float* __restrict__ gconv, int n_conv, float* params,
                                                      float* m, float* v, float* grad_out, float out_scale, Hp hp,
                                                      const int64_t* step_dev) {
    __shared__ float red[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    float a0 = 0.f, a1 = 0.f;
    if (p < po::total) {
        const float* base;
        int64_t stride;
        int cnt;
        if (p < po::up) {
            base = garm + p;
            stride = po::arm_block;
            cnt = n_arm;
        } else if (p < po::syn_w1) {
            const int st = (p - po::up) >> 2;
            base = gup + (int64_t)st * kUpMaxCta * 4 + ((p - po::up) & 3);
            stride = 4;
            cnt = nup.n[st];
        } else if (p < po::cv1_w) {
            base = gsyn + (p - po::syn_w1);
            stride = po::syn_block;
            cnt = n_syn;
        } else {
            base = gconv + (p - po::cv1_w);
            stride = po::conv_block;
            cnt = n_conv;
        }
        int q = wid;
        for (; q + 8 < cnt; q += 16) {
            a0 += __ldg(base + (int64_t)q * stride);
            a1 += __ldg(base + (int64_t)(q + 8) * stride);
        }
        if (q < cnt) a0 += __ldg(base + (int64_t)q * stride);
    }
    red[wid][lane] = a0 + a1;
    __syncthreads();
    if (wid != 0 || p >= po::total) return;
    float gsum = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) gsum += red[w][lane];
    if (grad_out) {
        grad_out[p] = gsum * out_scale;
        return;
    }
    const double t = (double)(*step_dev + 1);
    const float bc1 = (float)(1.0 - pow((double)hp.beta1, t));
    const float bc2 = (float)(1.0 - pow((double)hp.beta2, t));
    const float mi = hp.beta1 * m[p] + (1.f - hp.beta1) * gsum;
    const float vi = hp.beta2 * v[p] + (1.f - hp.beta2) * gsum * gsum;
    m[p] = mi;
    v[p] = vi;
    params[p] -= hp.lr * (mi / bc1) / (sqrtf(vi / bc2) + hp.eps);
}

// Loss record in FP64 from the rate and squared-error partials; optional history slot
// rd[step - base]; optional step increment.  One CTA.
__global__ void k_finish(const double* rate_part, int n_rate, const double* se_part, int n_se, double inv_hw,
                         double inv_3hw, double lambda, double* rd, int64_t* step_dev, int64_t* base_step,
                         int mark_base, int increment) {
    __shared__ double sr[256], ss[256];
    double r = 0.0, e = 0.0;
    for (int q = threadIdx.x; q < n_rate; q += blockDim.x) r += rate_part[q];
    for (int q = threadIdx.x; q < n_se; q += blockDim.x) e += se_part[q];
    sr[threadIdx.x] = r;
    ss[threadIdx.x] = e;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            ss[threadIdx.x] += ss[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rate = sr[0], mse = ss[0] * inv_3hw;
        const double loss = mse + lambda * rate * inv_hw;
        if (rd) {
            int64_t slot = 0;
            if (step_dev && base_step) slot = *step_dev - *base_step;
            rd[3 * slot + 0] = loss;
            rd[3 * slot + 1] = rate;
            rd[3 * slot + 2] = mse;
        }
        if (mark_base && step_dev && base_step) *base_step = *step_dev;
        if (increment && step_dev) *step_dev += 1;
    }
}

__global__ void k_mark_base(const int64_t* step_dev, int64_t* base_step) { *base_step = *step_dev; }

int grid_for(int64_t n, int threads, int per_sm) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

void launch_relax(const Work& w, const float* y, const int64_t* step_dev, int64_t step_host, uint64_t seed,
                  int relax, cudaStream_t s) {
    k_relax<<<grid_for(w.N, 256, 8), 256, 0, s>>>(y, w.yt, w.N, seed, step_dev, step_host, relax);
}

void launch_gather(const Work& w, const float* params, int relax, float* grad_out, float* y, float* m, float* v,
                   const Hp& hp, const int64_t* step_dev, cudaStream_t s) {
    (void)params;
    const int64_t n_cells = 4 * (int64_t)w.g.h[kNIfce] * w.g.w[kNIfce];
    k_ifce_cells<<<grid_for(n_cells, 128, 8), 128, 0, s>>>(w.g, w.dR[0], w.dR[1], w.dR[2], w.dIf);
    k_gather<<<grid_for(w.N, 256, 8), 256, 0, s>>>(w.g, w.dYd, w.dS, w.dR[0], w.dR[1], w.dIf, w.dYsyn,
                                                   relax == kRelaxHard ? 1 : 0, grad_out, y, m, v, hp, step_dev);
}

void launch_param_reduce(const Work& w, float* params, float* m, float* v, float* grad_out, float out_scale,
                         const Hp& hp, const int64_t* step_dev, cudaStream_t s) {
    UpCounts nu;
    for (int st = 1; st < kL; ++st) nu.n[st - 1] = w.n_cta_up[st];
    k_param_reduce<<<(po::total + 31) / 32, 256, 0, s>>>(w.gpart_arm, w.n_cta_arm, w.gpart_up, nu, w.gpart_syn,
                                                         w.n_cta_syn, w.gpart_conv, w.n_cta_conv, params, m, v,
                                                         grad_out, out_scale, hp, step_dev);
}

void launch_finish(const Work& w, const Hp& hp, int have_arm, int have_conv, double* rd_out, int64_t* step_dev,
                   int mark_base, int increment, cudaStream_t s) {
    k_finish<<<1, 256, 0, s>>>(w.rate_part, have_arm ? w.n_cta_arm : 0, w.se_part, have_conv ? w.n_cta_conv : 0,
                               1.0 / (double)w.HW, 1.0 / (3.0 * (double)w.HW), (double)hp.lambda, rd_out, step_dev,
                               w.base_step, mark_base, increment);
}

void launch_mark_base(const Work& w, const int64_t* step_dev, cudaStream_t s) {
    k_mark_base<<<1, 1, 0, s>>>(step_dev, w.base_step);
}

}  // namespace cc
