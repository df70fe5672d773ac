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

// IFCE gradient of a latent of grid g >= 3: sum over the finer grids k' = 0..2 of the block of
// grid-k' latents whose IFCE reads it, channel g - k' - 1 of dR_k'.  One warp per latent.
__global__ void k_ifce_pool(Geom g, const float* dR0, const float* dR1, const float* dR2, float* dIf) {
    const int lane = threadIdx.x & 31;
    const int64_t first = g.off[kNIfce], n = g.off[kL] - first;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = wid; j < n; j += nw) {
        const int64_t i = first + j;
        const int gg = grid_of(g, i);
        const int li = (int)(i - g.off[gg]);
        const int r = li / g.w[gg], c = li - r * g.w[gg];
        float acc = 0.f;
        for (int kp = 0; kp < kNIfce; ++kp) {
            const float* dR = kp == 0 ? dR0 : (kp == 1 ? dR1 : dR2);
            const int sh = gg - kp, ch = gg - kp - 1;
            const int hk = g.h[kp], wk = g.w[kp];
            const int r0 = r << sh, c0 = c << sh;
            const int bh = min(1 << sh, hk - r0), bw = min(1 << sh, wk - c0);
            const float* plane = dR + (int64_t)ch * hk * wk;
            for (int e = lane; e < bh * bw; e += 32) {
                const int rr = e / bw, cc = e - rr * bw;
                acc += plane[(int64_t)(r0 + rr) * wk + c0 + cc];
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) dIf[j] = acc;
    }
}

// Latent gradient: direct rate term + the 16 context users + IFCE users + upsampling/synthesis,
// then Adam on (y, m, v) or a copy to grad_out.
__global__ void k_gather(Geom g, const float* __restrict__ dYd, const float* __restrict__ dS,
                         const float* __restrict__ dR0, const float* __restrict__ dR1,
                         const float* __restrict__ dIf, const float* __restrict__ dYsyn, int zero_grad,
                         float* grad_out, float* y, float* m, float* v, Hp hp, const int64_t* step_dev) {
    __shared__ float s_bc[2];
    if (!grad_out) {
        if (threadIdx.x == 0) {
            const double t = (double)(*step_dev + 1);
            s_bc[0] = (float)(1.0 - pow((double)hp.beta1, t));
            s_bc[1] = (float)(1.0 - pow((double)hp.beta2, t));
        }
        __syncthreads();
    }
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
        } else if (k >= kNIfce) {
            acc += dIf[i - g.off[kNIfce]];
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
__global__ void k_param_reduce(const float* __restrict__ garm, int n_arm, const float* __restrict__ gup,
                               int2 n_up0, int2 n_up1, int2 n_up2, int2 n_up3, int2 n_up4, int2 n_up5,
                               const float* __restrict__ gsyn, int n_syn, const float* __restrict__ gconv,
                               int n_conv, float* params, float* m, float* v, float* grad_out,
                               float out_scale, Hp hp, const int64_t* step_dev) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= po::total) return;
    float s0 = 0.f, s1 = 0.f;
    if (p < po::up) {
        for (int q = 0; q + 1 < n_arm; q += 2) {
            s0 += garm[(int64_t)q * po::arm_block + p];
            s1 += garm[(int64_t)(q + 1) * po::arm_block + p];
        }
        if (n_arm & 1) s0 += garm[(int64_t)(n_arm - 1) * po::arm_block + p];
    } else if (p < po::syn_w1) {
        const int st = (p - po::up) >> 2, tap = (p - po::up) & 3;
        const int2 nn[6] = {n_up0, n_up1, n_up2, n_up3, n_up4, n_up5};
        for (int pass = 0; pass < 2; ++pass) {
            const int cnt = pass == 0 ? nn[st].x : nn[st].y;
            const float* base = gup + ((int64_t)(st * 2 + pass) * kUpMaxCta) * 4;
            for (int q = 0; q < cnt; ++q) s0 += base[q * 4 + tap];
        }
    } else if (p < po::cv1_w) {
        const int j = p - po::syn_w1;
        for (int q = 0; q + 1 < n_syn; q += 2) {
            s0 += gsyn[(int64_t)q * po::syn_block + j];
            s1 += gsyn[(int64_t)(q + 1) * po::syn_block + j];
        }
        if (n_syn & 1) s0 += gsyn[(int64_t)(n_syn - 1) * po::syn_block + j];
    } else {
        const int j = p - po::cv1_w;
        for (int q = 0; q < n_conv; ++q) s0 += gconv[(int64_t)q * po::conv_block + j];
    }
    const float gsum = s0 + s1;
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
    const int64_t n_coarse = w.N - w.g.off[kNIfce];
    if (n_coarse > 0) k_ifce_pool<<<grid_for(n_coarse * 32, 256, 8), 256, 0, s>>>(w.g, w.dR[0], w.dR[1], w.dR[2], w.dIf);
    k_gather<<<grid_for(w.N, 256, 8), 256, 0, s>>>(w.g, w.dYd, w.dS, w.dR[0], w.dR[1], w.dIf, w.dYsyn,
                                                   relax == kRelaxHard ? 1 : 0, grad_out, y, m, v, hp, step_dev);
}

void launch_param_reduce(const Work& w, float* params, float* m, float* v, float* grad_out, float out_scale,
                         const Hp& hp, const int64_t* step_dev, cudaStream_t s) {
    int2 nu[6];
    for (int st = 1; st < kL; ++st) nu[st - 1] = make_int2(w.n_cta_up[st][0], w.n_cta_up[st][1]);
    k_param_reduce<<<(po::total + 127) / 128, 128, 0, s>>>(w.gpart_arm, w.n_cta_arm, w.gpart_up, nu[0], nu[1], nu[2],
                                                           nu[3], nu[4], nu[5], w.gpart_syn, w.n_cta_syn, w.gpart_conv,
                                                           w.n_cta_conv, params, m, v, grad_out, out_scale, hp, step_dev);
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
