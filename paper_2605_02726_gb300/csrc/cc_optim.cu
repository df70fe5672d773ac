// Relaxation of the latents, assembly of the latent gradient (gather form), Adam (Sec. IV-B),
// fixed-order reduction of the per-CTA parameter gradients and the FP64 loss record (Eq. 10).
// Each kernel has a body over (arguments, CTA index within the job, CTA count of the job), a
// single-job entry and a multi-job entry.
#include "cc_kernels.h"
#include "cc_upfwd.cuh"

namespace cc {
namespace {

// ---------------------------------------------------------------------------------------------
// a1: y~ = y + u(seed, step, i) | s_T(s_T(y) + sigma n) (Eq. 13, in its schedule) | rint(y) | y
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void relax_body(const RelaxArgs& a, int cta, int ncta) {
    __shared__ ProxyAt s_px;  // the proxy at this step, once per CTA
    __shared__ int64_t s_step;
    if (threadIdx.x == 0) {
        s_step = a.step_dev ? *a.step_dev : a.step_host;
        s_px = proxy_at(a.hp, s_step);
    }
    __syncthreads();
    const int64_t step = s_step;
    for (int64_t i = cta * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)ncta * blockDim.x) {
        const float v = a.y[i];
        float jac;
        a.yt[i] = a.relax == kRelaxNoise ? relax_latent(a.hp, s_px, v, step, i, jac)
                                         : (a.relax == kRelaxHard ? rintf(v) : v);
    }
}
__global__ void k_relax(const __grid_constant__ RelaxArgs a) {
    pdl_enter();
    relax_body(a, blockIdx.x, gridDim.x);
}
__global__ void k_relax_b(Batch<RelaxArgs> b) {
    __shared__ RelaxArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    relax_body(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

// ---------------------------------------------------------------------------------------------
// IFCE gradient reaching the coarse grids g >= 3, first stage.  A latent of grid g is read by
// the IFCE of grid k' (k' = 0..2) at every position of the 2^(g-k') x 2^(g-k') block under it,
// through channel g - k' - 1 of dR_k'.  Every such block is a union of the blocks under the
// grid-3 cells, so per grid-3 cell and per g: Q[g-3][cell] = sum_k' (block of 2^(3-k') x 2^(3-k')
// under the cell of dR_k' channel g - k' - 1).  One thread per (g, cell); fixed-size unrolled
// loads.  The gather kernel adds Q over the 2^(g-3) x 2^(g-3) cells under each grid-g latent.
// Hyperlatent grid q (the shape of grid 4 + q) is input 6 - k' + q of IFCE k', i.e. channel
// 2 + (4 + q) - k' as well: its plane is Q[4 + q], the same formula with "g" = 7 + q.
// ---------------------------------------------------------------------------------------------
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

// one row of a B-wide block, clipped to the plane
template <int B>
__device__ __forceinline__ float row_sum_clipped(const float* __restrict__ plane, int h, int w, int r, int c0) {
    float acc = 0.f;
    if (r < h)
#pragma unroll
        for (int cc = 0; cc < B; ++cc)
            if (c0 + cc < w) acc += __ldg(plane + (int64_t)r * w + c0 + cc);
    return acc;
}

// Eight consecutive threads per (g, cell): thread p sums row p of the 8x8 block of dR0, row p of
// the 4x4 block of dR1 (p < 4) and row p of the 2x2 block of dR2 (p < 2); the eight partial sums
// are added by shuffles in a fixed order.
__device__ __forceinline__ void ifce_body(const IfceArgs& a, int cta, int ncta) {
    const Geom& g = a.g;
    const int n3 = g.h[3] * g.w[3];
    const int64_t n0 = (int64_t)g.h[0] * g.w[0], n1 = (int64_t)g.h[1] * g.w[1], n2 = (int64_t)g.h[2] * g.w[2];
    const int64_t total = (4 + g.nh) * (int64_t)n3 * 8;  // a multiple of 8: the 8 threads of a task share a warp
    // the loop runs while any lane of the warp has a task, so that every lane takes part in the shuffles
    for (int64_t e = cta * (int64_t)blockDim.x + threadIdx.x; e - (int)(threadIdx.x & 31) < total;
         e += (int64_t)ncta * blockDim.x) {
        const bool live = e < total;
        const int64_t task = live ? e >> 3 : 0;
        const int p = (int)(e & 7);
        const int gg = 3 + (int)(task / n3), cell = (int)(task % n3);
        const int r3 = cell / g.w[3], c3 = cell - r3 * g.w[3];
        float acc = 0.f;
        if (live) {
            acc = row_sum_clipped<8>(a.dR0 + (gg - 1) * n0, g.h[0], g.w[0], 8 * r3 + p, 8 * c3);
            if (p < 4) acc += row_sum_clipped<4>(a.dR1 + (gg - 2) * n1, g.h[1], g.w[1], 4 * r3 + p, 4 * c3);
            if (p < 2) acc += row_sum_clipped<2>(a.dR2 + (gg - 3) * n2, g.h[2], g.w[2], 2 * r3 + p, 2 * c3);
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (live && p == 0) a.Q[task] = acc;
    }
}
__global__ void k_ifce_cells(const __grid_constant__ IfceArgs a) {
    pdl_enter();
    ifce_body(a, blockIdx.x, gridDim.x);
}
__global__ void k_ifce_cells_b(Batch<IfceArgs> b) {
    __shared__ IfceArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    ifce_body(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}
// Encoder iterations: the first forward upsampling stage after the entropy model and the IFCE cell
// sums in one launch.  CTAs [0, n_up) run the stage, the others the cell sums, which read only the
// entropy model's IFCE-input gradients and are read only by the gather; the iteration's chain of
// dependent launches is one launch shorter.  Both bodies are light (few registers, no shared
// memory), so sharing one launch configuration costs neither of them occupancy.
// The launch's first thread also copies the step to the iteration's snapshot (every earlier
// launch of the iteration has completed: the step is the one this iteration updates with).
__global__ void __launch_bounds__(kUpThreads) k_up_fwd_ifce(const __grid_constant__ UpFwdArgs u,
                                                            const __grid_constant__ IfceArgs f, int n_up,
                                                            const int64_t* step_dev, int64_t* step_snap) {
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) *step_snap = *step_dev;
    if ((int)blockIdx.x < n_up)
        up_fwd_body(u, blockIdx.x, n_up);
    else
        ifce_body(f, blockIdx.x - n_up, gridDim.x - n_up);
}

// ---------------------------------------------------------------------------------------------
// Latent gradient: direct rate term + the 16 context users + IFCE users + upsampling/synthesis,
// then Adam on (y, m, v) or a copy to grad_out.  `a` must be in shared memory (its grid tables are
// indexed with a runtime grid number).  The per-launch scalars (1/w of every grid, the Adam bias
// corrections, the proxy at this step and the next) are computed once per CTA; a latent
// finds its row by a float reciprocal corrected to the exact quotient, and latents whose 16
// context users all lie inside the grid load them without bounds tests.
// ---------------------------------------------------------------------------------------------
struct GatherScalars {
    float invw[kG];
    float bc1, bc2;
    ProxyAt px, px_next;
    int64_t step;
};

// r = li / w, c = li % w for 0 <= li < 2^22: the float estimate is within one of the quotient
// there, and one correction makes it exact; larger indices take the integer division.
__device__ __forceinline__ void row_col(int li, int w, float invw, int& r, int& c) {
    if (li < (1 << 22)) {
        r = (int)((float)li * invw);
        c = li - r * w;
        if (c < 0) {
            --r;
            c += w;
        } else if (c >= w) {
            ++r;
            c -= w;
        }
    } else {
        r = li / w;
        c = li - r * w;
    }
}

__device__ __forceinline__ void gather_body(const GatherArgs& a, int cta, int ncta) {
    // the per-launch scalars on four warps at once (the grid tables are read from `a`)
    __shared__ GatherScalars sc;
    {
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0 && wid < 3) {
            const int64_t step = a.step_dev ? *a.step_dev : a.step_host;
            if (wid == 0) {
                sc.step = step;
                sc.bc1 = sc.bc2 = 1.f;
                if (!a.grad_out) adam_bias_corrections(step + 1, a.hp.beta1, a.hp.beta2, sc.bc1, sc.bc2);
            } else if (wid == 1) {
                sc.px = proxy_at(a.hp, step);
            } else {
                sc.px_next = proxy_at(a.hp, step + 1);
            }
        } else if (wid == 3 && lane < kG) {
            sc.invw[lane] = a.g.w[lane] > 0 ? 1.f / (float)a.g.w[lane] : 0.f;
        }
    }
    __syncthreads();
    const Geom& g = a.g;
    const int64_t step = sc.step;
    const int64_t N = g.off[kG];  // with hyperlatent grids, their latents too
    const float* __restrict__ dS = a.dS;
    for (int64_t i = cta * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)ncta * blockDim.x) {
        const int k = grid_of(g, i);
        const int hk = g.h[k], wk = g.w[k];
        const int li = (int)(i - g.off[k]);
        int r, c;
        row_col(li, wk, sc.invw[k], r, c);
        // latent i is slot n of the latent at (r - dy_n, c - dx_n): plane n at li - dy_n*wk - dx_n
        const float* p0 = dS + g.off[k] + li;
        float v[kNCtx];
        if (r + 3 < hk && c >= 3 && c + 3 < wk) {
#pragma unroll
            for (int n = 0; n < kNCtx; ++n) v[n] = __ldg(p0 + (int64_t)n * N - ctx_dy(n) * wk - ctx_dx(n));
        } else {
#pragma unroll
            for (int n = 0; n < kNCtx; ++n) {
                const int rr = r - ctx_dy(n), cc = c - ctx_dx(n);
                v[n] = (rr < hk && cc >= 0 && cc < wk) ? __ldg(p0 + (int64_t)n * N - ctx_dy(n) * wk - ctx_dx(n)) : 0.f;
            }
        }
        // (hyperlatents reach neither the upsampling nor the synthesis)
        float acc = a.dYd[i] + (k < kL ? a.dYsyn[i] : 0.f);
#pragma unroll
        for (int n = 0; n < kNCtx; ++n) acc += v[n];
        // IFCE users, as blocks summed with all their loads in flight (unrolled, clipped to the grid)
        if (k == 1) {  // 2x2 block of dR0 channel 0
            acc += block_sum_clipped<2>(a.dR0, g.h[0], g.w[0], 2 * r, 2 * c);
        } else if (k == 2) {  // 4x4 block of dR0 channel 1, 2x2 block of dR1 channel 0
            const int64_t n0 = (int64_t)g.h[0] * g.w[0];
            acc += block_sum_clipped<4>(a.dR0 + n0, g.h[0], g.w[0], 4 * r, 4 * c);
            acc += block_sum_clipped<2>(a.dR1, g.h[1], g.w[1], 2 * r, 2 * c);
        } else if (k == kNIfce) {
            acc += a.dIf[li];
        } else if (k > kNIfce) {
            // grid k >= 4: the 2^(k-3) x 2^(k-3) grid-3 cells under (r, c), plane k-3 of Q;
            // hyperlatent grid k = 7 + q: the grid of level 4 + q, plane 4 + q
            const int lev = k < kL ? k : kHB + (k - kL);
            const int sh = lev - kNIfce, h3 = g.h[kNIfce], w3 = g.w[kNIfce];
            const float* plane = a.dIf + (int64_t)(k < kL ? sh : k - kNIfce) * h3 * w3;
            const int r0 = r << sh, c0 = c << sh;
            acc += sh == 1 ? block_sum_clipped<2>(plane, h3, w3, r0, c0)
                 : sh == 2 ? block_sum_clipped<4>(plane, h3, w3, r0, c0)
                           : block_sum_clipped<8>(plane, h3, w3, r0, c0);
        }
        if (a.zero_grad) acc = 0.f;
        const float yi = a.y[i];
        if (a.proxy && a.hp.noise_mode != 0) {  // chain rule through y~ = Q_train(y)
            float jac;
            relax_latent(a.hp, sc.px, yi, step, i, jac);
            acc *= jac;
        }
        if (a.grad_out) {
            a.grad_out[i] = acc;
        } else {
            float yn = yi;
            if (!sc.px.hard) {  // the hard-round stage leaves the latents (and their moments) alone
                const float mi = a.hp.beta1 * a.m[i] + (1.f - a.hp.beta1) * acc;
                const float vi = a.hp.beta2 * a.v[i] + (1.f - a.hp.beta2) * acc * acc;
                a.m[i] = mi;
                a.v[i] = vi;
                yn = yi - sc.px.lr * (mi / sc.bc1) / (sqrtf(vi / sc.bc2) + a.hp.eps);
                a.y[i] = yn;
            }
            if (a.yt_next) {
                float jac;
                a.yt_next[i] = relax_latent(a.hp, sc.px_next, yn, step + 1, i, jac);
            }
        }
    }
}
__global__ void __launch_bounds__(256, 4) k_gather(const __grid_constant__ GatherArgs a) {
    __shared__ GatherArgs sa;
    param_fetch(a, sa);
    gather_body(sa, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256, 4) k_gather_b(Batch<GatherArgs> b) {
    __shared__ GatherArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    gather_body(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

// ---------------------------------------------------------------------------------------------
// Fixed-order sum of the per-CTA partial parameter gradients, then Adam or a scaled copy.
// A CTA owns 32 consecutive parameters (one per lane); its 32 warps take interleaved rows of the
// partials (coalesced across lanes, all of a warp's rows in flight at once when they number at
// most 16, the usual case) and their sums are added in warp order.  The Adam operands (step,
// moments, parameter) are loaded before the partials, so their round trip overlaps.  A job has
// kReduceCtas CTAs.
// ---------------------------------------------------------------------------------------------
constexpr int kReduceCtas = (po::total_h + 31) / 32;  // CTAs past the job's parameters return
constexpr int kReduceThreads = 256, kReduceWarps = kReduceThreads / 32;  // (the gather's CTA size: see k_gather_reduce)

__device__ __forceinline__ void reduce_body(const ReduceArgs& a, int cta) {
    __shared__ float red[kReduceWarps][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int p = cta * 32 + lane;
    const int n_par = a.hyper ? po::total_h : po::total;
    const bool adam = !a.grad_out && wid == 0 && p < n_par;
    int64_t step = 0;
    float m0 = 0.f, v0 = 0.f, p0 = 0.f;
    if (adam) {
        step = *a.step_dev;
        m0 = a.m[p];
        v0 = a.v[p];
        p0 = a.params[p];
    }
    float acc = 0.f;
    if (p < n_par) {
        const float* base;
        int64_t stride;
        int cnt;
        const int arm_row = a.hyper ? po::arm_block_h : po::arm_block;
        if (p < po::up) {
            base = a.garm + p;
            stride = arm_row;
            cnt = a.n_arm;
        } else if (p >= po::total) {  // hyperlatent IFCE weights: entries 756.. of the ARM rows
            base = a.garm + po::arm_block + (p - po::ifce_h);
            stride = arm_row;
            cnt = a.n_arm;
        } else if (p < po::syn_w1) {
            const int st = (p - po::up) >> 2;
            base = a.gup + (int64_t)st * kUpMaxCta * 4 + ((p - po::up) & 3);
            stride = 4;
            cnt = a.nup[st];
        } else if (p < po::cv1_w) {
            base = a.gsyn + (p - po::syn_w1);
            stride = po::syn_block;
            cnt = a.n_syn;
        } else {
            base = a.gconv + (p - po::cv1_w);
            stride = po::conv_block;
            cnt = a.n_conv;
        }
        // rows wid, wid + 32, ..., 16 per pass, added as a fixed pairwise tree
        constexpr int RW = kReduceWarps, kU = 16;
        for (int q = wid; q < cnt; q += kU * RW) {
            float v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) v[u] = q + RW * u < cnt ? __ldg(base + (int64_t)(q + RW * u) * stride) : 0.f;
#pragma unroll
            for (int w = kU / 2; w > 0; w >>= 1)
#pragma unroll
                for (int u = 0; u < w; ++u) v[u] += v[u + w];
            acc += v[0];
        }
    }
    red[wid][lane] = acc;
    __syncthreads();
    if (wid != 0 || p >= n_par) return;
    float gsum = 0.f;
#pragma unroll
    for (int w = 0; w < kReduceWarps; ++w) gsum += red[w][lane];
    if (a.grad_out) {
        a.grad_out[p] = gsum * a.out_scale;
        return;
    }
    if (a.hp.nn_opt == 1 && soap_param(p)) {  // updated by the SOAP kernel that follows
        a.gsoap[p] = gsum;
        return;
    }
    float bc1, bc2;
    adam_bias_corrections(step + 1, a.hp.beta1, a.hp.beta2, bc1, bc2);
    const float lr = proxy_at(a.hp, step).lr;
    const float mi = a.hp.beta1 * m0 + (1.f - a.hp.beta1) * gsum;
    const float vi = a.hp.beta2 * v0 + (1.f - a.hp.beta2) * gsum * gsum;
    a.m[p] = mi;
    a.v[p] = vi;
    a.params[p] = p0 - lr * (mi / bc1) / (sqrtf(vi / bc2) + a.hp.eps);
}
__global__ void __launch_bounds__(kReduceThreads) k_param_reduce(const __grid_constant__ ReduceArgs a) {
    __shared__ ReduceArgs sa;
    param_fetch(a, sa);
    reduce_body(sa, blockIdx.x);
}
__global__ void __launch_bounds__(kReduceThreads) k_param_reduce_b(Batch<ReduceArgs> b) {
    __shared__ ReduceArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    reduce_body(sa, blockIdx.x - b.cta_begin[j]);
}

// ---------------------------------------------------------------------------------------------
// Loss record in FP64 from the rate and squared-error partials; optional history slot
// rd[(step - base) * rd_stride]; optional step increment.  One CTA of 256 threads per job.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void finish_body(const FinishArgs& a) {
    __shared__ double sr[256], ss[256];
    int64_t step = 0, base = 0;  // loaded up front: their round trip overlaps the partials'
    if (threadIdx.x == 0 && a.step_dev) {
        step = *a.step_dev;
        if (a.base_step) base = *a.base_step;
    }
    double r = 0.0, e = 0.0;
    for (int q = threadIdx.x; q < a.n_rate; q += blockDim.x) r += a.rate_part[q];
    for (int q = threadIdx.x; q < a.n_se; q += blockDim.x) e += a.se_part[q];
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
        const double rate = sr[0], mse = ss[0] * a.inv_3hw;
        const double loss = mse + a.lambda * rate * a.inv_hw;
        if (a.rd) {
            int64_t slot = 0;
            if (a.step_dev && a.base_step) slot = step - base;
            double* o = a.rd + slot * a.rd_stride;
            o[0] = loss;
            o[1] = rate;
            o[2] = mse;
        }
        if (a.mark_base && a.step_dev && a.base_step) *a.base_step = step;
        if (a.increment && a.step_dev) *a.step_dev = step + 1;
    }
}
__global__ void k_finish(const __grid_constant__ FinishArgs a) {
    pdl_enter();
    finish_body(a);
}
__global__ void k_finish_b(Batch<FinishArgs> b) {
    __shared__ FinishArgs sa;
    batch_fetch(b.args, blockIdx.x, sa);
    finish_body(sa);
}

// Encoder iterations: the parameter reduction (the first kReduceCtas CTAs), the loss record with the
// step increment (the next CTA) and the latent gather (the others) in one launch.  The reduction
// reads only the per-CTA partial gradients and the record only the rate and squared-error partials,
// all written before the gather, and no part reads what another writes: the reduction and the
// gather read the step from the iteration's snapshot, not from the word the finish increments.  So
// they run beside the gather instead of after it: two launches fewer on the iteration's dependent
// chain.  The reduction CTAs and the finish come first so that the launch stays one wave at the
// gather's four CTAs per SM.
__global__ void __launch_bounds__(256, 4) k_gather_reduce(const __grid_constant__ GatherArgs g,
                                                          const __grid_constant__ ReduceArgs r,
                                                          const __grid_constant__ FinishArgs f) {
    if ((int)blockIdx.x < kReduceCtas) {
        __shared__ ReduceArgs sr;
        param_fetch(r, sr);
        reduce_body(sr, blockIdx.x);
    } else if ((int)blockIdx.x == kReduceCtas) {
        pdl_enter();
        finish_body(f);
    } else {
        __shared__ GatherArgs sg;
        param_fetch(g, sg);
        gather_body(sg, blockIdx.x - (kReduceCtas + 1), gridDim.x - (kReduceCtas + 1));
    }
}

__global__ void k_mark_base(const int64_t* step_dev, int64_t* base_step) { *base_step = *step_dev; }

// ---------------------------------------------------------------------------------------------
// Seeded initial state (no counterpart in the paper, which does not give its initialisation):
// latents 0.01 n_i, n_i the Box-Muller normal of the counter hash at (seed, step -1, i); hidden
// weights (ARM W1, W2, the IFCE matrices, synthesis W1) 2 u_p / sqrt(fan_in), u_p the uniform of
// the hash at (seed, step -2, p); bicubic taps; every other parameter, the moments and the step 0.
// (Negative steps: the encoder's own draws use steps >= 0.)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float init_param(uint64_t seed, int p, int nh) {
    int fan = 0;  // an IFCE's fan-in counts its hyperlatent inputs when there are some
    if (p >= po::arm_w1 && p < po::arm_b1) fan = 20;
    else if (p >= po::arm_w2 && p < po::arm_b2) fan = 16;
    else if (p >= po::if_w0 && p < po::if_b0) fan = ifce_nin(0) + nh;
    else if (p >= po::if_w1 && p < po::if_b1) fan = ifce_nin(1) + nh;
    else if (p >= po::if_w2 && p < po::if_b2) fan = ifce_nin(2) + nh;
    else if (p >= po::syn_w1 && p < po::syn_b1) fan = 7;
    else if (p >= po::ifce_h) fan = ifce_nin((p - po::ifce_h) / (kF * kNH)) + nh;
    if (fan) return 2.f * counter_uniform(seed, -2, p) / sqrtf((float)fan);
    if (p >= po::up && p < po::syn_w1) {  // Keys cubic (a = -0.75) at 1.75, 1.25, 0.75, 0.25
        const int j = (p - po::up) & 3;
        return j == 0 ? -0.03515625f : j == 1 ? -0.10546875f : j == 2 ? 0.26171875f : 0.87890625f;
    }
    return 0.f;
}
__global__ void k_init_state(const __grid_constant__ InitArgs a) {
    const int n_par = a.nh ? po::total_h : po::total;
    const int64_t n_all = a.N + n_par;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_all; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < a.N) {
            a.y[e] = 0.01f * counter_gauss(a.seed, -1, e);
            a.m_lat[e] = 0.f;
            a.v_lat[e] = 0.f;
        } else {
            const int p = (int)(e - a.N);
            a.params[p] = init_param(a.seed, p, a.nh);
            a.m_par[p] = 0.f;
            a.v_par[p] = 0.f;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.step = 0;
}
__global__ void k_mark_base_b(Batch<FinishArgs> b) {
    if (threadIdx.x == 0) *b.args[blockIdx.x].base_step = *b.args[blockIdx.x].step_dev;
}

}  // namespace

int grid_for(int64_t n, int threads, int per_sm) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ---- argument builders
RelaxArgs relax_args(const Work& w, const float* y, const int64_t* step_dev, int64_t step_host, const Hp& hp,
                     int relax) {
    RelaxArgs a;
    a.y = y;
    a.yt = w.yt;
    a.N = w.N;
    a.step_dev = step_dev;
    a.step_host = step_host;
    a.hp = hp;
    a.relax = relax;
    a.pad_ = 0;
    return a;
}
IfceArgs ifce_args(const Work& w) {
    IfceArgs a;
    a.g = w.g;
    a.dR0 = w.dR[0];
    a.dR1 = w.dR[1];
    a.dR2 = w.dR[2];
    a.Q = w.dIf;
    return a;
}
GatherArgs gather_args(const Work& w, int relax, float* grad_out, float* y, float* m, float* v, const Hp& hp,
                       const int64_t* step_dev, int64_t step_host, bool relax_next) {
    GatherArgs a;
    a.g = w.g;
    a.dYd = w.dYd;
    a.dS = w.dS;
    a.dR0 = w.dR[0];
    a.dR1 = w.dR[1];
    a.dIf = w.dIf;
    a.dYsyn = w.dYsyn;
    a.grad_out = grad_out;
    a.y = y;
    a.m = m;
    a.v = v;
    a.step_dev = step_dev;
    a.step_host = step_host;
    a.yt_next = (relax_next && !grad_out) ? w.yt : nullptr;
    a.hp = hp;
    a.zero_grad = relax == kRelaxHard ? 1 : 0;
    a.proxy = relax == kRelaxNoise ? 1 : 0;
    return a;
}
ReduceArgs reduce_args(const Work& w, float* params, float* m, float* v, float* grad_out, float out_scale,
                       const Hp& hp, const int64_t* step_dev) {
    ReduceArgs a;
    a.gsoap = w.grad_params;
    a.hyper = w.g.nh > 0 ? 1 : 0;
    a.garm = w.gpart_arm;
    a.gup = w.gpart_up;
    a.gsyn = w.gpart_syn;
    a.gconv = w.gpart_conv;
    a.params = params;
    a.m = m;
    a.v = v;
    a.grad_out = grad_out;
    a.step_dev = step_dev;
    a.hp = hp;
    a.n_arm = w.n_cta_arm;
    a.n_syn = w.n_cta_syn;
    a.n_conv = w.n_cta_conv;
    for (int st = 1; st < kL; ++st) a.nup[st - 1] = w.n_cta_up[st];
    a.out_scale = out_scale;
    return a;
}
FinishArgs finish_args(const Work& w, const Hp& hp, int have_arm, int have_conv, double* rd, int rd_stride,
                       int64_t* step_dev, int mark_base, int increment) {
    FinishArgs a;
    a.rate_part = w.rate_part;
    a.se_part = w.se_part;
    a.rd = rd;
    a.step_dev = step_dev;
    a.base_step = w.base_step;
    a.inv_hw = 1.0 / (double)w.HW;
    a.inv_3hw = 1.0 / (3.0 * (double)w.HW);
    a.lambda = (double)hp.lambda;
    a.n_rate = have_arm ? w.n_cta_arm : 0;
    a.n_se = have_conv ? w.n_cta_conv : 0;
    a.rd_stride = rd_stride;
    a.mark_base = mark_base;
    a.increment = increment;
    a.pad_ = 0;
    return a;
}

int relax_ctas(const Work& w) { return grid_for(w.N, 256, 8); }
int ifce_ctas(const Work& w) { return grid_for(8 * (4 + w.g.nh) * (int64_t)w.g.h[kNIfce] * w.g.w[kNIfce], 128, 16); }
int gather_ctas(const Work& w) { return grid_for(w.N, 256, 4); }  // one wave at 4 CTAs per SM
int reduce_ctas() { return kReduceCtas; }

// ---- single-job launches
void launch_relax(const Work& w, const float* y, const int64_t* step_dev, int64_t step_host, const Hp& hp,
                  int relax, cudaStream_t s) {
    launch_pdl(k_relax, relax_ctas(w), 256, 0, s, relax_args(w, y, step_dev, step_host, hp, relax));
}

void launch_up_fwd_ifce(const Work& w, const float* params, int m, const int64_t* step_dev, cudaStream_t s) {
    const int n_up = up_fwd_ctas(w, m);
    const int n_if = grid_for(8 * (4 + w.g.nh) * (int64_t)w.g.h[kNIfce] * w.g.w[kNIfce], kUpThreads, 8);
    launch_pdl(k_up_fwd_ifce, n_up + n_if, kUpThreads, 0, s, up_fwd_args(w, params, m), ifce_args(w), n_up, step_dev,
               w.step_snap);
}

void launch_gather(const Work& w, const float* params, int relax, float* grad_out, float* y, float* m, float* v,
                   const Hp& hp, const int64_t* step_dev, int64_t step_host, cudaStream_t s, bool relax_next) {
    (void)params;
    if (!w.ifce_early) launch_pdl(k_ifce_cells, ifce_ctas(w), 128, 0, s, ifce_args(w));
    launch_pdl(k_gather, gather_ctas(w), 256, 0, s,
               gather_args(w, relax, grad_out, y, m, v, hp, step_dev, step_host, relax_next));
}

void launch_gather_reduce(const Work& w, float* y, float* m_lat, float* v_lat, float* params, float* m_par,
                          float* v_par, const Hp& hp, int64_t* step_dev, double* rd_out, cudaStream_t s,
                          bool relax_next) {
    static_assert(kReduceThreads == 256, "the reduction shares the gather's CTA size");
    constexpr int lead = kReduceCtas + 1;  // the reduction's CTAs and the finish
    const int ng = gather_ctas(w) > lead + 1 ? gather_ctas(w) - lead : 1;
    launch_pdl(k_gather_reduce, lead + ng, 256, 0, s,
               gather_args(w, kRelaxNoise, nullptr, y, m_lat, v_lat, hp, w.step_snap, 0, relax_next),
               reduce_args(w, params, m_par, v_par, nullptr, 1.f, hp, w.step_snap),
               finish_args(w, hp, 1, 1, rd_out, 3, step_dev, 0, 1));
}

void launch_param_reduce(const Work& w, float* params, float* m, float* v, float* grad_out, float out_scale,
                         const Hp& hp, const int64_t* step_dev, cudaStream_t s) {
    launch_pdl(k_param_reduce, kReduceCtas, kReduceThreads, 0, s, reduce_args(w, params, m, v, grad_out, out_scale, hp, step_dev));
}

void launch_finish(const Work& w, const Hp& hp, int have_arm, int have_conv, double* rd_out, int64_t* step_dev,
                   int mark_base, int increment, cudaStream_t s) {
    launch_pdl(k_finish, 1, 256, 0, s, finish_args(w, hp, have_arm, have_conv, rd_out, 3, step_dev, mark_base, increment));
}

void launch_init_state(const InitArgs& a, cudaStream_t s) {
    k_init_state<<<grid_for(a.N + po::total_h, 256, 8), 256, 0, s>>>(a);
}

void launch_mark_base(const Work& w, const int64_t* step_dev, cudaStream_t s) {
    k_mark_base<<<1, 1, 0, s>>>(step_dev, w.base_step);
}

// ---- multi-job launches
void launch_relax_b(const Batch<RelaxArgs>& b, cudaStream_t s) { launch_pdl(k_relax_b, b.total_ctas, 256, 0, s, b); }
void launch_ifce_b(const Batch<IfceArgs>& b, cudaStream_t s) { launch_pdl(k_ifce_cells_b, b.total_ctas, 128, 0, s, b); }
void launch_gather_b(const Batch<GatherArgs>& b, cudaStream_t s) { launch_pdl(k_gather_b, b.total_ctas, 256, 0, s, b); }
void launch_reduce_b(const Batch<ReduceArgs>& b, cudaStream_t s) {
    launch_pdl(k_param_reduce_b, b.total_ctas, kReduceThreads, 0, s, b);
}
void launch_finish_b(const Batch<FinishArgs>& b, cudaStream_t s) { launch_pdl(k_finish_b, b.njobs, 256, 0, s, b); }
void launch_mark_base_b(const Batch<FinishArgs>& b, cudaStream_t s) { k_mark_base_b<<<b.njobs, 32, 0, s>>>(b); }

}  // namespace cc
