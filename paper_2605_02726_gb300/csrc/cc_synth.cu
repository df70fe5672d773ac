// Upsampling cascade of the encoder step (Sec. III-B, Eq. 7), stages 6..2 forward, and the
// adjoint of every stage with the tap gradients (per-CTA partials, reduced in a fixed order).
// Stage 1 forward is fused into the synthesis kernels (cc_syn.cu).
#include "cc_kernels.h"

namespace cc {
namespace {

// ---------------------------------------------------------------------------------------------
// Upsampling stage s (grid s -> grid s-1), forward, stages 6..2.  Output up[m], m = s-1, holds
// the channels of grids m+1..6: channel 0 comes from y~^(m+1), channel j >= 1 from up[m+1][j-1].
// Separable 4x4 polyphase taps with replicate (clamped) indices, cropped to the grid size.
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ void up_fwd_body(const UpFwdArgs& a, int cta, int ncta) {
    const int64_t total = (int64_t)a.nch * a.ht * a.wt;
    const float tp[4] = {__ldg(a.taps), __ldg(a.taps + 1), __ldg(a.taps + 2), __ldg(a.taps + 3)};
    for (int64_t e = cta * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)ncta * blockDim.x) {
        const int j = (int)(e / ((int64_t)a.ht * a.wt));
        const int rem = (int)(e - (int64_t)j * a.ht * a.wt);
        const int y = rem / a.wt, x = rem - y * a.wt;
        const float* S = j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * a.hs * a.ws;
        const int fy = poly_first(y), fx = poly_first(x);
        float wy[4], wx[4];
        poly_w(y, tp, wy);
        poly_w(x, tp, wx);
        float acc = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float* row = S + clampi(fy + p, 0, a.hs - 1) * a.ws;
            float rs = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) rs = fmaf(wx[q], __ldg(row + clampi(fx + q, 0, a.ws - 1)), rs);
            acc = fmaf(wy[p], rs, acc);
        }
        a.dst[e] = acc;
    }
}
__global__ void k_up_fwd(UpFwdArgs a) {
    __shared__ UpFwdArgs sa;
    param_fetch(a, sa);
    up_fwd_body(sa, blockIdx.x, gridDim.x);
}
__global__ void k_up_fwd_b(Batch<UpFwdArgs> b) {
    __shared__ UpFwdArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    up_fwd_body(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

// ---------------------------------------------------------------------------------------------
// Upsampling adjoint, stage s: D = d up[s-1] (7-s channels at grid s-1) -> dS_s at grid s.
// Pass A (columns): T[j][py][ox] = sum_tau h_tau G_tau, G_tau = sum of D[j][oy][ox] over the
//   output rows oy that read input row py through tap tau; dh_tau += G_tau * R[j][py][ox] with R
//   the forward row-pass value.
// Pass B (rows): dS[j][py][px] = sum_tau h_tau G'_tau over T; dh_tau += G'_tau * S[j][py][px].
// ---------------------------------------------------------------------------------------------

// G[tau] for input index p along an axis with n_in inputs and n_out (cropped) outputs, reading
// the output-side values through `get(o)`.
template <typename F>
__device__ __forceinline__ void gather_taps(int p, int n_in, int n_out, F get, float (&G)[4]) {
    G[0] = G[1] = G[2] = G[3] = 0.f;
    if (p >= 2 && p <= n_in - 3) {
        const int o0 = 2 * p - 3;  // outputs 2p-3 .. 2p+4 use taps a b c d d c b a
        const int tt[8] = {0, 1, 2, 3, 3, 2, 1, 0};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int o = o0 + q;
            if (o < n_out) G[tt[q]] += get(o);
        }
    } else {
        const int lo = max(0, 2 * p - 7), hi = min(n_out - 1, 2 * p + 8);
        for (int o = lo; o <= hi; ++o) {
            const int f = poly_first(o);
            const float v = get(o);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float u = clampi(f + q, 0, n_in - 1) == p ? v : 0.f;
                const int t = poly_tap(o, q);
                G[0] += t == 0 ? u : 0.f;
                G[1] += t == 1 ? u : 0.f;
                G[2] += t == 2 ? u : 0.f;
                G[3] += t == 3 ? u : 0.f;
            }
        }
    }
}

// One CTA per (channel j, input row py) pair (grid-stride): pass A builds the row T[j][py][.]
// in shared memory from the <= 8 output rows that read input row py, pass B gathers it along x.
__device__ __forceinline__ void up_adj_body(const UpAdjArgs& a, int cta, int ncta) {
    extern __shared__ float sTrow[];  // wt floats
    const float tp[4] = {__ldg(a.taps), __ldg(a.taps + 1), __ldg(a.taps + 2), __ldg(a.taps + 3)};
    float dh[4] = {0.f, 0.f, 0.f, 0.f};
    const int npairs = a.nch * a.hs;
    for (int pair = cta; pair < npairs; pair += ncta) {
        const int j = pair / a.hs, py = pair - j * a.hs;
        const float* Dj = a.D + (int64_t)j * a.ht * a.wt;
        const float* S = (j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * a.hs * a.ws) + (int64_t)py * a.ws;
        for (int ox = threadIdx.x; ox < a.wt; ox += blockDim.x) {
            float G[4];
            gather_taps(py, a.hs, a.ht, [&](int oy) { return __ldg(Dj + (int64_t)oy * a.wt + ox); }, G);
            sTrow[ox] = tp[0] * G[0] + tp[1] * G[1] + tp[2] * G[2] + tp[3] * G[3];
            const int fx = poly_first(ox);
            float wx[4];
            poly_w(ox, tp, wx);
            float R = 0.f;  // forward row-pass value at (py, ox)
#pragma unroll
            for (int q = 0; q < 4; ++q) R = fmaf(wx[q], __ldg(S + clampi(fx + q, 0, a.ws - 1)), R);
#pragma unroll
            for (int q = 0; q < 4; ++q) dh[q] = fmaf(G[q], R, dh[q]);
        }
        __syncthreads();
        for (int px = threadIdx.x; px < a.ws; px += blockDim.x) {
            float G[4];
            gather_taps(px, a.ws, a.wt, [&](int ox) { return sTrow[ox]; }, G);
            const float d = tp[0] * G[0] + tp[1] * G[1] + tp[2] * G[2] + tp[3] * G[3];
            const float sv = __ldg(S + px);
#pragma unroll
            for (int q = 0; q < 4; ++q) dh[q] = fmaf(G[q], sv, dh[q]);
            const int64_t si = (int64_t)py * a.ws + px;
            if (j == 0)
                a.out0[si] = d;
            else
                a.outup[(int64_t)(j - 1) * a.hs * a.ws + si] = d;
        }
        __syncthreads();
    }
    __shared__ float scratch[4 * (kUpThreads / 32)];
    block_sum<4>(dh, scratch);
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) a.gpart[cta * 4 + q] = dh[q];
}
__global__ void __launch_bounds__(kUpThreads) k_up_adj(UpAdjArgs a) {
    __shared__ UpAdjArgs sa;
    param_fetch(a, sa);
    up_adj_body(sa, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kUpThreads) k_up_adj_b(Batch<UpAdjArgs> b) {
    __shared__ UpAdjArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    up_adj_body(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

int up_grid(int64_t total) {
    int64_t b = (total + kUpThreads - 1) / kUpThreads;
    if (b < 1) b = 1;
    return (int)(b < kUpMaxCta ? b : kUpMaxCta);
}

}  // namespace

int up_adj_grid(int64_t pairs) { return (int)(pairs < kUpMaxCta ? (pairs < 1 ? 1 : pairs) : kUpMaxCta); }

void synth_init_attributes() {
    cudaFuncSetAttribute(k_up_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * (int)sizeof(float));
    cudaFuncSetAttribute(k_up_adj_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * (int)sizeof(float));
    syn_init_attributes();
}

// ---- argument builders and CTA counts
UpFwdArgs up_fwd_args(const Work& w, const float* params, int m) {  // stage s = m + 1 -> up[m]
    const Geom& g = w.g;
    UpFwdArgs a;
    a.src0 = w.yt + g.off[m + 1];
    a.srcup = w.up[m + 1];
    a.dst = w.up[m];
    a.taps = params + po::up + 4 * m;
    a.hs = g.h[m + 1];
    a.ws = g.w[m + 1];
    a.ht = g.h[m];
    a.wt = g.w[m];
    a.nch = kL - 1 - m;
    a.pad_ = 0;
    return a;
}
int up_fwd_ctas(const Work& w, int m) { return up_grid((int64_t)(kL - 1 - m) * w.g.h[m] * w.g.w[m]); }

UpAdjArgs up_adj_args(const Work& w, const float* params, int st) {  // stage st: grid st -> grid st-1
    const Geom& g = w.g;
    UpAdjArgs a;
    a.D = st == 1 ? w.dz : w.dup[st - 1];
    a.src0 = w.yt + g.off[st];
    a.srcup = w.up[st];
    a.out0 = w.dYsyn + g.off[st];
    a.outup = w.dup[st];
    a.gpart = w.gpart_up + (st - 1) * kUpMaxCta * 4;
    a.taps = params + po::up + 4 * (st - 1);
    a.hs = g.h[st];
    a.ws = g.w[st];
    a.ht = g.h[st - 1];
    a.wt = g.w[st - 1];
    a.nch = kL - st;
    a.pad_ = 0;
    return a;
}

// ---- single-job launches
void launch_up_forward(const Work& w, const float* params, cudaStream_t s) {
    for (int m = kL - 2; m >= 1; --m) launch_pdl(k_up_fwd, up_fwd_ctas(w, m), kUpThreads, 0, s, up_fwd_args(w, params, m));
}

void launch_up_adjoint(const Work& w, const float* params, cudaStream_t s) {
    for (int st = 1; st < kL; ++st)
        launch_pdl(k_up_adj, w.n_cta_up[st], kUpThreads, (size_t)w.g.w[st - 1] * sizeof(float), s, up_adj_args(w, params, st));
}

// ---- multi-job launches (max_wt: the widest row any job's stage reads, for the shared row buffer)
void launch_up_fwd_b(const Batch<UpFwdArgs>& b, cudaStream_t s) { launch_pdl(k_up_fwd_b, b.total_ctas, kUpThreads, 0, s, b); }
void launch_up_adj_b(const Batch<UpAdjArgs>& b, int max_wt, cudaStream_t s) {
    launch_pdl(k_up_adj_b, b.total_ctas, kUpThreads, (size_t)max_wt * sizeof(float), s, b);
}

}  // namespace cc
