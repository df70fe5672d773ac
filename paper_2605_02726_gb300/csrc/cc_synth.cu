// Reconstruction side of the encoder step: upsampling cascade (Sec. III-B, Eq. 7), synthesis
// 1x1 MLP with stabilizer (Eq. 8, Eq. 9), two residual 3x3 convolutions, distortion (Eq. 10) and
// the adjoint of each.  Every parameter-gradient sum is reduced per CTA in a fixed order.
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

// Stage-1 upsampling of S_1 = [y~^(1), up[1]] at full-resolution pixel (y, x): z[1..6].
__device__ __forceinline__ void dense_latents(const Geom& g, const float* yt, const float* up1,
                                              const float (&tp)[4], int y, int x, float (&z)[kL]) {
    const int hs = g.h[1], ws = g.w[1];
    z[0] = __ldg(yt + (int64_t)y * g.W + x);
    const int fy = poly_first(y), fx = poly_first(x);
    int ro[4], co[4];
    float wy[4], wx[4];
    poly_w(y, tp, wy);
    poly_w(x, tp, wx);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        ro[p] = clampi(fy + p, 0, hs - 1) * ws;
        co[p] = clampi(fx + p, 0, ws - 1);
    }
    const int64_t n1 = (int64_t)hs * ws;
#pragma unroll
    for (int j = 1; j < kL; ++j) {
        const float* S = j == 1 ? yt + g.off[1] : up1 + (int64_t)(j - 2) * n1;
        float acc = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float rs = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) rs = fmaf(wx[q], __ldg(S + ro[p] + co[q]), rs);
            acc = fmaf(wy[p], rs, acc);
        }
        z[j] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
// Synthesis MLP forward: t = W2 gelu(W1 z + b1) + b2 + Ws z + bs.  One thread per pixel.
// ---------------------------------------------------------------------------------------------

// shared weight layout of the synthesis kernels
constexpr int ss_w1 = 0;      // [40][8] (7 used, 8th = bias b1)
constexpr int ss_w2 = 320;    // [3][40]
constexpr int ss_ws = 440;    // [3][8]  (7 used, 8th = b2 + bs)
constexpr int ss_total = 464;

__device__ __forceinline__ void load_syn_weights(const float* P, float* sW) {
    for (int j = threadIdx.x; j < ss_total; j += blockDim.x) {
        float v;
        if (j < ss_w2) {
            const int o = j >> 3, i = j & 7;
            v = i < 7 ? P[po::syn_w1 + o * 7 + i] : P[po::syn_b1 + o];
        } else if (j < ss_ws) {
            v = P[po::syn_w2 + (j - ss_w2)];
        } else {
            const int o = (j - ss_ws) >> 3, i = (j - ss_ws) & 7;
            v = i < 7 ? P[po::syn_ws + o * 7 + i] : P[po::syn_b2 + o] + P[po::syn_bs + o];
        }
        sW[j] = v;
    }
}

template <int PASS>
__device__ __forceinline__ void syn_fwd_body(const SynArgs& a, int cta, int ncta) {
    __shared__ __align__(16) float sW[ss_total];
    load_syn_weights(a.params, sW);
    const float tp[4] = {a.params[po::up], a.params[po::up + 1], a.params[po::up + 2], a.params[po::up + 3]};
    __syncthreads();
    const Geom& g = a.g;
    for (int64_t p = cta * (int64_t)blockDim.x + threadIdx.x; p < a.HW; p += (int64_t)ncta * blockDim.x) {
        const int y = (int)(p / g.W), x = (int)(p - (int64_t)y * g.W);
        float z[kL];
        dense_latents(g, a.yt, a.up1, tp, y, x, z);
        float t0 = sW[ss_ws + 7], t1 = sW[ss_ws + 15], t2 = sW[ss_ws + 23];
#pragma unroll
        for (int i = 0; i < kL; ++i) {
            t0 = fmaf(sW[ss_ws + i], z[i], t0);
            t1 = fmaf(sW[ss_ws + 8 + i], z[i], t1);
            t2 = fmaf(sW[ss_ws + 16 + i], z[i], t2);
        }
#pragma unroll 4
        for (int o = 0; o < kSH; ++o) {
            const float4 w0 = *reinterpret_cast<const float4*>(sW + ss_w1 + o * 8);
            const float4 w1 = *reinterpret_cast<const float4*>(sW + ss_w1 + o * 8 + 4);
            float acc = w1.w;
            acc = fmaf(w0.x, z[0], acc);
            acc = fmaf(w0.y, z[1], acc);
            acc = fmaf(w0.z, z[2], acc);
            acc = fmaf(w0.w, z[3], acc);
            acc = fmaf(w1.x, z[4], acc);
            acc = fmaf(w1.y, z[5], acc);
            acc = fmaf(w1.z, z[6], acc);
            if (PASS == PASS_FWD_STORE) a.act[(int64_t)o * a.HW + p] = acc;
            const float h = gelu_f(acc);
            t0 = fmaf(sW[ss_w2 + o], h, t0);
            t1 = fmaf(sW[ss_w2 + kSH + o], h, t1);
            t2 = fmaf(sW[ss_w2 + 2 * kSH + o], h, t2);
        }
        a.t[p] = t0;
        a.t[a.HW + p] = t1;
        a.t[2 * a.HW + p] = t2;
    }
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads) k_syn_fwd(SynArgs a) {
    __shared__ SynArgs sa;
    param_fetch(a, sa);
    syn_fwd_body<PASS>(sa, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads) k_syn_fwd_b(Batch<SynArgs> b) {
    __shared__ SynArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    syn_fwd_body<PASS>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

// ---------------------------------------------------------------------------------------------
// Synthesis MLP adjoint, one thread per pixel, rounds of 128 pixels.  dz = W1^T da + Ws^T dt,
// da = (W2^T dt) * gelu'(a).  Parameter gradients as staged outer products:
//   U rows: da 0-39, dt 40-42, zero 43-47;   V rows: z 0-6, one 7, g 8-47.
//   blocks (U0, V0): da x [z, 1] -> (0..32 step 8, 0);  dt x [z, 1] -> (40, 0);  dt x g -> (40, 8..40).
// ---------------------------------------------------------------------------------------------
constexpr int kSLd = kSynThreads + 4;
constexpr int kSBlocks = 11;
constexpr int kSChunks = 11;
constexpr int kSTasks = kSBlocks * kSChunks;  // 121
__constant__ unsigned char c_sblk_u[kSBlocks] = {0, 8, 16, 24, 32, 40, 40, 40, 40, 40, 40};
__constant__ unsigned char c_sblk_v[kSBlocks] = {0, 0, 0, 0, 0, 0, 8, 16, 24, 32, 40};
__constant__ unsigned char c_schunk[kSChunks + 1] = {0, 12, 24, 36, 48, 60, 72, 84, 96, 108, 120, 128};

__device__ int syn_grad_index(int u, int v) {  // index relative to po::syn_w1, or -1
    if (u < 40) {
        if (v < 7) return (po::syn_w1 - po::syn_w1) + u * 7 + v;
        if (v == 7) return (po::syn_b1 - po::syn_w1) + u;
        return -1;
    }
    if (u < 43) {
        const int o = u - 40;
        if (v < 7) return (po::syn_ws - po::syn_w1) + o * 7 + v;
        if (v == 7) return (po::syn_bs - po::syn_w1) + o;  // b2 takes the same sum
        if (v < 48) return (po::syn_w2 - po::syn_w1) + o * kSH + (v - 8);
    }
    return -1;
}

template <int PASS>
__device__ __forceinline__ void syn_bwd_body(const SynArgs& a, int cta, int ncta) {
    extern __shared__ float4 smem4[];
    float* sW = reinterpret_cast<float*>(smem4);
    float* sU = sW + ss_total;
    float* sV = sU + 48 * kSLd;
    float* sAcc = sV + 48 * kSLd;
    load_syn_weights(a.params, sW);
    const float tp[4] = {a.params[po::up], a.params[po::up + 1], a.params[po::up + 2], a.params[po::up + 3]};
    const int tid = threadIdx.x;
    for (int j = tid; j < kSTasks * 64; j += kSynThreads) sAcc[j] = 0.f;
    for (int j = tid; j < kSLd; j += kSynThreads) {
        for (int r = 43; r < 48; ++r) sU[r * kSLd + j] = 0.f;
        sV[7 * kSLd + j] = 1.f;
    }
    __syncthreads();
    const Geom& g = a.g;
    const int64_t HW = a.HW;
    const int64_t n_rounds = (HW + kSynThreads - 1) / kSynThreads;
    for (int64_t rd = cta; rd < n_rounds; rd += ncta) {
        const int64_t p = rd * kSynThreads + tid;
        const bool valid = p < HW;
        const int64_t pc = valid ? p : HW - 1;
        const int y = (int)(pc / g.W), x = (int)(pc - (int64_t)y * g.W);
        float z[kL];
        dense_latents(g, a.yt, a.up1, tp, y, x, z);
        const float m = valid ? 1.f : 0.f;
        const float dt0 = a.dt[pc] * m, dt1 = a.dt[HW + pc] * m, dt2 = a.dt[2 * HW + pc] * m;
        float dz[kL];
#pragma unroll
        for (int i = 0; i < kL; ++i)
            dz[i] = sW[ss_ws + i] * dt0 + sW[ss_ws + 8 + i] * dt1 + sW[ss_ws + 16 + i] * dt2;
#pragma unroll 4
        for (int o = 0; o < kSH; ++o) {
            const float4 w0 = *reinterpret_cast<const float4*>(sW + ss_w1 + o * 8);
            const float4 w1 = *reinterpret_cast<const float4*>(sW + ss_w1 + o * 8 + 4);
            float acc;
            if (PASS == PASS_BWD_LOAD) {
                acc = a.act[(int64_t)o * HW + pc];
            } else {
                acc = w1.w;
                acc = fmaf(w0.x, z[0], acc);
                acc = fmaf(w0.y, z[1], acc);
                acc = fmaf(w0.z, z[2], acc);
                acc = fmaf(w0.w, z[3], acc);
                acc = fmaf(w1.x, z[4], acc);
                acc = fmaf(w1.y, z[5], acc);
                acc = fmaf(w1.z, z[6], acc);
            }
            const float dg = sW[ss_w2 + o] * dt0 + sW[ss_w2 + kSH + o] * dt1 + sW[ss_w2 + 2 * kSH + o] * dt2;
            const float da = dg * gelu_grad_f(acc);
            sU[o * kSLd + tid] = da;
            sV[(8 + o) * kSLd + tid] = gelu_f(acc) * m;
            dz[0] = fmaf(w0.x, da, dz[0]);
            dz[1] = fmaf(w0.y, da, dz[1]);
            dz[2] = fmaf(w0.z, da, dz[2]);
            dz[3] = fmaf(w0.w, da, dz[3]);
            dz[4] = fmaf(w1.x, da, dz[4]);
            dz[5] = fmaf(w1.y, da, dz[5]);
            dz[6] = fmaf(w1.z, da, dz[6]);
        }
        sU[40 * kSLd + tid] = dt0;
        sU[41 * kSLd + tid] = dt1;
        sU[42 * kSLd + tid] = dt2;
#pragma unroll
        for (int i = 0; i < kL; ++i) sV[i * kSLd + tid] = z[i] * m;
        if (valid) {
            a.dYsyn0[p] = dz[0];
#pragma unroll
            for (int j = 1; j < kL; ++j) a.dz[(int64_t)(j - 1) * HW + p] = dz[j];
        }
        __syncthreads();
        if (tid < kSTasks) {
            const int blk = tid / kSChunks, ch = tid - blk * kSChunks;
            const float* U = sU + c_sblk_u[blk] * kSLd;
            const float* V = sV + c_sblk_v[blk] * kSLd;
            float acc[8][8];
            float* A = sAcc + tid * 64;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = A[i * 8 + j];
            for (int l = c_schunk[ch]; l < c_schunk[ch + 1]; l += 4) {
                float4 u[8], v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) u[i] = *reinterpret_cast<const float4*>(U + i * kSLd + l);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = *reinterpret_cast<const float4*>(V + j * kSLd + l);
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float s = acc[i][j];
                        s = fmaf(u[i].x, v[j].x, s);
                        s = fmaf(u[i].y, v[j].y, s);
                        s = fmaf(u[i].z, v[j].z, s);
                        s = fmaf(u[i].w, v[j].w, s);
                        acc[i][j] = s;
                    }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) A[i * 8 + j] = acc[i][j];
        }
        __syncthreads();
    }
    float* gp = a.gpart + (int64_t)cta * po::syn_block;
    for (int e = tid; e < kSBlocks * 64; e += kSynThreads) {
        const int blk = e >> 6, pq = e & 63;
        const int u = c_sblk_u[blk] + (pq >> 3), v = c_sblk_v[blk] + (pq & 7);
        const int idx = syn_grad_index(u, v);
        if (idx < 0) continue;
        float sum = 0.f;
        for (int ch = 0; ch < kSChunks; ++ch) sum += sAcc[(blk * kSChunks + ch) * 64 + pq];
        gp[idx] = sum;
        if (u >= 40 && u < 43 && v == 7) gp[po::syn_b2 - po::syn_w1 + (u - 40)] = sum;
    }
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads, 2) k_syn_bwd(SynArgs a) {
    __shared__ SynArgs sa;
    param_fetch(a, sa);
    syn_bwd_body<PASS>(sa, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads, 2) k_syn_bwd_b(Batch<SynArgs> b) {
    __shared__ SynArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    syn_bwd_body<PASS>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
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

size_t syn_bwd_smem_bytes() { return (size_t)(ss_total + 2 * 48 * kSLd + kSTasks * 64) * sizeof(float); }


void synth_init_attributes() {
    cudaFuncSetAttribute(k_up_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * (int)sizeof(float));
    cudaFuncSetAttribute(k_up_adj_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * (int)sizeof(float));
    const int sm = (int)syn_bwd_smem_bytes();
    cudaFuncSetAttribute(k_syn_bwd<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_syn_bwd<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_syn_bwd_b<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_syn_bwd_b<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
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

SynArgs syn_args(const Work& w, const float* params) {
    SynArgs a;
    a.g = w.g;
    a.HW = w.HW;
    a.yt = w.yt;
    a.up1 = w.up[1];
    a.params = params;
    a.t = w.t;
    a.dt = w.dt;
    a.act = w.act_syn;
    a.dYsyn0 = w.dYsyn;
    a.dz = w.dz;
    a.gpart = w.gpart_syn;
    return a;
}
int syn_fwd_ctas(const Work& w) {
    const int64_t blocks = (w.HW + kSynThreads - 1) / kSynThreads, cap = (int64_t)num_sms() * 16;
    return (int)(blocks < cap ? blocks : cap);
}

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
    for (int m = kL - 2; m >= 1; --m) k_up_fwd<<<up_fwd_ctas(w, m), kUpThreads, 0, s>>>(up_fwd_args(w, params, m));
}

void launch_syn_forward(const Work& w, const float* params, int pass, cudaStream_t s) {
    const SynArgs a = syn_args(w, params);
    if (pass == PASS_FWD_STORE)
        k_syn_fwd<PASS_FWD_STORE><<<syn_fwd_ctas(w), kSynThreads, 0, s>>>(a);
    else
        k_syn_fwd<PASS_FWD><<<syn_fwd_ctas(w), kSynThreads, 0, s>>>(a);
}

void launch_syn_backward(const Work& w, const float* params, int pass, cudaStream_t s) {
    const SynArgs a = syn_args(w, params);
    const size_t sm = syn_bwd_smem_bytes();
    if (pass == PASS_BWD_LOAD)
        k_syn_bwd<PASS_BWD_LOAD><<<w.n_cta_syn, kSynThreads, sm, s>>>(a);
    else
        k_syn_bwd<PASS_FWD_BWD><<<w.n_cta_syn, kSynThreads, sm, s>>>(a);
}

void launch_up_adjoint(const Work& w, const float* params, cudaStream_t s) {
    for (int st = 1; st < kL; ++st)
        k_up_adj<<<w.n_cta_up[st], kUpThreads, (size_t)w.g.w[st - 1] * sizeof(float), s>>>(up_adj_args(w, params, st));
}

// ---- multi-job launches (max_wt: the widest row any job's stage reads, for the shared row buffer)
void launch_up_fwd_b(const Batch<UpFwdArgs>& b, cudaStream_t s) { k_up_fwd_b<<<b.total_ctas, kUpThreads, 0, s>>>(b); }
void launch_syn_fwd_b(const Batch<SynArgs>& b, cudaStream_t s) {
    k_syn_fwd_b<PASS_FWD><<<b.total_ctas, kSynThreads, 0, s>>>(b);
}
void launch_syn_bwd_b(const Batch<SynArgs>& b, cudaStream_t s) {
    k_syn_bwd_b<PASS_FWD_BWD><<<b.total_ctas, kSynThreads, syn_bwd_smem_bytes(), s>>>(b);
}
void launch_up_adj_b(const Batch<UpAdjArgs>& b, int max_wt, cudaStream_t s) {
    k_up_adj_b<<<b.total_ctas, kUpThreads, (size_t)max_wt * sizeof(float), s>>>(b);
}

}  // namespace cc
