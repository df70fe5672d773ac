// Upsampling cascade of the encoder step (Sec. III-B, Eq. 7): the forward stages as per-stage
// kernels (stages 3 and 2 in the encoder iteration, whose entropy-model launch computes stages
// 6..4; every stage when decoding), and the adjoint of every stage with the tap gradients
// (per-CTA partials, reduced in a fixed order).  Stage 1 forward is fused into the synthesis
// kernels (cc_syn.cu).
#include "cc_kernels.h"
#include "cc_upfwd.cuh"

namespace cc {
namespace {

__global__ void k_up_fwd(const __grid_constant__ UpFwdArgs a) {
    pdl_enter();
    up_fwd_body(a, blockIdx.x, gridDim.x);
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
//
// Output o reads inputs poly_first(o) .. poly_first(o)+3 (clamped), so input p is read only by
// outputs 2p-3 .. 2p+4.  A CTA owns a tile of ty input rows by kUpTX input columns of one
// channel and stages in shared memory the D block those outputs span (zero outside the grid),
// the T block pass B needs and the clamped S columns of the row pass: every D element is read
// from L2 about (2ty+6)/(2ty) times instead of four times.
// ---------------------------------------------------------------------------------------------
constexpr int kUpDC = 2 * kUpTX + 6;  // D and T columns: outputs 2*px0-3 .. 2*px0+2*kUpTX+2
constexpr int kUpSC = kUpTX + 4;      // S columns px0-2 .. px0+kUpTX+1 (clamped)
constexpr int kUpSmemFloats = (2 * kUpTYMax + 6) * kUpDC + kUpTYMax * kUpDC + kUpTYMax * kUpSC;

// G[tau] for input p (of n_in) from the eight outputs 2p-3+q, q = 0..7, whose values are v(q)
// (zero for outputs outside the grid): output 2p-3+q reads p through tap a b c d d c b a.  The
// replicate clamp folds the virtual inputs beyond a border onto it, so input 0 also collects the
// outputs of virtual inputs -1 and -2 (window positions q-2, q-4) and input n_in-1 those of n_in
// and n_in+1 (q+2, q+4); every other input is read only through its own window.
template <typename F>
__device__ __forceinline__ void taps_of_input(int p, int n_in, F v, float (&G)[4]) {
    float u[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) u[q] = v(q);
    if (p == 0 || p == n_in - 1) {
        float w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float x = u[q];
            if (p == 0) {
                if (q >= 2) x += u[q - 2];
                if (q >= 4) x += u[q - 4];
            }
            if (p == n_in - 1) {
                if (q + 2 <= 7) x += u[q + 2];
                if (q + 4 <= 7) x += u[q + 4];
            }
            w[q] = x;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = w[q];
    }
    G[0] = u[0] + u[7];
    G[1] = u[1] + u[6];
    G[2] = u[2] + u[5];
    G[3] = u[3] + u[4];
}

// Pass A of a tile of TY input rows: thread t < 2 kUpDC takes column c = t mod kUpDC of the D
// block and half of the tile's rows (R = TY/2, group t / kUpDC), sliding a register window of the
// 2R + 6 output rows those inputs read down the column: each D value is loaded from shared memory
// once per thread instead of once per input row that reads it.
template <int TY>
__device__ __forceinline__ void up_adj_pass_a(const UpAdjArgs& a, const float* sD, float* sT, const float* sS,
                                              int py0, int px0, int c0, const float (&tp)[4], float (&dh)[4]) {
    constexpr int R = TY / 2;
    const int t = threadIdx.x;
    if (t >= 2 * kUpDC) return;
    const int grp = t >= kUpDC ? 1 : 0, c = t - grp * kUpDC;
    const int ox = c0 + c;
    const bool col_ok = ox >= 0 && ox < a.wt;
    const bool own = ox >= 2 * px0 && ox < 2 * px0 + 2 * kUpTX;  // this tile owns (py, ox) for dh
    float win[2 * R + 6];
#pragma unroll
    for (int k = 0; k < 2 * R + 6; ++k) win[k] = sD[(2 * grp * R + k) * kUpDC + c];
    float wx[4];
    poly_w(ox, tp, wx);
    const int so = poly_first(ox) - (px0 - 2);  // S column of the row pass (owned ox only)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int tr = grp * R + r, py = py0 + tr;
        float T = 0.f;
        if (col_ok && py < a.hs) {
            float G[4];
            taps_of_input(py, a.hs, [&](int q) { return win[2 * r + q]; }, G);
            T = tp[0] * G[0] + tp[1] * G[1] + tp[2] * G[2] + tp[3] * G[3];
            if (own) {
                const float* srow = sS + tr * kUpSC + so;
                float Rv = 0.f;  // forward row-pass value at (py, ox)
#pragma unroll
                for (int q = 0; q < 4; ++q) Rv = fmaf(wx[q], srow[q], Rv);
#pragma unroll
                for (int q = 0; q < 4; ++q) dh[q] = fmaf(G[q], Rv, dh[q]);
            }
        }
        sT[tr * kUpDC + c] = T;
    }
}

__device__ __forceinline__ void up_adj_body(const UpAdjArgs& a, int cta, int ncta) {
    discard_dead(a.dead, cta, ncta);
    extern __shared__ float smem_up[];
    float* sD = smem_up;                                // [2ty+6][kUpDC]
    float* sT = sD + (2 * kUpTYMax + 6) * kUpDC;        // [ty][kUpDC]
    float* sS = sT + kUpTYMax * kUpDC;                  // [ty][kUpSC]
    const float tp[4] = {__ldg(a.taps), __ldg(a.taps + 1), __ldg(a.taps + 2), __ldg(a.taps + 3)};
    float dh[4] = {0.f, 0.f, 0.f, 0.f};
    const int ty = a.ty;
    const int nty = (a.hs + ty - 1) / ty, ntx = (a.ws + kUpTX - 1) / kUpTX;
    const int tiles = a.nch * nty * ntx;
    for (int tile = cta; tile < tiles; tile += ncta) {
        const int j = tile / (nty * ntx);
        const int rem = tile - j * nty * ntx;
        const int py0 = (rem / ntx) * ty, px0 = (rem - (rem / ntx) * ntx) * kUpTX;
        const int r0 = 2 * py0 - 3, c0 = 2 * px0 - 3;
        const float* Dj = a.D + (int64_t)j * a.ht * a.wt;
        const float* S = j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * a.hs * a.ws;
        // the tiles by asynchronous global -> shared copies (all of a thread's copies in flight at
        // once); cells outside the grid are stored as zeros
        const int nd = (2 * ty + 6) * kUpDC;
        for (int e = threadIdx.x; e < nd; e += blockDim.x) {
            const int r = e / kUpDC, c = e - r * kUpDC;
            const int gr = r0 + r, gc = c0 + c;
            if (gr >= 0 && gr < a.ht && gc >= 0 && gc < a.wt)
                cp_async4(sD + e, Dj + (int64_t)gr * a.wt + gc);
            else
                sD[e] = 0.f;
        }
        for (int e = threadIdx.x; e < ty * kUpSC; e += blockDim.x) {
            const int r = e / kUpSC, c = e - r * kUpSC;
            const int py = py0 + r;
            if (py < a.hs)
                cp_async4(sS + e, S + (int64_t)py * a.ws + clampi(px0 - 2 + c, 0, a.ws - 1));
            else
                sS[e] = 0.f;
        }
        cp_async_wait_all();
        __syncthreads();
        // pass A: T over output columns c0 .. c0+kUpDC-1 of the tile's input rows
        switch (ty) {
            case 16: up_adj_pass_a<16>(a, sD, sT, sS, py0, px0, c0, tp, dh); break;
            case 8: up_adj_pass_a<8>(a, sD, sT, sS, py0, px0, c0, tp, dh); break;
            case 4: up_adj_pass_a<4>(a, sD, sT, sS, py0, px0, c0, tp, dh); break;
            default: up_adj_pass_a<2>(a, sD, sT, sS, py0, px0, c0, tp, dh); break;
        }
        __syncthreads();
        // pass B: the tile's inputs from T
        for (int e = threadIdx.x; e < ty * kUpTX; e += blockDim.x) {
            const int r = e / kUpTX, c = e - r * kUpTX;
            const int py = py0 + r, px = px0 + c;
            if (py < a.hs && px < a.ws) {
                float G[4];
                const float* row = sT + r * kUpDC + 2 * c;
                taps_of_input(px, a.ws, [&](int q) { return row[q]; }, G);
                const float d = tp[0] * G[0] + tp[1] * G[1] + tp[2] * G[2] + tp[3] * G[3];
                const float sv = sS[r * kUpSC + c + 2];
#pragma unroll
                for (int q = 0; q < 4; ++q) dh[q] = fmaf(G[q], sv, dh[q]);
                const int64_t si = (int64_t)py * a.ws + px;
                if (j == 0)
                    a.out0[si] = d;
                else
                    a.outup[(int64_t)(j - 1) * a.hs * a.ws + si] = d;
            }
        }
        __syncthreads();
    }
    __shared__ float scratch[4 * (kUpAdjThreads / 32)];
    block_sum<4>(dh, scratch);
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) a.gpart[cta * 4 + q] = dh[q];
}
__global__ void __launch_bounds__(kUpAdjThreads, 4) k_up_adj(const __grid_constant__ UpAdjArgs a) {
    pdl_enter();
    up_adj_body(a, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kUpAdjThreads, 4) k_up_adj_b(Batch<UpAdjArgs> b) {
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

// Tile height of stage s's adjoint: the tallest of 16, 8, 4, 2 rows that still gives two CTAs per
// SM, so the fine stages read the fewest halo rows and the coarse ones keep enough CTAs.
int up_adj_ty(int nch, int hs, int ws) {
    const int64_t want = 2 * (int64_t)num_sms();
    const int64_t ntx = (ws + kUpTX - 1) / kUpTX;
    for (int ty = kUpTYMax; ty > 2; ty /= 2)
        if ((int64_t)nch * ((hs + ty - 1) / ty) * ntx >= want) return ty;
    return 2;
}
int up_adj_ctas(int nch, int hs, int ws) {
    const int ty = up_adj_ty(nch, hs, ws);
    const int64_t tiles = (int64_t)nch * ((hs + ty - 1) / ty) * ((ws + kUpTX - 1) / kUpTX);
    return (int)(tiles < kUpMaxCta ? (tiles < 1 ? 1 : tiles) : kUpMaxCta);
}

void synth_init_attributes() {
    cudaFuncSetAttribute(k_up_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpSmemFloats * (int)sizeof(float));
    cudaFuncSetAttribute(k_up_adj_b, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpSmemFloats * (int)sizeof(float));
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
    a.ty = up_adj_ty(a.nch, a.hs, a.ws);
    a.dead = DeadRanges{};
    if (w.discard_dead && st == 1 && w.zden) {  // read last by the synthesis adjoint
        a.dead.p[0] = w.zden;
        a.dead.n[0] = 6 * w.HW;
        a.dead.p[1] = w.dt;
        a.dead.n[1] = 3 * w.HW;
    } else if (w.discard_dead && st == 2) {  // read last by stage 1
        a.dead.p[0] = w.dz;
        a.dead.n[0] = 6 * w.HW;
    }
    return a;
}

// ---- single-job launches
void launch_up_forward(const Work& w, const float* params, int m_hi, cudaStream_t s) {
    for (int m = m_hi; m >= 1; --m) launch_pdl(k_up_fwd, up_fwd_ctas(w, m), kUpThreads, 0, s, up_fwd_args(w, params, m));
}

void launch_up_adjoint(const Work& w, const float* params, cudaStream_t s) {
    for (int st = 1; st < kL; ++st)
        launch_pdl(k_up_adj, w.n_cta_up[st], kUpAdjThreads, kUpSmemFloats * sizeof(float), s, up_adj_args(w, params, st));
}

// ---- multi-job launches
void launch_up_fwd_b(const Batch<UpFwdArgs>& b, cudaStream_t s) { launch_pdl(k_up_fwd_b, b.total_ctas, kUpThreads, 0, s, b); }
void launch_up_adj_b(const Batch<UpAdjArgs>& b, cudaStream_t s) {
    launch_pdl(k_up_adj_b, b.total_ctas, kUpAdjThreads, kUpSmemFloats * sizeof(float), s, b);
}

}  // namespace cc
