// Synthesis of the encoder step: the last upsampling stage (Sec. III-B, Eq. 7) fused with the 1x1
// MLP 7 -> 40 (GELU) -> 3 and its linear stabilizer 7 -> 3 (Eq. 8, Eq. 9), forward and adjoint.
//
// The forward runs one thread per pixel and keeps the 6 upsampled dense-latent channels for the
// adjoint.  The adjoint runs on tensor cores, one warp per unit of 16 consecutive pixels (the M
// dimension of mma.sync.m16n8k8): lane (g, t) owns pixels g and g + 8 of the unit and loads the
// dense-latent channels t and t + 4 of both (channel 7 is the constant 1 that carries the
// first-layer bias), i.e. exactly its A fragment.  Products run as TF32 MMAs
// with the hi/lo split of cc_mma.cuh (FP32-level accuracy), accumulator fragments feed the next
// product through the K permutation, weight fragments are pre-split per lane in shared memory.
// Parameter gradients are MMAs over the pixel dimension from a warp-private transposed tile,
// accumulated in registers for the whole kernel and added across the 4 warps in a fixed order:
// one partial gradient per CTA.
#include "cc_kernels.h"
#include "cc_mma.cuh"

namespace cc {
namespace {

constexpr int kWarps = kSynThreads / 32;  // 4
constexpr int kSld = 20;                  // staging stride (16 pixels + 4)
// staging rows: U = [dA 0..39, dT 40..42, zero 43..47], V = [Z 48..55, G 56..95]
constexpr int U_DA = 0, U_DT = 40, V_Z = 48, V_G = 56, S_ROWS = 96;
constexpr int kStage = S_ROWS * kSld;
// B-fragment table
constexpr int FR_W1 = 0, FR_W2 = 5, FR_WS = 10, FR_BW1 = 11, FR_N = 16;

__device__ float bfrag_syn(const float* P, int f, int g, int t, int which) {
    if (f < FR_W2) {  // layer 1: B[k = channel][n = unit] = W1aug[unit][channel], channel 7 = bias
        const int unit = f * 8 + g, ch = t + 4 * which;
        return ch < 7 ? P[po::syn_w1 + unit * 7 + ch] : P[po::syn_b1 + unit];
    }
    if (f < FR_WS) {  // layer 2, K permuted: B[k][n = out] = W2[out][unit(k)]
        const int kc = f - FR_W2, u = kc * 8 + 2 * t + which;
        return g < 3 ? P[po::syn_w2 + g * kSH + u] : 0.f;
    }
    if (f < FR_BW1) {  // stabilizer: B[k = channel][n = out], channel 7 carries b2 + bs
        const int ch = t + 4 * which;
        if (g >= 3) return 0.f;
        return ch < 7 ? P[po::syn_ws + g * 7 + ch] : P[po::syn_b2 + g] + P[po::syn_bs + g];
    }
    {  // adjoint of layer 1: B[k = unit (permuted)][n = channel] = W1[unit][channel]
        const int kc = f - FR_BW1, o = kc * 8 + 2 * t + which;
        return g < 7 ? P[po::syn_w1 + o * 7 + g] : 0.f;
    }
}

__device__ __forceinline__ void build_frags(const float* P, float4* sFr) {
    for (int j = threadIdx.x; j < FR_N * 32; j += blockDim.x) {
        const int f = j >> 5, l = j & 31;
        uint32_t h0, l0, h1, l1;
        split2(bfrag_syn(P, f, l >> 2, l & 3, 0), h0, l0);
        split2(bfrag_syn(P, f, l >> 2, l & 3, 1), h1, l1);
        sFr[j] = make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(l0), __uint_as_float(l1));
    }
}

// Stage-1 sampling geometry of one full-resolution pixel: 4 rows and 4 columns of grid 1 and
// their tap weights (polyphase, replicate padding).
struct Samp {
    int ro[4], co[4];
    float wy[4], wx[4];
    int64_t p;
};

__device__ __forceinline__ Samp sample_at(const Geom& g, float rcpW, const float (&tp)[4], int64_t p) {
    Samp s;
    s.p = p;
    const int pi = (int)p;
    int y = __float2int_rz(__int2float_rn(pi) * rcpW);
    y -= (y * g.W > pi) ? 1 : 0;
    y += ((y + 1) * g.W <= pi) ? 1 : 0;
    const int x = pi - y * g.W;
    const int hs = g.h[1], ws = g.w[1];
    const int fy = poly_first(y), fx = poly_first(x);
    poly_w(y, tp, s.wy);
    poly_w(x, tp, s.wx);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        s.ro[q] = clampi(fy + q, 0, hs - 1) * ws;
        s.co[q] = clampi(fx + q, 0, ws - 1);
    }
    return s;
}

// Dense-latent channel j (0..7) at a sampled pixel: 0 = y~ of grid 0, 1..6 = stage-1 upsampling of
// S_1 = [y~^(1), up[1]], 7 = the constant 1.
__device__ __forceinline__ float dense_ch(const SynArgs& a, const Samp& s, int j, int64_t n1) {
    if (j == 0) return __ldg(a.yt + s.p);
    if (j >= 7) return 1.f;
    const float* S = j == 1 ? a.yt + a.g.off[1] : a.up1 + (int64_t)(j - 2) * n1;
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float rs = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) rs = fmaf(s.wx[q], __ldg(S + s.ro[r] + s.co[q]), rs);
        acc = fmaf(s.wy[r], rs, acc);
    }
    return acc;
}

// ---------------------------------------------------------------------------------------------
// Forward: t = W2 gelu(W1 z + b1) + b2 + Ws z + bs.  One thread per pixel (SIMT: the forward is
// short and latency-bound, and a thread per pixel keeps the register count, hence the number of
// resident warps, where the tensor-core form cannot).
// ---------------------------------------------------------------------------------------------
// Hidden-unit weights, two layouts of the same 480 floats.  PACKED: per pair of units (o, o + 1),
// 24 floats interleaved so that every 16-byte load gives two (unit o, unit o + 1) register pairs for
// the packed two-wide FMAs: W1[o][i], W1[o+1][i] for i = 0..6, b1[o], b1[o+1], then W2[0..2][o],
// W2[0..2][o+1], 0, 0 (six 16-byte loads).  Otherwise per unit o, 12 floats: W1[o][0..6], b1[o],
// W2[0..2][o], 0 (three 16-byte loads).
constexpr int ss_unit = 0;   // [20][24] or [40][12]
constexpr int ss_ws = 480;   // [3][8]  (7 used, 8th = b2 + bs)
constexpr int ss_total = 504;
static_assert(kSH % 2 == 0, "hidden units in pairs");

template <bool PACKED>
__device__ __forceinline__ void load_syn_weights(const float* P, float* sW) {
    for (int j = threadIdx.x; j < ss_total; j += blockDim.x) {
        float v;
        if (j < ss_ws && !PACKED) {
            const int o = j / 12, i = j - o * 12;
            v = i < 7 ? P[po::syn_w1 + o * 7 + i] : i == 7 ? P[po::syn_b1 + o] : i < 11 ? P[po::syn_w2 + (i - 8) * kSH + o] : 0.f;
        } else if (j < ss_ws) {
            const int pr = j / 24, i = j - pr * 24;
            const int o = 2 * pr + (i < 16 ? (i & 1) : (i - 16) / 3);
            if (i < 14) v = P[po::syn_w1 + o * 7 + (i >> 1)];
            else if (i < 16) v = P[po::syn_b1 + o];
            else if (i < 22) v = P[po::syn_w2 + ((i - 16) % 3) * kSH + o];
            else v = 0.f;
        } else {
            const int o = (j - ss_ws) >> 3, i = (j - ss_ws) & 7;
            v = i < 7 ? P[po::syn_ws + o * 7 + i] : P[po::syn_b2 + o] + P[po::syn_bs + o];
        }
        sW[j] = v;
    }
}

// PACKED: the hidden units' first layer and GELU as packed two-wide FP32 operations (the
// single-job kernel, whose arguments stay in the parameter space); otherwise the same operations
// one unit at a time (the multi-job kernel, whose arguments in shared memory leave too few
// registers for the pairs).  Both give the same bits.
template <int PASS, bool PACKED>
__device__ __forceinline__ void syn_fwd_body(const SynArgs& a, int cta, int ncta) {
    __shared__ __align__(16) float sW[ss_total];
    __shared__ float sRaw[po::syn_block];  // the synthesis parameters, staged in one round trip
    load_syn_weights<PACKED>(stage_params(a.params, po::syn_w1, po::syn_block, sRaw), sW);
    const float tp[4] = {a.params[po::up], a.params[po::up + 1], a.params[po::up + 2], a.params[po::up + 3]};
    __syncthreads();
    const float rcpW = 1.f / (float)a.g.W;
    const int64_t n1 = (int64_t)a.g.h[1] * a.g.w[1];
    for (int64_t p = cta * (int64_t)blockDim.x + threadIdx.x; p < a.HW; p += (int64_t)ncta * blockDim.x) {
        const Samp sp = sample_at(a.g, rcpW, tp, p);
        float z[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) z[j] = dense_ch(a, sp, j, n1);
        if (a.zden)  // kept for the adjoint
#pragma unroll
            for (int j = 1; j < 7; ++j) a.zden[(int64_t)(j - 1) * a.HW + p] = z[j];
        float t0 = sW[ss_ws + 7], t1 = sW[ss_ws + 15], t2 = sW[ss_ws + 23];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            t0 = fmaf(sW[ss_ws + i], z[i], t0);
            t1 = fmaf(sW[ss_ws + 8 + i], z[i], t1);
            t2 = fmaf(sW[ss_ws + 16 + i], z[i], t2);
        }
        // the hidden units: packed in pairs (each unit gets exactly the scalar operations, in the same
        // order) or one at a time; the output layer scalar in unit order either way
        if constexpr (PACKED) {
            float2 zz[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) zz[i] = make_float2(z[i], z[i]);
#pragma unroll 1
            for (int pr = 0; pr < kSH / 2; ++pr) {
                const float4* q = reinterpret_cast<const float4*>(sW + ss_unit + pr * 24);
                const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3], q4 = q[4], q5 = q[5];
                float2 acc = make_float2(q3.z, q3.w);
                acc = __ffma2_rn(make_float2(q0.x, q0.y), zz[0], acc);
                acc = __ffma2_rn(make_float2(q0.z, q0.w), zz[1], acc);
                acc = __ffma2_rn(make_float2(q1.x, q1.y), zz[2], acc);
                acc = __ffma2_rn(make_float2(q1.z, q1.w), zz[3], acc);
                acc = __ffma2_rn(make_float2(q2.x, q2.y), zz[4], acc);
                acc = __ffma2_rn(make_float2(q2.z, q2.w), zz[5], acc);
                acc = __ffma2_rn(make_float2(q3.x, q3.y), zz[6], acc);
                if (PASS == PASS_FWD_STORE) {
                    a.act[(int64_t)(2 * pr) * a.HW + p] = acc.x;
                    a.act[(int64_t)(2 * pr + 1) * a.HW + p] = acc.y;
                }
                const float2 h = gelu2_f(acc);
                t0 = fmaf(q4.x, h.x, t0);
                t1 = fmaf(q4.y, h.x, t1);
                t2 = fmaf(q4.z, h.x, t2);
                t0 = fmaf(q4.w, h.y, t0);
                t1 = fmaf(q5.x, h.y, t1);
                t2 = fmaf(q5.y, h.y, t2);
            }
        } else {
#pragma unroll 4
            for (int o = 0; o < kSH; ++o) {
                const float4 w0 = *reinterpret_cast<const float4*>(sW + ss_unit + o * 12);
                const float4 w1 = *reinterpret_cast<const float4*>(sW + ss_unit + o * 12 + 4);
                const float4 w2 = *reinterpret_cast<const float4*>(sW + ss_unit + o * 12 + 8);
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
                t0 = fmaf(w2.x, h, t0);
                t1 = fmaf(w2.y, h, t1);
                t2 = fmaf(w2.z, h, t2);
            }
        }
        a.t[p] = t0;
        a.t[a.HW + p] = t1;
        a.t[2 * a.HW + p] = t2;
    }
}

// ---------------------------------------------------------------------------------------------
// Adjoint: dG = W2^T dt, dA = dG * gelu'(a), dz = W1^T dA + Ws^T dt; parameter gradients
//   W1, b1 += dA [z, 1]^T;  Ws, bs (= b2) += dt [z, 1]^T;  W2 += dt G^T.
// ---------------------------------------------------------------------------------------------
__device__ int syn_wgrad_index(int T, int row, int col, int* second) {  // relative to po::syn_w1
    *second = -1;
    const int rw1 = po::syn_w1, rb1 = po::syn_b1 - rw1, rw2 = po::syn_w2 - rw1, rb2 = po::syn_b2 - rw1,
              rws = po::syn_ws - rw1, rbs = po::syn_bs - rw1;
    if (T <= 2) {
        if (T < 2 || row < 8) {
            const int o = T * 16 + row;
            return col < 7 ? o * 7 + col : rb1 + o;
        }
        if (row >= 11) return -1;
        const int c = row - 8;
        if (col < 7) return rws + c * 7 + col;
        *second = rb2 + c;
        return rbs + c;
    }
    if (row < 8 || row >= 11) return -1;
    return rw2 + (row - 8) * kSH + (T - 3) * 8 + col;
}

template <int PASS>
__device__ __forceinline__ void syn_bwd_body(const SynArgs& a, int cta, int ncta) {
    discard_dead(a.dead, cta, ncta);
    extern __shared__ float4 smem4[];
    float4* sFr = smem4;
    float* sStage = reinterpret_cast<float*>(smem4 + FR_N * 32);
    // the synthesis parameters staged in one round trip (through the staging area, free until the
    // first unit), then the fragment table and W2 / Ws for the SIMT parts, read as float2 per lane
    const float* P = stage_params(a.params, po::syn_w1, po::syn_block, sStage);
    build_frags(P, sFr);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, gq = lane >> 2, tq = lane & 3;
    __shared__ __align__(16) float sW2[kC * kSH + kC * 8];  // W2 [3][40], Ws [3][8] (column 7 zero)
    for (int j = tid; j < kC * kSH + kC * 8; j += blockDim.x) {
        float v;
        if (j < kC * kSH) {
            v = P[po::syn_w2 + j];
        } else {
            const int c = (j - kC * kSH) >> 3, ch = (j - kC * kSH) & 7;
            v = ch < 7 ? P[po::syn_ws + c * 7 + ch] : 0.f;
        }
        sW2[j] = v;
    }
    __syncthreads();
    float* st = sStage + wid * kStage;
    for (int j = lane; j < kSld; j += 32)
        for (int r = U_DT + 3; r < V_Z; ++r) st[r * kSld + j] = 0.f;
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int T = 0; T < 8; ++T)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[T][q] = 0.f;

    const int64_t HW = a.HW;
    const int64_t n_units = (HW + 15) / 16;
    for (int64_t u = (int64_t)cta * kWarps + wid; u < n_units; u += (int64_t)ncta * kWarps) {
        const int64_t pA = u * 16 + gq, pB = pA + 8;
        const bool vA = pA < HW, vB = pB < HW;
        const int64_t qA = vA ? pA : HW - 1, qB = vB ? pB : HW - 1;
        // dense-latent channels t and t + 4 (0: y~ of grid 0, 1..6: kept by the forward, 7: one)
        auto zval = [&](int j, int64_t q) {
            return j == 0 ? __ldg(a.yt + q) : (j >= 7 ? 1.f : __ldg(a.zden + (int64_t)(j - 1) * HW + q));
        };
        const float zA0 = zval(tq, qA), zB0 = zval(tq, qB);
        const float zA1 = zval(tq + 4, qA), zB1 = zval(tq + 4, qB);
        const AFrag Z = make_a(zA0, zB0, zA1, zB1);
        const float mA = vA ? 1.f : 0.f, mB = vB ? 1.f : 0.f;
        float dtA[3], dtB[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dtA[c] = a.dt[(int64_t)c * HW + qA] * mA;
            dtB[c] = a.dt[(int64_t)c * HW + qB] * mB;
        }
        float d1[5][4];
        if (PASS == PASS_BWD_LOAD) {
#pragma unroll
            for (int nt = 0; nt < 5; ++nt)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int uu = nt * 8 + 2 * tq + cc;
                    d1[nt][cc] = a.act[(int64_t)uu * HW + qA];
                    d1[nt][2 + cc] = a.act[(int64_t)uu * HW + qB];
                }
        } else {
#pragma unroll
            for (int nt = 0; nt < 5; ++nt) {
                float e[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int q = 0; q < 4; ++q) d1[nt][q] = 0.f;
                mma3(d1[nt], e, Z, sFr[(FR_W1 + nt) * 32 + lane]);
                add4(d1[nt], e);
            }
        }
        // dA = (W2^T dt) * gelu'(a); stage dA and G = gelu(a)
        float dz[4], ez[4] = {0.f, 0.f, 0.f, 0.f};
        {
            float2 ws[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) ws[c] = *reinterpret_cast<const float2*>(sW2 + kC * kSH + c * 8 + 2 * tq);
            dz[0] = dtA[0] * ws[0].x + dtA[1] * ws[1].x + dtA[2] * ws[2].x;
            dz[1] = dtA[0] * ws[0].y + dtA[1] * ws[1].y + dtA[2] * ws[2].y;
            dz[2] = dtB[0] * ws[0].x + dtB[1] * ws[1].x + dtB[2] * ws[2].x;
            dz[3] = dtB[0] * ws[0].y + dtB[1] * ws[1].y + dtB[2] * ws[2].y;
        }
#pragma unroll
        for (int nt = 0; nt < 5; ++nt) {
            float da[4];
            float2 w2[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) w2[c] = *reinterpret_cast<const float2*>(sW2 + c * kSH + nt * 8 + 2 * tq);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int cc = q & 1;
                const float* dtp = q < 2 ? dtA : dtB;
                const float dg = cc == 0 ? dtp[0] * w2[0].x + dtp[1] * w2[1].x + dtp[2] * w2[2].x
                                         : dtp[0] * w2[0].y + dtp[1] * w2[1].y + dtp[2] * w2[2].y;
                float gv, gd;
                gelu_fg(d1[nt][q], gv, gd);
                da[q] = dg * gd;
                const int uu = nt * 8 + 2 * tq + cc;
                const int col = q < 2 ? gq : gq + 8;
                st[(U_DA + uu) * kSld + col] = da[q];
                st[(V_G + uu) * kSld + col] = gv;
            }
            mma3(dz, ez, chain(da), sFr[(FR_BW1 + nt) * 32 + lane]);
        }
        add4(dz, ez);
        // dz: channels 2t, 2t+1 of pixels A (dz[0..1]) and B (dz[2..3]); channel 7 is the bias slot
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int ch = 2 * tq + cc;
            if (ch == 0) {
                if (vA) a.dYsyn0[pA] = dz[cc];
                if (vB) a.dYsyn0[pB] = dz[2 + cc];
            } else if (ch < 7) {
                if (vA) a.dz[(int64_t)(ch - 1) * HW + pA] = dz[cc];
                if (vB) a.dz[(int64_t)(ch - 1) * HW + pB] = dz[2 + cc];
            }
        }
        // stage dt (rows 40..42) and z (rows 48..55)
        if (tq < 3) {
            st[(U_DT + tq) * kSld + gq] = tq == 0 ? dtA[0] : (tq == 1 ? dtA[1] : dtA[2]);
            st[(U_DT + tq) * kSld + gq + 8] = tq == 0 ? dtB[0] : (tq == 1 ? dtB[1] : dtB[2]);
        }
        st[(V_Z + tq) * kSld + gq] = zA0;
        st[(V_Z + tq) * kSld + gq + 8] = zB0;
        st[(V_Z + tq + 4) * kSld + gq] = zA1;
        st[(V_Z + tq + 4) * kSld + gq + 8] = zB1;
        __syncwarp();
        // fragments by ldmatrix (rows of 16 bytes at an 80-byte stride: 16-byte aligned, and eight
        // rows fall on disjoint banks): an A fragment is the matrices (rows 0-7, k 0-3), (8-15, 0-3),
        // (0-7, 4-7), (8-15, 4-7); a pair of B fragments (8 rows each) is (first, k 0-3),
        // (first, 4-7), (second, 0-3), (second, 4-7)
        const int mi = lane >> 3, ri = lane & 7;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k0 = ks * 8;
            const float* arow = st + (ri + (mi & 1) * 8) * kSld + k0 + (mi >> 1) * 4;
            const float* brow = st + ri * kSld + k0 + (mi & 1) * 4;
            auto afrag = [&](int row0) {
                uint32_t r[4];
                ldsm_x4(r, arow + row0 * kSld);
                AFrag f;
#pragma unroll
                for (int q = 0; q < 4; ++q) split_u(r[q], f.h[q], f.l[q]);
                return f;
            };
            auto bpair = [&](int row0a, int row0b, AFrag& fa, AFrag& fb) {
                uint32_t r[4];
                ldsm_x4(r, brow + ((mi >> 1) ? row0b : row0a) * kSld);
                split_u(r[0], fa.h[0], fa.l[0]);
                split_u(r[1], fa.h[1], fa.l[1]);
                split_u(r[2], fb.h[0], fb.l[0]);
                split_u(r[3], fb.h[1], fb.l[1]);
            };
            const AFrag U0 = afrag(0), U1 = afrag(16), U2 = afrag(32);
            AFrag VZ, G[5];
            bpair(V_Z, V_G, VZ, G[0]);
            bpair(V_G + 8, V_G + 16, G[1], G[2]);
            bpair(V_G + 24, V_G + 32, G[3], G[4]);
            mma3b(acc[0], U0, VZ);
            mma3b(acc[1], U1, VZ);
            mma3b(acc[2], U2, VZ);
#pragma unroll
            for (int n = 0; n < 5; ++n) mma3b(acc[3 + n], U2, G[n]);
        }
        __syncwarp();
    }
    // add the warps' tiles in warp order and write this CTA's partial
    __syncthreads();
    float* sAcc = sStage;  // [warp][8][32][4]
#pragma unroll
    for (int T = 0; T < 8; ++T)
#pragma unroll
        for (int q = 0; q < 4; ++q) sAcc[((wid * 8 + T) * 32 + lane) * 4 + q] = acc[T][q];
    __syncthreads();
    float* gp = a.gpart + (int64_t)cta * po::syn_block;
    for (int e = tid; e < 8 * 32 * 4; e += kSynThreads) {
        const int T = e >> 7, l = (e >> 2) & 31, q = e & 3;
        const int row = (l >> 2) + (q >= 2 ? 8 : 0), col = 2 * (l & 3) + (q & 1);
        int second;
        const int idx = syn_wgrad_index(T, row, col, &second);
        if (idx < 0) continue;
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += sAcc[((w * 8 + T) * 32 + l) * 4 + q];
        gp[idx] = s;
        if (second >= 0) gp[second] = s;
    }
}

// 8 resident CTAs per SM (at most 64 registers): the forward is latency-bound, and the extra
// warps pay for the few spilled registers.
template <int PASS>
__global__ void __launch_bounds__(kSynThreads, 8) k_syn_fwd(const __grid_constant__ SynArgs a) {
    pdl_enter();
    syn_fwd_body<PASS, true>(a, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads, 8) k_syn_fwd_b(Batch<SynArgs> b) {
    __shared__ SynArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    syn_fwd_body<PASS, false>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads, 4) k_syn_bwd(const __grid_constant__ SynArgs a) {
    pdl_enter();
    syn_bwd_body<PASS>(a, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kSynThreads, 4) k_syn_bwd_b(Batch<SynArgs> b) {
    __shared__ SynArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    syn_bwd_body<PASS>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

size_t syn_bwd_smem() { return (size_t)FR_N * 32 * sizeof(float4) + (size_t)kWarps * kStage * sizeof(float); }

}  // namespace

void syn_init_attributes() {
    const int sm = (int)syn_bwd_smem();
    cudaFuncSetAttribute(k_syn_bwd<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_syn_bwd<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_syn_bwd_b<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_syn_bwd_b<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

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
    a.zden = w.zden;
    a.gpart = w.gpart_syn;
    a.dead = DeadRanges{};
    if (w.discard_dead) {
        a.dead.p[0] = w.t;
        a.dead.n[0] = 3 * w.HW;
    }
    return a;
}

// One wave at the forward's 8 resident CTAs per SM, each thread looping over its pixels (2 or 3
// at 512 x 768): faster than two waves of one or two pixels a thread.
int syn_fwd_ctas(const Work& w) {
    const int64_t blocks = (w.HW + kSynThreads - 1) / kSynThreads, cap = (int64_t)num_sms() * 8;
    return (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
}

void launch_syn_forward(const Work& w, const float* params, int pass, cudaStream_t s) {
    const SynArgs a = syn_args(w, params);
    if (pass == PASS_FWD_STORE)
        launch_pdl(k_syn_fwd<PASS_FWD_STORE>, syn_fwd_ctas(w), kSynThreads, 0, s, a);
    else
        launch_pdl(k_syn_fwd<PASS_FWD>, syn_fwd_ctas(w), kSynThreads, 0, s, a);
}

void launch_syn_backward(const Work& w, const float* params, int pass, cudaStream_t s) {
    const SynArgs a = syn_args(w, params);
    if (pass == PASS_BWD_LOAD)
        launch_pdl(k_syn_bwd<PASS_BWD_LOAD>, w.n_cta_syn, kSynThreads, syn_bwd_smem(), s, a);
    else
        launch_pdl(k_syn_bwd<PASS_FWD_BWD>, w.n_cta_syn, kSynThreads, syn_bwd_smem(), s, a);
}

void launch_syn_fwd_b(const Batch<SynArgs>& b, cudaStream_t s) {
    launch_pdl(k_syn_fwd_b<PASS_FWD>, b.total_ctas, kSynThreads, 0, s, b);
}
void launch_syn_bwd_b(const Batch<SynArgs>& b, cudaStream_t s) {
    launch_pdl(k_syn_bwd_b<PASS_FWD_BWD>, b.total_ctas, kSynThreads, syn_bwd_smem(), s, b);
}

}  // namespace cc
