// Entropy model of the encoder step (Sec. III-A, Eqs. 2-5, 9, 11) and its adjoint, on tensor cores.
//
// Per latent: the 16 causal neighbours of the relaxed latents (zero outside the grid), the IFCE of
// grids 0..2 on nearest-neighbour co-located coarser values, the ARM MLP 20 -> 16 -> 16 -> 2 with
// ReLU plus the linear stabilizer, log-scale clamped to [-5, 5], Laplace interval mass and rate
// -log2 max(P, 2^-16).  Adjoint: dL/dbits = lambda/(HW) gives dmu, dlogb, then the MLP adjoint
// gives dL/dc; context gradients are written as 16 planes dS[n][i] and gathered by their source
// latent later (fixed order, no atomics).
//
// Work unit: one warp, 16 latents (the M dimension of mma.sync.m16n8k8).  The products
// (latents x features) . (features x units) run as TF32 tensor-core MMAs with a three-pass split
// x = hi + lo (hi = tf32(x), lo = tf32(x - hi); D += lo*Bhi + hi*Blo + hi*Bhi), which keeps the
// result at FP32 accuracy.  An accumulator fragment feeds the next layer as its A fragment without
// data movement: the K order of the next layer is permuted so that the k-slot t of an 8-wide chunk
// is unit 2t and slot t+4 is unit 2t+1, and the B fragments (weights, pre-split per lane in shared
// memory) are laid out with the same permutation.
//
// Parameter gradients are sums over latents of outer products, i.e. GEMMs with K = latents: each
// warp transposes its 16 latents' factors into a private [feature][latent] shared tile and runs
// the 6 dense m16n8 output tiles (W1 and b1, W2, the IFCE weights) over K = 16 per work unit,
// accumulating in registers for the whole kernel.  The thin ones (b2, W3, Ws, b3 = bs: one or two
// gradient rows) are per-lane FMAs on values the lane already holds.  The 4 warps' accumulators
// are added in a fixed order at the end: one partial gradient per CTA.
//
// The first CTA also computes the coarse forward upsampling stages 6..4 (it needs none of the
// entropy model's results, and the other CTAs take the latents), so that they cost no launch.
#include "cc_kernels.h"
#include "cc_mma.cuh"
#include "cc_upfwd.cuh"

namespace cc {
namespace {

constexpr int kWarps = 4;
constexpr int kT = kWarps * 32;
constexpr int kSld = 20;  // staging row stride: 16 latents + 4 (conflict-free fragment reads)
// staging rows: U (gradient side) then V (activation side)
constexpr int U_DA1 = 0, U_DA2 = 16, U_O = 32;
constexpr int V_C = 48, V_H1 = 72, V_R = 88, S_ROWS = 96;
constexpr int kStage = S_ROWS * kSld;  // floats per warp
// B-fragment table (per fragment, per lane: b0 hi, b1 hi, b0 lo, b1 lo)
constexpr int FR_W1 = 0, FR_W2 = 6, FR_W3 = 10, FR_WS = 12, FR_BW2 = 15, FR_BW1 = 19, FR_N = 25;
constexpr int kIfceSm = 72;  // IFCE weights and biases, flat vector order (offsets relative to if_w0)

// Value of entry `which` (0: b0, 1: b1) of B fragment f for lane (g, t), from the flat parameters.
__device__ float bfrag_value(const float* P, int f, int g, int t, int which) {
    if (f < FR_W2) {  // layer 1: B[k = feature][n = unit] = W1aug[unit][feature], feature 20 = bias
        const int kc = f >> 1, nt = f & 1, unit = nt * 8 + g, feat = kc * 8 + t + 4 * which;
        return feat < 20 ? P[po::arm_w1 + unit * 20 + feat] : (feat == 20 ? P[po::arm_b1 + unit] : 0.f);
    }
    if (f < FR_W3) {  // layer 2, K permuted: B[k][n] = W2[n][unit(k)]
        const int kc = (f - FR_W2) >> 1, nt = (f - FR_W2) & 1, n = nt * 8 + g, u = kc * 8 + 2 * t + which;
        return P[po::arm_w2 + n * 16 + u];
    }
    if (f < FR_WS) {  // output from h2, K permuted, N = 8 (mu, s, zeros)
        const int kc = f - FR_W3, u = kc * 8 + 2 * t + which;
        return g < 2 ? P[po::arm_w3 + g * 16 + u] : 0.f;
    }
    if (f < FR_BW2) {  // stabilizer from c, N = 8 (mu, s, zeros)
        const int kc = f - FR_WS, feat = kc * 8 + t + 4 * which;
        return (g < 2 && feat < 20) ? P[po::arm_ws + g * 20 + feat] : 0.f;
    }
    if (f < FR_BW1) {  // adjoint of layer 2: B[k = o (permuted)][n = i] = W2[o][i]
        const int kc = (f - FR_BW2) >> 1, nt = (f - FR_BW2) & 1, o = kc * 8 + 2 * t + which, i = nt * 8 + g;
        return P[po::arm_w2 + o * 16 + i];
    }
    {  // adjoint of layer 1: B[k = o (permuted)][n = feature] = W1[o][feature]
        const int kc = (f - FR_BW1) / 3, nt = (f - FR_BW1) % 3, o = kc * 8 + 2 * t + which, feat = nt * 8 + g;
        return feat < 20 ? P[po::arm_w1 + o * 20 + feat] : 0.f;
    }
}


struct LatentPos {
    int k, r, c, li;
    bool valid;
    int64_t i;
};

// position of latent i; the row is li / w via a float reciprocal, corrected to the exact quotient
__device__ __forceinline__ LatentPos locate(const Geom& g, const float* rcp_w, int64_t i, int64_t N) {
    LatentPos p;
    p.valid = i < N;
    p.i = p.valid ? i : N - 1;
    p.k = grid_of(g, p.i);
    p.li = (int)(p.i - g.off[p.k]);
    const int w = g.w[p.k];
    int r = __float2int_rz(__int2float_rn(p.li) * rcp_w[p.k]);
    r -= (r * w > p.li) ? 1 : 0;
    r += ((r + 1) * w <= p.li) ? 1 : 0;
    p.r = r;
    p.c = p.li - r * w;
    return p;
}

// Context feature f (0..23) of a latent: neighbours 0..15, IFCE outputs 16..19, one (20), zeros.
__device__ __forceinline__ float neighbour(const Geom& g, const float* yt, const LatentPos& p, int dy, int dx) {
    const int rr = p.r + dy, cc = p.c + dx, w = g.w[p.k];
    return (rr >= 0 && cc >= 0 && cc < w) ? __ldg(yt + g.off[p.k] + rr * w + cc) : 0.f;
}

// IFCE inputs j = t and j = t + 4 of a latent (lane t of its quad; zero where j >= nin): the
// nearest-neighbour co-located values of grids k+1+j.
__device__ __forceinline__ void ifce_inputs(const Geom& g, const float* yt, const LatentPos& p, int t, float& r0,
                                            float& r1) {
    const int nin = ifce_nin(p.k);
    auto at = [&](int j) {
        const int gj = p.k + 1 + j;
        const int rr = min(p.r >> (j + 1), g.h[gj] - 1), cc = min(p.c >> (j + 1), g.w[gj] - 1);
        return __ldg(yt + g.off[gj] + rr * g.w[gj] + cc);
    };
    r0 = t < nin ? at(t) : 0.f;
    r1 = t + 4 < nin ? at(t + 4) : 0.f;
}

// IFCE output t of a latent in lane t of its quad: each lane forms the products of its two inputs
// with all four output rows, and a transposing butterfly over the quad (lanes t ^ 2, then t ^ 1)
// leaves the sum of output t in lane t.  All 32 lanes take part in the shuffles.
__device__ __forceinline__ float ifce_out(const float* sIf, int k, int t, float r0, float r1) {
    const int nin = ifce_nin(k);
    const int wo = ifce_w_off(k < kNIfce ? k : 0) - po::if_w0, bo = ifce_b_off(k < kNIfce ? k : 0) - po::if_w0;
    float part[kF];
#pragma unroll
    for (int o = 0; o < kF; ++o) {
        const float w0 = t < nin ? sIf[wo + o * nin + t] : 0.f;
        const float w1 = t + 4 < nin ? sIf[wo + o * nin + t + 4] : 0.f;
        part[o] = fmaf(w1, r1, w0 * r0);
    }
    const bool b1 = t & 2, b0 = t & 1;
    float keep0 = b1 ? part[2] : part[0], keep1 = b1 ? part[3] : part[1];
    keep0 += __shfl_xor_sync(0xffffffffu, b1 ? part[0] : part[2], 2);
    keep1 += __shfl_xor_sync(0xffffffffu, b1 ? part[1] : part[3], 2);
    float keep = b0 ? keep1 : keep0;
    keep += __shfl_xor_sync(0xffffffffu, b0 ? keep0 : keep1, 1);
    return nin > 0 ? keep + sIf[bo + t] : 0.f;
}

// Parameter index of weight-gradient tile T, row, column (-1: padding).
__device__ int wgrad_index(int T, int row, int col) {
    if (T <= 2) {
        const int f = T * 8 + col;
        return f < 20 ? po::arm_w1 + row * 20 + f : (f == 20 ? po::arm_b1 + row : -1);
    }
    if (T <= 4) return po::arm_w2 + row * 16 + (T - 3) * 8 + col;
    if (row < 2 || row >= 14) return -1;  // T == 5: IFCE output gradients x IFCE inputs
    const int k = (row - 2) >> 2, o = (row - 2) & 3, nin = ifce_nin(k);
    if (col < nin) return ifce_w_off(k) + o * nin + col;
    if (col == 6) return ifce_b_off(k) + o;
    return -1;
}

// The coarse forward upsampling stages of CTA 0, out of line: inlined, their registers would
// shape the allocation of the latent loop.
__device__ __noinline__ void coarse_upsampling(const ArmArgs& a, float* sm) {
#pragma unroll 1
    for (int q = 0; q < kUpArmStages; ++q) up_fwd_stage_cta(a.upc[q], sm, kWarps * kStage);
}

template <int PASS>
__device__ __forceinline__ void arm_body(const ArmArgs& a, int cta, int ncta) {
    constexpr bool BWD = pass_bwd(PASS);
    extern __shared__ float4 smem4[];
    float4* sFr = smem4;                                             // [FR_N][32]
    float* sIf = reinterpret_cast<float*>(smem4 + FR_N * 32);        // [kIfceSm]
    float* sStage = sIf + kIfceSm;                                   // [kWarps][kStage]
    __shared__ Geom g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;

    __shared__ float rcp_w[kL];
    if (tid == 0) g = a.g;
    if (tid < kL) rcp_w[tid] = 1.f / (float)a.g.w[tid];
    // the entropy-model and IFCE parameters staged in one round trip, through the staging area
    // (free until the coarse stages and the first unit)
    const float* P = stage_params(a.params, 0, po::arm_block, sStage);
    for (int j = tid; j < FR_N * 32; j += kT) {
        const int f = j >> 5, l = j & 31;
        const float v0 = bfrag_value(P, f, l >> 2, l & 3, 0);
        const float v1 = bfrag_value(P, f, l >> 2, l & 3, 1);
        uint32_t h0, l0, h1, l1;
        split2(v0, h0, l0);
        split2(v1, h1, l1);
        sFr[j] = make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(l0), __uint_as_float(l1));
    }
    for (int j = tid; j < kIfceSm; j += kT) sIf[j] = P[po::if_w0 + j];

    // per-lane constants of the SIMT parts, read as float2 (units / features 2t, 2t+1 of a tile)
    __shared__ __align__(16) float sC[16 + 2 * 16 + 2 * 24];  // b2 [16], W3 [2][16], Ws [2][24] (zero-padded)
    for (int j = tid; j < 96; j += kT) {
        float v;
        if (j < 16) v = P[po::arm_b2 + j];
        else if (j < 48) v = P[po::arm_w3 + (j - 16)];
        else {
            const int o = (j - 48) / 24, f = (j - 48) % 24;
            v = f < 20 ? P[po::arm_ws + o * 20 + f] : 0.f;
        }
        sC[j] = v;
    }
    const float2* b2c = reinterpret_cast<const float2*>(sC) + tq;          // [nt * 4]
    const float2* w3c = reinterpret_cast<const float2*>(sC + 16) + tq;     // [o * 8 + nt * 4]
    const float2* wsc = reinterpret_cast<const float2*>(sC + 48) + tq;     // [o * 12 + nt * 4]
    const float mu_b = P[po::arm_b3] + P[po::arm_bs];
    const float s_b = P[po::arm_b3 + 1] + P[po::arm_bs + 1];
    __syncthreads();  // (the staged parameters are dead from here: the staging area is reused)
    // context slots t, t+4, t+8, t+12 of this lane, packed 5 bits each: dy + 3 (2 bits), dx + 3 (3 bits)
    int nd = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) nd |= ((ctx_dy(tq + 4 * q) + 3) | ((ctx_dx(tq + 4 * q) + 3) << 2)) << (5 * q);

    // CTA 0 computes the coarse forward upsampling stages (it takes no latents when there are
    // other CTAs), staged through the weight-gradient staging area before its constant rows are
    // set; each stage ends with a barrier, so its output is visible to the next.
    //   Units: with W warps in all, no warp takes more than Q = ceil(units / W); the warps of CTAs
    // 1.. take units [0, U1) round-robin (U1 = min(units, Q * their number)) and the warps of CTA 0
    // only the rest [U1, units), so that the coarse stages do not lengthen the launch.
    // (units < 2^31: images are at most 16384 x 16384)
    const int64_t N = a.N;
    const int n_units = (int)((N + 15) / 16);
    int u_first = cta * kWarps + wid, u_step = ncta * kWarps, u_end = n_units;
    if (a.upc_on) {
        if (cta == 0) coarse_upsampling(a, sStage);
        if (ncta > 1) {
            const int w_all = ncta * kWarps, w_reg = w_all - kWarps;
            const int q_max = (int)(((int64_t)n_units + w_all - 1) / w_all);
            const int u1 = (int)std::min<int64_t>(n_units, (int64_t)q_max * w_reg);
            if (cta > 0) {
                u_first = (cta - 1) * kWarps + wid;
                u_step = w_reg;
                u_end = u1;
            } else {
                u_first = u1 + wid;
                u_step = kWarps;
            }
        }
    }

    float* st = sStage + wid * kStage;
    if (BWD) {  // constant staging rows: C one (20) and zeros (21-23), R one (6) and zero (7), U_O zeros (0, 1, 14, 15)
        for (int j = lane; j < kSld; j += 32) {
            st[(V_C + 20) * kSld + j] = 1.f;
            st[(V_C + 21) * kSld + j] = 0.f;
            st[(V_C + 22) * kSld + j] = 0.f;
            st[(V_C + 23) * kSld + j] = 0.f;
            st[(V_R + 6) * kSld + j] = 1.f;
            st[(V_R + 7) * kSld + j] = 0.f;
            st[(U_O + 0) * kSld + j] = 0.f;
            st[(U_O + 1) * kSld + j] = 0.f;
            st[(U_O + 14) * kSld + j] = 0.f;
            st[(U_O + 15) * kSld + j] = 0.f;
        }
        __syncwarp();
    }
    float acc[6][4];
#pragma unroll
    for (int T = 0; T < 6; ++T)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[T][q] = 0.f;
    // per-lane sums: b2 of units 2t+cc (+8nt); W3[o][2t+cc (+8nt)]; Ws[o][t + 4q] (q = 5, t = 0: b3 = bs)
    float sb2[2][2], sw3[2][2][2], sws[6][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            sb2[nt][cc] = 0.f;
            sw3[nt][cc][0] = sw3[nt][cc][1] = 0.f;
        }
#pragma unroll
    for (int q = 0; q < 6; ++q) sws[q][0] = sws[q][1] = 0.f;
    float rate_acc = 0.f;

    for (int u = u_first; u < u_end; u += u_step) {
        const LatentPos pA = locate(g, rcp_w, (int64_t)u * 16 + gq, N);
        const LatentPos pB = locate(g, rcp_w, (int64_t)u * 16 + gq + 8, N);
        // ---- context features f in {t, t+4, 8+t, 12+t, 16+t, 20+t} of latents A (row g) and B (row g+8)
        float rA0, rA1, rB0, rB1;  // IFCE inputs tq and tq + 4 of latents A and B
        ifce_inputs(g, a.yt, pA, tq, rA0, rA1);
        ifce_inputs(g, a.yt, pB, tq, rB0, rB1);
        float cA[6], cB[6];
        int ndy[4], ndx[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ndy[q] = ((nd >> (5 * q)) & 3) - 3;
            ndx[q] = ((nd >> (5 * q + 2)) & 7) - 3;
        }
        cA[0] = neighbour(g, a.yt, pA, ndy[0], ndx[0]);
        cA[1] = neighbour(g, a.yt, pA, ndy[1], ndx[1]);
        cA[2] = neighbour(g, a.yt, pA, ndy[2], ndx[2]);
        cA[3] = neighbour(g, a.yt, pA, ndy[3], ndx[3]);
        cA[4] = ifce_out(sIf, pA.k, tq, rA0, rA1);
        cA[5] = tq == 0 ? 1.f : 0.f;
        cB[0] = neighbour(g, a.yt, pB, ndy[0], ndx[0]);
        cB[1] = neighbour(g, a.yt, pB, ndy[1], ndx[1]);
        cB[2] = neighbour(g, a.yt, pB, ndy[2], ndx[2]);
        cB[3] = neighbour(g, a.yt, pB, ndy[3], ndx[3]);
        cB[4] = ifce_out(sIf, pB.k, tq, rB0, rB1);
        cB[5] = cA[5];
        const AFrag C0 = make_a(cA[0], cB[0], cA[1], cB[1]);
        const AFrag C1 = make_a(cA[2], cB[2], cA[3], cB[3]);
        const AFrag C2 = make_a(cA[4], cB[4], cA[5], cB[5]);

        float d1[2][4], d2[2][4];
        float muA, sA, muB, sB;
        if (PASS == PASS_BWD_LOAD) {
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int uu = nt * 8 + 2 * tq + cc;
                    d1[nt][cc] = a.act[(int64_t)uu * N + pA.i];
                    d1[nt][2 + cc] = a.act[(int64_t)uu * N + pB.i];
                    d2[nt][cc] = a.act[(int64_t)(16 + uu) * N + pA.i];
                    d2[nt][2 + cc] = a.act[(int64_t)(16 + uu) * N + pB.i];
                }
            muA = a.act[(int64_t)32 * N + pA.i];
            sA = a.act[(int64_t)33 * N + pA.i];
            muB = a.act[(int64_t)32 * N + pB.i];
            sB = a.act[(int64_t)33 * N + pB.i];
        } else {
            // layer 1 (bias through the constant feature 20)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float e[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int q = 0; q < 4; ++q) d1[nt][q] = 0.f;
                mma3(d1[nt], e, C0, sFr[(FR_W1 + 0 * 2 + nt) * 32 + lane]);
                mma3(d1[nt], e, C1, sFr[(FR_W1 + 1 * 2 + nt) * 32 + lane]);
                mma3(d1[nt], e, C2, sFr[(FR_W1 + 2 * 2 + nt) * 32 + lane]);
                add4(d1[nt], e);
            }
            float h1[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) h1[nt][q] = fmaxf(d1[nt][q], 0.f);
            const AFrag H10 = chain(h1[0]), H11 = chain(h1[1]);
            // layer 2
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const float2 bb = b2c[nt * 4];
                d2[nt][0] = bb.x;
                d2[nt][1] = bb.y;
                d2[nt][2] = bb.x;
                d2[nt][3] = bb.y;
                float e[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(d2[nt], e, H10, sFr[(FR_W2 + 0 * 2 + nt) * 32 + lane]);
                mma3(d2[nt], e, H11, sFr[(FR_W2 + 1 * 2 + nt) * 32 + lane]);
                add4(d2[nt], e);
            }
            float h2[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) h2[nt][q] = fmaxf(d2[nt][q], 0.f);
            const AFrag H20 = chain(h2[0]), H21 = chain(h2[1]);
            // output (mu, s) + stabilizer
            float dout[4];
            dout[0] = tq == 0 ? mu_b : 0.f;
            dout[1] = tq == 0 ? s_b : 0.f;
            dout[2] = dout[0];
            dout[3] = dout[1];
            {
                float e[4] = {0.f, 0.f, 0.f, 0.f}, f2[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(dout, e, H20, sFr[(FR_W3 + 0) * 32 + lane]);
                mma3(dout, e, H21, sFr[(FR_W3 + 1) * 32 + lane]);
                mma3(f2, e2, C0, sFr[(FR_WS + 0) * 32 + lane]);
                mma3(f2, e2, C1, sFr[(FR_WS + 1) * 32 + lane]);
                mma3(f2, e2, C2, sFr[(FR_WS + 2) * 32 + lane]);
                add4(e, e2);
                add4(f2, e);
                add4(dout, f2);
            }
            const int q0 = lane & ~3;
            muA = __shfl_sync(0xffffffffu, dout[0], q0);
            sA = __shfl_sync(0xffffffffu, dout[1], q0);
            muB = __shfl_sync(0xffffffffu, dout[2], q0);
            sB = __shfl_sync(0xffffffffu, dout[3], q0);
            if (PASS == PASS_FWD_STORE) {
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        const int uu = nt * 8 + 2 * tq + cc;
                        if (pA.valid) {
                            a.act[(int64_t)uu * N + pA.i] = d1[nt][cc];
                            a.act[(int64_t)(16 + uu) * N + pA.i] = d2[nt][cc];
                        }
                        if (pB.valid) {
                            a.act[(int64_t)uu * N + pB.i] = d1[nt][2 + cc];
                            a.act[(int64_t)(16 + uu) * N + pB.i] = d2[nt][2 + cc];
                        }
                    }
                if (tq == 0 && pA.valid) {
                    a.act[(int64_t)32 * N + pA.i] = muA;
                    a.act[(int64_t)33 * N + pA.i] = sA;
                }
                if (tq == 0 && pB.valid) {
                    a.act[(int64_t)32 * N + pB.i] = muB;
                    a.act[(int64_t)33 * N + pB.i] = sB;
                }
            }
        }
        // ---- Laplace mass: lanes with even t take latent A, odd t latent B
        const bool odd = tq & 1;
        const LatentPos& pm = odd ? pB : pA;
        const float mu = odd ? muB : muA, s = odd ? sB : sA;
        const float logb = fminf(fmaxf(s, kLogbMin), kLogbMax);
        const LapOut L = laplace_mass(__ldg(a.yt + pm.i), mu, logb);
        if (tq < 2 && pm.valid) rate_acc += -log2f(fmaxf(L.p, kPMin));
        if (!BWD) continue;

        const float dp = (pm.valid && L.p >= kPMin) ? -a.gscale / (L.p * 0.69314718055994531f) : 0.f;
        const float dyd = dp * L.dp_dy;
        const float dmu = -dyd;
        const float ds = (s >= kLogbMin && s <= kLogbMax) ? dp * L.dp_dlogb : 0.f;
        if (tq < 2 && pm.valid) a.dYd[pm.i] = dyd;
        const int q0 = lane & ~3;
        const float dmuA = __shfl_sync(0xffffffffu, dmu, q0), dsA = __shfl_sync(0xffffffffu, ds, q0);
        const float dmuB = __shfl_sync(0xffffffffu, dmu, q0 + 1), dsB = __shfl_sync(0xffffffffu, ds, q0 + 1);

        // dA2 = (dout . W3) masked by a2 > 0
        float da2[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const float2 m = w3c[nt * 4], sv = w3c[8 + nt * 4];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const float wm = cc ? m.y : m.x, ws = cc ? sv.y : sv.x;
                const float vA = dmuA * wm + dsA * ws;
                const float vB = dmuB * wm + dsB * ws;
                da2[nt][cc] = d2[nt][cc] > 0.f ? vA : 0.f;
                da2[nt][2 + cc] = d2[nt][2 + cc] > 0.f ? vB : 0.f;
            }
        }
        const AFrag DA20 = chain(da2[0]), DA21 = chain(da2[1]);
        // dA1 = (dA2 . W2) masked by a1 > 0
        float da1[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
            for (int q = 0; q < 4; ++q) da1[nt][q] = 0.f;
            float e[4] = {0.f, 0.f, 0.f, 0.f};
            mma3(da1[nt], e, DA20, sFr[(FR_BW2 + 0 * 2 + nt) * 32 + lane]);
            mma3(da1[nt], e, DA21, sFr[(FR_BW2 + 1 * 2 + nt) * 32 + lane]);
            add4(da1[nt], e);
#pragma unroll
            for (int q = 0; q < 4; ++q) da1[nt][q] = d1[nt][q] > 0.f ? da1[nt][q] : 0.f;
        }
        const AFrag DA10 = chain(da1[0]), DA11 = chain(da1[1]);
        // dC = dA1 . W1 + dout . Ws
        float dc[3][4];
#pragma unroll
        for (int nt = 0; nt < 3; ++nt) {
            const float2 m = wsc[nt * 4], sv = wsc[12 + nt * 4];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const float wm = cc ? m.y : m.x, ws = cc ? sv.y : sv.x;
                dc[nt][cc] = dmuA * wm + dsA * ws;
                dc[nt][2 + cc] = dmuB * wm + dsB * ws;
            }
            float e[4] = {0.f, 0.f, 0.f, 0.f};
            mma3(dc[nt], e, DA10, sFr[(FR_BW1 + 0 * 3 + nt) * 32 + lane]);
            mma3(dc[nt], e, DA11, sFr[(FR_BW1 + 1 * 3 + nt) * 32 + lane]);
            add4(dc[nt], e);
        }
        // context-gradient planes (features 0..15)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int f = nt * 8 + 2 * tq + cc;
                if (pA.valid) a.dS[(int64_t)f * N + pA.i] = dc[nt][cc];
                if (pB.valid) a.dS[(int64_t)f * N + pB.i] = dc[nt][2 + cc];
            }
        // IFCE output gradients df[0..3] (features 16..19 live in lanes t = 0, 1 of tile 2)
        float dfA[4], dfB[4];
        dfA[0] = __shfl_sync(0xffffffffu, dc[2][0], q0);
        dfA[1] = __shfl_sync(0xffffffffu, dc[2][1], q0);
        dfA[2] = __shfl_sync(0xffffffffu, dc[2][0], q0 + 1);
        dfA[3] = __shfl_sync(0xffffffffu, dc[2][1], q0 + 1);
        dfB[0] = __shfl_sync(0xffffffffu, dc[2][2], q0);
        dfB[1] = __shfl_sync(0xffffffffu, dc[2][3], q0);
        dfB[2] = __shfl_sync(0xffffffffu, dc[2][2], q0 + 1);
        dfB[3] = __shfl_sync(0xffffffffu, dc[2][3], q0 + 1);
        // IFCE input gradients dr_j = sum_o W_k[o][j] df[o]; lane t writes j = t and t + 4
        auto write_dr = [&](const LatentPos& p, const float (&df)[4]) {
            const int nin = ifce_nin(p.k);
            if (nin > 0 && p.valid) {
                float* dR = p.k == 0 ? a.dR0 : (p.k == 1 ? a.dR1 : a.dR2);
                const int nk = g.h[p.k] * g.w[p.k];
                const int wo = ifce_w_off(p.k) - po::if_w0;
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    const int j = tq + 4 * jj;
                    if (j < nin) {
                        float v = 0.f;
#pragma unroll
                        for (int o = 0; o < kF; ++o) v = fmaf(sIf[wo + o * nin + j], df[o], v);
                        dR[(int64_t)j * nk + p.li] = v;
                    }
                }
            }
        };
        write_dr(pA, dfA);
        write_dr(pB, dfB);
        // ---- stage the outer-product factors, transposed to [feature][latent]
        const float mA = pA.valid ? 1.f : 0.f, mB = pB.valid ? 1.f : 0.f;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int uu = nt * 8 + 2 * tq + cc;
                st[(U_DA1 + uu) * kSld + gq] = da1[nt][cc] * mA;
                st[(U_DA1 + uu) * kSld + gq + 8] = da1[nt][2 + cc] * mB;
                st[(U_DA2 + uu) * kSld + gq] = da2[nt][cc] * mA;
                st[(U_DA2 + uu) * kSld + gq + 8] = da2[nt][2 + cc] * mB;
                st[(V_H1 + uu) * kSld + gq] = fmaxf(d1[nt][cc], 0.f);
                st[(V_H1 + uu) * kSld + gq + 8] = fmaxf(d1[nt][2 + cc], 0.f);
                // thin parameter gradients (d mu, d log b are zero for latents past the end)
                const float hA = fmaxf(d2[nt][cc], 0.f), hB = fmaxf(d2[nt][2 + cc], 0.f);
                sb2[nt][cc] += da2[nt][cc] * mA + da2[nt][2 + cc] * mB;
                sw3[nt][cc][0] = fmaf(dmuA, hA, fmaf(dmuB, hB, sw3[nt][cc][0]));
                sw3[nt][cc][1] = fmaf(dsA, hA, fmaf(dsB, hB, sw3[nt][cc][1]));
            }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            sws[q][0] = fmaf(dmuA, cA[q], fmaf(dmuB, cB[q], sws[q][0]));
            sws[q][1] = fmaf(dsA, cA[q], fmaf(dsB, cB[q], sws[q][1]));
        }
        {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                st[(V_C + tq + 4 * q) * kSld + gq] = cA[q];
                st[(V_C + tq + 4 * q) * kSld + gq + 8] = cB[q];
            }
            // U_O rows t, t+4, t+8, t+12: 2..13 df of grid (row-2)/4; 0, 1, 14, 15 zero (preset)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = tq + 4 * q;
                if (row < 2 || row >= 14) continue;
                const int kk = (row - 2) >> 2, o = (row - 2) & 3;
                const float vA = pA.k == kk ? sel(dfA, o) : 0.f;
                const float vB = pB.k == kk ? sel(dfB, o) : 0.f;
                st[(U_O + row) * kSld + gq] = vA * mA;
                st[(U_O + row) * kSld + gq + 8] = vB * mB;
            }
            // R rows t and t+4 (rows 6, 7 are the preset one and zero)
            st[(V_R + tq) * kSld + gq] = rA0;
            st[(V_R + tq) * kSld + gq + 8] = rB0;
            if (tq < 2) {
                st[(V_R + tq + 4) * kSld + gq] = rA1;
                st[(V_R + tq + 4) * kSld + gq + 8] = rB1;
            }
        }
        __syncwarp();
        // ---- parameter-gradient tiles over K = 16 latents (two k-steps of 8), fragments by ldmatrix:
        // an A fragment (16 rows) is matrices (rows 0-7, k 0-3), (8-15, 0-3), (0-7, 4-7), (8-15, 4-7);
        // a pair of B fragments (8 rows each) is (rows of the first, k 0-3), (first, 4-7),
        // (second, 0-3), (second, 4-7).
        {
            const int mi = lane >> 3, ri = lane & 7;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int k0 = ks * 8;
                const float* arow = st + (ri + (mi & 1) * 8) * kSld + k0 + (mi >> 1) * 4;  // + row0 * kSld
                const float* brow = st + ri * kSld + k0 + (mi & 1) * 4;                    // + first/second row0
                auto afrag = [&](int row0) {
                    uint32_t r[4];
                    ldsm_x4(r, arow + row0 * kSld);
                    AFrag f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) split_u(r[q], f.h[q], f.l[q]);
                    return f;
                };
                auto bpair = [&](int row0a, int row0b, AFrag& fa, AFrag& fb) {  // (b0, b1) in h[0..1], l[0..1]
                    uint32_t r[4];
                    ldsm_x4(r, brow + ((mi >> 1) ? row0b : row0a) * kSld);
                    split_u(r[0], fa.h[0], fa.l[0]);
                    split_u(r[1], fa.h[1], fa.l[1]);
                    split_u(r[2], fb.h[0], fb.l[0]);
                    split_u(r[3], fb.h[1], fb.l[1]);
                };
                {
                    const AFrag UA1 = afrag(U_DA1);
                    AFrag VC0, VC1, VC2, VR;
                    bpair(V_C, V_C + 8, VC0, VC1);
                    mma3b(acc[0], UA1, VC0);
                    mma3b(acc[1], UA1, VC1);
                    bpair(V_C + 16, V_R, VC2, VR);
                    mma3b(acc[2], UA1, VC2);
                    const AFrag UO = afrag(U_O);
                    mma3b(acc[5], UO, VR);
                }
                {
                    const AFrag UA2 = afrag(U_DA2);
                    AFrag VH10, VH11;
                    bpair(V_H1, V_H1 + 8, VH10, VH11);
                    mma3b(acc[3], UA2, VH10);
                    mma3b(acc[4], UA2, VH11);
                }
            }
        }
        __syncwarp();
    }

    // rate partial of this CTA
    {
        float v[1] = {rate_acc};
        __shared__ float scratch[kT / 32];
        block_sum<1>(v, scratch);
        if (tid == 0) a.rate_part[cta] = (double)v[0];
    }
    if constexpr (BWD) {
    // the 4 warps' gradient tiles and per-lane sums, added in warp order
    float simt[24];  // sb2 (4), sw3 (8), sws (12), each summed over the 8 lanes of the same t
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            simt[nt * 2 + cc] = sb2[nt][cc];
            simt[4 + (nt * 2 + cc) * 2] = sw3[nt][cc][0];
            simt[4 + (nt * 2 + cc) * 2 + 1] = sw3[nt][cc][1];
        }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        simt[12 + 2 * q] = sws[q][0];
        simt[12 + 2 * q + 1] = sws[q][1];
    }
#pragma unroll
    for (int j = 0; j < 24; ++j) {
        simt[j] += __shfl_xor_sync(0xffffffffu, simt[j], 4);
        simt[j] += __shfl_xor_sync(0xffffffffu, simt[j], 8);
        simt[j] += __shfl_xor_sync(0xffffffffu, simt[j], 16);
    }
    __syncthreads();
    float* sAcc = sStage;                         // [warp][T][lane][4]
    float* sSimt = sStage + kWarps * 6 * 32 * 4;  // [warp][t][24]
#pragma unroll
    for (int T = 0; T < 6; ++T)
#pragma unroll
        for (int q = 0; q < 4; ++q) sAcc[((wid * 6 + T) * 32 + lane) * 4 + q] = acc[T][q];
    if (lane < 4)
#pragma unroll
        for (int j = 0; j < 24; ++j) sSimt[(wid * 4 + lane) * 24 + j] = simt[j];
    __syncthreads();
    float* gp = a.gpart + (int64_t)cta * po::arm_block;
    for (int e = tid; e < 6 * 32 * 4; e += kT) {
        const int T = e >> 7, l = (e >> 2) & 31, q = e & 3;
        const int row = (l >> 2) + (q >= 2 ? 8 : 0), col = 2 * (l & 3) + (q & 1);
        const int idx = wgrad_index(T, row, col);
        if (idx < 0) continue;
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += sAcc[((w * 6 + T) * 32 + l) * 4 + q];
        gp[idx] = s;
    }
    if (tid < 4 * 24) {
        const int t = tid / 24, j = tid - t * 24;
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += sSimt[(w * 4 + t) * 24 + j];
        if (j < 4) {
            gp[po::arm_b2 + (j >> 1) * 8 + 2 * t + (j & 1)] = s;
        } else if (j < 12) {
            const int jj = j - 4, u = (jj >> 2) * 8 + 2 * t + ((jj >> 1) & 1), o = jj & 1;
            gp[po::arm_w3 + o * 16 + u] = s;
        } else {
            const int q = (j - 12) >> 1, o = (j - 12) & 1, f = t + 4 * q;
            if (q < 5) {
                gp[po::arm_ws + o * 20 + f] = s;
            } else if (t == 0) {
                gp[po::arm_b3 + o] = s;
                gp[po::arm_bs + o] = s;
            }
        }
    }
    }  // BWD
}

template <int PASS>
__global__ void __launch_bounds__(kT, 3) k_arm(const __grid_constant__ ArmArgs a) {
    __shared__ ArmArgs sa;
    param_fetch(a, sa);
    arm_body<PASS>(sa, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kT, 3) k_arm_b(Batch<ArmArgs> b) {
    __shared__ ArmArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    arm_body<PASS>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

}  // namespace

size_t arm_smem_bytes(int pass) {  // staging tiles: weight-gradient factors, or the coarse upsampling in CTA 0
    (void)pass;
    return (size_t)FR_N * 32 * sizeof(float4) + (size_t)(kIfceSm + kWarps * kStage) * sizeof(float);
}

int arm_grid(int64_t N) {
    const int64_t units = (N + 15) / 16;
    const int64_t ctas = (units + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)num_sms() * 3;  // 3 resident CTAs per SM
    return (int)(ctas < cap ? (ctas < 1 ? 1 : ctas) : cap);
}

ArmArgs arm_args(const Work& w, const float* params, float grad_scale) {
    ArmArgs a;
    for (int q = 0; q < kUpArmStages; ++q) a.upc[q] = up_fwd_args(w, params, kL - 2 - q);
    a.upc_on = 1;
    a.pad2_ = 0;
    a.pad_ = 0;
    a.g = w.g;
    a.N = w.N;
    a.yt = w.yt;
    a.params = params;
    a.gscale = grad_scale;
    a.dS = w.dS;
    a.dR0 = w.dR[0];
    a.dR1 = w.dR[1];
    a.dR2 = w.dR[2];
    a.dYd = w.dYd;
    a.act = w.act_arm;
    a.gpart = w.gpart_arm;
    a.rate_part = w.rate_part;
    return a;
}

void launch_arm(const Work& w, const float* params, int pass, float grad_scale, cudaStream_t s) {
    ArmArgs a = arm_args(w, params, grad_scale);
    if (pass == PASS_BWD_LOAD) a.upc_on = 0;  // the upsampled grids are still in the workspace
    const size_t sm = arm_smem_bytes(pass);
    const int grid = w.n_cta_arm;
    switch (pass) {
        case PASS_FWD: launch_pdl(k_arm<PASS_FWD>, grid, kT, sm, s, a); break;
        case PASS_FWD_STORE: launch_pdl(k_arm<PASS_FWD_STORE>, grid, kT, sm, s, a); break;
        case PASS_FWD_BWD: launch_pdl(k_arm<PASS_FWD_BWD>, grid, kT, sm, s, a); break;
        default: launch_pdl(k_arm<PASS_BWD_LOAD>, grid, kT, sm, s, a); break;
    }
}

void launch_arm_b(const Batch<ArmArgs>& b, int pass, cudaStream_t s) {
    const size_t sm = arm_smem_bytes(pass);
    switch (pass) {
        case PASS_FWD: launch_pdl(k_arm_b<PASS_FWD>, b.total_ctas, kT, sm, s, b); break;
        case PASS_FWD_STORE: launch_pdl(k_arm_b<PASS_FWD_STORE>, b.total_ctas, kT, sm, s, b); break;
        case PASS_FWD_BWD: launch_pdl(k_arm_b<PASS_FWD_BWD>, b.total_ctas, kT, sm, s, b); break;
        default: launch_pdl(k_arm_b<PASS_BWD_LOAD>, b.total_ctas, kT, sm, s, b); break;
    }
}

void arm_init_attributes() {
    const int sm = (int)arm_smem_bytes(PASS_FWD_BWD);
    cudaFuncSetAttribute(k_arm<PASS_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm<PASS_FWD_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm_b<PASS_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm_b<PASS_FWD_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm_b<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_arm_b<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

}  // namespace cc
