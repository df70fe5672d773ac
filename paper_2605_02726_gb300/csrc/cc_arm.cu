// Entropy model of the encoder step (Sec. III-A, Eqs. 2-5, 9, 11) and its adjoint.
//
// One thread per latent, all grids in one launch.  Per latent: the 16 causal neighbours of the
// relaxed latents (zero outside the grid), the IFCE of grids 0..2 on nearest-neighbour co-located
// coarser values, the ARM MLP 20 -> 16 -> 16 -> 2 with ReLU plus the linear stabilizer, log-scale
// clamped to [-5, 5], Laplace interval mass, rate -log2 max(P, 2^-16).
//
// Adjoint (same kernel, recomputed or from stored activations): dL/dbits = lambda/(HW) gives
// dmu, dlogb, then the MLP adjoint gives dL/dc.  Context gradients are not scattered: they are
// written as 16 planes dS[n][i] and gathered by their source latent in the gather kernel, which
// keeps every sum in a fixed order (bit-reproducible, no atomics).
//
// Parameter gradients are outer-product sums over latents.  Each round of 128 latents stages the
// factors in shared memory (U = gradients, V = activations, [row][latent]) and 114 threads each
// update an 8x8 register block over a slice of the latents; the 6 slices of a block are added
// in a fixed order at the end, giving one partial gradient per CTA (reduced later in fixed order).
#include "cc_kernels.h"

namespace cc {
namespace {

constexpr int kT = kArmThreads;
constexpr int kLd = kT + 4;          // staging row stride (floats): 16 B aligned, skewed banks
constexpr int kURows = 56, kVRows = 64;
constexpr int kChunks = 6;
constexpr int kBlocks = 19;
constexpr int kTasks = kBlocks * kChunks;  // 114 <= kT
constexpr int kWSm = 768;            // shared copy of ARM + IFCE weights (re-laid out, see below)

// Shared weight layout: W1 [16][20] @0, b1 @320, W2 [16][16] @336, b2 @592, W3 [2][16] @608,
// Ws [2][20] @640 (16 B aligned, unlike the flat vector), b3 + bs @680, IFCE as in the flat vector.
constexpr int sw_w1 = 0, sw_b1 = 320, sw_w2 = 336, sw_b2 = 592, sw_w3 = 608, sw_ws = 640, sw_bo = 680;

// Staging rows.  U: da1 0-15, da2 16-31, dmu 32, ds 33, (zero 34-39), df0 40-43, df1 44-47,
// df2 48-51, (zero 52-55).  V: c 0-19, one 20, (zero 21-23), h1 24-39, h2 40-55, r 56-61,
// one 62, (zero 63).
__constant__ unsigned char c_blk_u[kBlocks] = {0, 0, 0, 8, 8, 8, 16, 16, 24, 24, 16, 24, 32, 32, 32, 32, 32, 40, 48};
__constant__ unsigned char c_blk_v[kBlocks] = {0, 8, 16, 0, 8, 16, 24, 32, 24, 32, 16, 16, 40, 48, 0, 8, 16, 56, 56};
__constant__ unsigned char c_chunk[kChunks + 1] = {0, 24, 48, 68, 88, 108, 128};

// Parameter index of staged product (u, v), or -1 if the product is padding.  A second index
// (b3 and bs share one sum) is returned in *second.
__device__ int arm_grad_index(int u, int v, int* second) {
    *second = -1;
    if (u < 16) {
        if (v < 20) return po::arm_w1 + u * 20 + v;
        if (v == 20) return po::arm_b1 + u;
        return -1;
    }
    if (u < 32) {
        int o = u - 16;
        if (v >= 24 && v < 40) return po::arm_w2 + o * 16 + (v - 24);
        if (v == 20) return po::arm_b2 + o;
        return -1;
    }
    if (u < 34) {
        int o = u - 32;
        if (v >= 40 && v < 56) return po::arm_w3 + o * 16 + (v - 40);
        if (v < 20) return po::arm_ws + o * 20 + v;
        if (v == 20) {
            *second = po::arm_bs + o;
            return po::arm_b3 + o;
        }
        return -1;
    }
    if (u >= 40 && u < 52) {
        int k = (u - 40) >> 2, o = (u - 40) & 3, nin = ifce_nin(k);
        if (v >= 56 && v < 56 + nin) return ifce_w_off(k) + o * nin + (v - 56);
        if (v == 62) return ifce_b_off(k) + o;
        return -1;
    }
    return -1;
}

struct ArmArgs {
    Geom g;
    int64_t N;
    const float* yt;
    const float* params;
    float gscale;       // dLoss / dbits
    float* dS;
    float* dR0;
    float* dR1;
    float* dR2;
    float* dYd;
    float* act;         // [34][N]
    float* gpart;       // [gridDim.x][756]
    double* rate_part;  // [gridDim.x]
};

template <int PASS>
__global__ void __launch_bounds__(kT, 2) k_arm(ArmArgs a) {
    constexpr bool BWD = pass_bwd(PASS);
    extern __shared__ float4 smem4[];
    float* sW = reinterpret_cast<float*>(smem4);
    float* sU = sW + kWSm;
    float* sV = sU + kURows * kLd;
    float* sAcc = sV + kVRows * kLd;
    const Geom& g = a.g;
    const int tid = threadIdx.x;

    for (int j = tid; j < po::arm_block; j += kT) {
        float v = a.params[j];
        int d;
        if (j < po::arm_ws) d = j;                                   // W1 b1 W2 b2 W3 b3->overwritten
        else if (j < po::arm_bs) d = sw_ws + (j - po::arm_ws);
        else if (j < po::if_w0) d = -1;                              // bs folded below
        else d = j;
        if (d >= 0 && j != po::arm_b3 && j != po::arm_b3 + 1) sW[d] = v;
    }
    if (tid < 2) sW[sw_bo + tid] = a.params[po::arm_b3 + tid] + a.params[po::arm_bs + tid];
    if (BWD) {
        for (int j = tid; j < kTasks * 64; j += kT) sAcc[j] = 0.f;
        // constant staging rows
        for (int j = tid; j < kLd; j += kT) {
            for (int r = 34; r < 40; ++r) sU[r * kLd + j] = 0.f;
            for (int r = 52; r < 56; ++r) sU[r * kLd + j] = 0.f;
            sV[20 * kLd + j] = 1.f;
            sV[21 * kLd + j] = 0.f;
            sV[22 * kLd + j] = 0.f;
            sV[23 * kLd + j] = 0.f;
            sV[62 * kLd + j] = 1.f;
            sV[63 * kLd + j] = 0.f;
        }
    }
    __syncthreads();

    const int64_t N = a.N;
    const int64_t n_rounds = (N + kT - 1) / kT;
    float rate_acc = 0.f;

    for (int64_t rd = blockIdx.x; rd < n_rounds; rd += gridDim.x) {
        const int64_t i = rd * kT + tid;
        const bool valid = i < N;
        const int64_t ic = valid ? i : N - 1;
        const int k = grid_of(g, ic);
        const int hk = g.h[k], wk = g.w[k];
        const int li = (int)(ic - g.off[k]);
        const int r = li / wk, c = li - r * wk;
        const float* yk = a.yt + g.off[k];

        float x[kAIn];
#pragma unroll
        for (int n = 0; n < kNCtx; ++n) {
            const int rr = r + ctx_dy(n), cc = c + ctx_dx(n);
            x[n] = (rr >= 0 && cc >= 0 && cc < wk) ? __ldg(yk + rr * wk + cc) : 0.f;
        }
        (void)hk;
        const int nin = ifce_nin(k);
        float rv[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            rv[j] = 0.f;
            if (j < nin) {
                const int gj = k + 1 + j;
                const int rr = min(r >> (j + 1), g.h[gj] - 1), cc = min(c >> (j + 1), g.w[gj] - 1);
                rv[j] = __ldg(a.yt + g.off[gj] + rr * g.w[gj] + cc);
            }
        }
#pragma unroll
        for (int o = 0; o < kF; ++o) {
            float acc = 0.f;
            if (nin > 0) {
                const float* Wf = sW + ifce_w_off(k) + o * nin;
                acc = sW[ifce_b_off(k) + o];
#pragma unroll
                for (int j = 0; j < 6; ++j)
                    if (j < nin) acc = fmaf(Wf[j], rv[j], acc);
            }
            x[kNCtx + o] = acc;
        }

        float a1[kAH], a2[kAH], mu, s;
        if (PASS == PASS_BWD_LOAD) {
#pragma unroll
            for (int o = 0; o < kAH; ++o) {
                a1[o] = a.act[(int64_t)o * N + ic];
                a2[o] = a.act[(int64_t)(16 + o) * N + ic];
            }
            mu = a.act[(int64_t)32 * N + ic];
            s = a.act[(int64_t)33 * N + ic];
        } else {
#pragma unroll
            for (int o = 0; o < kAH; ++o) {
                float acc = sW[sw_b1 + o];
#pragma unroll
                for (int q = 0; q < kAIn; q += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(sW + sw_w1 + o * kAIn + q);
                    acc = fmaf(w.x, x[q], acc);
                    acc = fmaf(w.y, x[q + 1], acc);
                    acc = fmaf(w.z, x[q + 2], acc);
                    acc = fmaf(w.w, x[q + 3], acc);
                }
                a1[o] = acc;
            }
#pragma unroll
            for (int o = 0; o < kAH; ++o) {
                float acc = sW[sw_b2 + o];
#pragma unroll
                for (int q = 0; q < kAH; q += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(sW + sw_w2 + o * kAH + q);
                    acc = fmaf(w.x, fmaxf(a1[q], 0.f), acc);
                    acc = fmaf(w.y, fmaxf(a1[q + 1], 0.f), acc);
                    acc = fmaf(w.z, fmaxf(a1[q + 2], 0.f), acc);
                    acc = fmaf(w.w, fmaxf(a1[q + 3], 0.f), acc);
                }
                a2[o] = acc;
            }
            float out[2];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                float acc = sW[sw_bo + o];
#pragma unroll
                for (int q = 0; q < kAH; q += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(sW + sw_w3 + o * kAH + q);
                    acc = fmaf(w.x, fmaxf(a2[q], 0.f), acc);
                    acc = fmaf(w.y, fmaxf(a2[q + 1], 0.f), acc);
                    acc = fmaf(w.z, fmaxf(a2[q + 2], 0.f), acc);
                    acc = fmaf(w.w, fmaxf(a2[q + 3], 0.f), acc);
                }
#pragma unroll
                for (int q = 0; q < kAIn; q += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(sW + sw_ws + o * kAIn + q);
                    acc = fmaf(w.x, x[q], acc);
                    acc = fmaf(w.y, x[q + 1], acc);
                    acc = fmaf(w.z, x[q + 2], acc);
                    acc = fmaf(w.w, x[q + 3], acc);
                }
                out[o] = acc;
            }
            mu = out[0];
            s = out[1];
            if (PASS == PASS_FWD_STORE && valid) {
#pragma unroll
                for (int o = 0; o < kAH; ++o) {
                    a.act[(int64_t)o * N + i] = a1[o];
                    a.act[(int64_t)(16 + o) * N + i] = a2[o];
                }
                a.act[(int64_t)32 * N + i] = mu;
                a.act[(int64_t)33 * N + i] = s;
            }
        }
        const float logb = fminf(fmaxf(s, kLogbMin), kLogbMax);
        const float yv = __ldg(a.yt + ic);
        const LapOut L = laplace_mass(yv, mu, logb);
        if (valid) rate_acc += -log2f(fmaxf(L.p, kPMin));

        if (BWD) {
            const float dp = (valid && L.p >= kPMin) ? -a.gscale / (L.p * 0.69314718055994531f) : 0.f;
            const float dyd = dp * L.dp_dy;
            const float dmu = -dyd;
            const float ds = (s >= kLogbMin && s <= kLogbMax) ? dp * L.dp_dlogb : 0.f;
            float da2[kAH], da1[kAH], dx[kAIn];
#pragma unroll
            for (int q = 0; q < kAH; ++q) {
                const float d = sW[sw_w3 + q] * dmu + sW[sw_w3 + kAH + q] * ds;
                da2[q] = a2[q] > 0.f ? d : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kAH; ++q) da1[q] = 0.f;
#pragma unroll
            for (int o = 0; o < kAH; ++o) {
#pragma unroll
                for (int q = 0; q < kAH; q += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(sW + sw_w2 + o * kAH + q);
                    da1[q] = fmaf(w.x, da2[o], da1[q]);
                    da1[q + 1] = fmaf(w.y, da2[o], da1[q + 1]);
                    da1[q + 2] = fmaf(w.z, da2[o], da1[q + 2]);
                    da1[q + 3] = fmaf(w.w, da2[o], da1[q + 3]);
                }
            }
#pragma unroll
            for (int q = 0; q < kAH; ++q) da1[q] = a1[q] > 0.f ? da1[q] : 0.f;
#pragma unroll
            for (int q = 0; q < kAIn; q += 4) {
                const float4 w0 = *reinterpret_cast<const float4*>(sW + sw_ws + q);
                const float4 w1 = *reinterpret_cast<const float4*>(sW + sw_ws + kAIn + q);
                dx[q] = w0.x * dmu + w1.x * ds;
                dx[q + 1] = w0.y * dmu + w1.y * ds;
                dx[q + 2] = w0.z * dmu + w1.z * ds;
                dx[q + 3] = w0.w * dmu + w1.w * ds;
            }
#pragma unroll
            for (int o = 0; o < kAH; ++o) {
#pragma unroll
                for (int q = 0; q < kAIn; q += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(sW + sw_w1 + o * kAIn + q);
                    dx[q] = fmaf(w.x, da1[o], dx[q]);
                    dx[q + 1] = fmaf(w.y, da1[o], dx[q + 1]);
                    dx[q + 2] = fmaf(w.z, da1[o], dx[q + 2]);
                    dx[q + 3] = fmaf(w.w, da1[o], dx[q + 3]);
                }
            }
            if (valid) {
#pragma unroll
                for (int n = 0; n < kNCtx; ++n) a.dS[(int64_t)n * N + i] = dx[n];
                a.dYd[i] = dyd;
                if (nin > 0) {
                    float* dR = k == 0 ? a.dR0 : (k == 1 ? a.dR1 : a.dR2);
                    const int nk = hk * wk;
#pragma unroll
                    for (int j = 0; j < 6; ++j)
                        if (j < nin) {
                            float acc = 0.f;
#pragma unroll
                            for (int o = 0; o < kF; ++o) acc = fmaf(sW[ifce_w_off(k) + o * nin + j], dx[kNCtx + o], acc);
                            dR[(int64_t)j * nk + li] = acc;
                        }
                }
            }
            // stage the outer-product factors (zero for padding latents)
            const float m = valid ? 1.f : 0.f;
#pragma unroll
            for (int q = 0; q < kAH; ++q) {
                sU[q * kLd + tid] = da1[q] * m;
                sU[(16 + q) * kLd + tid] = da2[q] * m;
                sV[(24 + q) * kLd + tid] = fmaxf(a1[q], 0.f) * m;
                sV[(40 + q) * kLd + tid] = fmaxf(a2[q], 0.f) * m;
            }
            sU[32 * kLd + tid] = dmu * m;
            sU[33 * kLd + tid] = ds * m;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                for (int o = 0; o < kF; ++o) sU[(40 + 4 * kk + o) * kLd + tid] = (k == kk) ? dx[kNCtx + o] * m : 0.f;
#pragma unroll
            for (int q = 0; q < kAIn; ++q) sV[q * kLd + tid] = x[q] * m;
#pragma unroll
            for (int j = 0; j < 6; ++j) sV[(56 + j) * kLd + tid] = rv[j] * m;
            __syncthreads();
            if (tid < kTasks) {
                const int blk = tid / kChunks, ch = tid - blk * kChunks;
                const float* U = sU + c_blk_u[blk] * kLd;
                const float* V = sV + c_blk_v[blk] * kLd;
                float acc[8][8];
                float* A = sAcc + tid * 64;
#pragma unroll
                for (int p = 0; p < 8; ++p)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[p][q] = A[p * 8 + q];
                for (int l = c_chunk[ch]; l < c_chunk[ch + 1]; l += 4) {
                    float4 u[8], v[8];
#pragma unroll
                    for (int p = 0; p < 8; ++p) u[p] = *reinterpret_cast<const float4*>(U + p * kLd + l);
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = *reinterpret_cast<const float4*>(V + q * kLd + l);
#pragma unroll
                    for (int p = 0; p < 8; ++p)
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            float t = acc[p][q];
                            t = fmaf(u[p].x, v[q].x, t);
                            t = fmaf(u[p].y, v[q].y, t);
                            t = fmaf(u[p].z, v[q].z, t);
                            t = fmaf(u[p].w, v[q].w, t);
                            acc[p][q] = t;
                        }
                }
#pragma unroll
                for (int p = 0; p < 8; ++p)
#pragma unroll
                    for (int q = 0; q < 8; ++q) A[p * 8 + q] = acc[p][q];
            }
            __syncthreads();
        }
    }

    // rate partial of this CTA
    {
        float v[1] = {rate_acc};
        __shared__ float scratch[kT / 32];
        block_sum<1>(v, scratch);
        if (tid == 0) a.rate_part[blockIdx.x] = (double)v[0];
    }
    if (BWD) {
        float* gp = a.gpart + (int64_t)blockIdx.x * po::arm_block;
        for (int e = tid; e < kBlocks * 64; e += kT) {
            const int blk = e >> 6, pq = e & 63;
            const int u = c_blk_u[blk] + (pq >> 3), v = c_blk_v[blk] + (pq & 7);
            int second;
            const int idx = arm_grad_index(u, v, &second);
            if (idx < 0) continue;
            float sum = 0.f;
            for (int ch = 0; ch < kChunks; ++ch) sum += sAcc[(blk * kChunks + ch) * 64 + pq];
            gp[idx] = sum;
            if (second >= 0) gp[second] = sum;
        }
    }
}

}  // namespace

size_t arm_smem_bytes(int pass) {
    if (!pass_bwd(pass)) return (size_t)kWSm * sizeof(float);
    return (size_t)(kWSm + (kURows + kVRows) * kLd + kTasks * 64) * sizeof(float);
}

int arm_grid(int64_t N) {
    const int64_t rounds = (N + kT - 1) / kT;
    const int64_t cap = (int64_t)num_sms() * 2;
    return (int)(rounds < cap ? rounds : cap);
}

void launch_arm(const Work& w, const float* params, int pass, float grad_scale, cudaStream_t s) {
    ArmArgs a;
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
    const size_t sm = arm_smem_bytes(pass);
    const int grid = w.n_cta_arm;
    switch (pass) {
        case PASS_FWD: k_arm<PASS_FWD><<<grid, kT, sm, s>>>(a); break;
        case PASS_FWD_STORE: k_arm<PASS_FWD_STORE><<<grid, kT, sm, s>>>(a); break;
        case PASS_FWD_BWD: k_arm<PASS_FWD_BWD><<<grid, kT, sm, s>>>(a); break;
        default: k_arm<PASS_BWD_LOAD><<<grid, kT, sm, s>>>(a); break;
    }
}

void arm_init_attributes() {
    const int big = (int)arm_smem_bytes(PASS_FWD_BWD);
    cudaFuncSetAttribute(k_arm<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_arm<PASS_BWD_LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace cc
