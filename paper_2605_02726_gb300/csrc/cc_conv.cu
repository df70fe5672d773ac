// Residual 3x3 convolutions of the synthesis (Sec. III-B, Table II: two 3 -> 3 post-filters),
// the distortion (Eq. 10) and their adjoint, on 16x32 pixel tiles with recomputed halos.
//   x1 = t + b1 + conv1(t),  xh = x1 + b2 + conv2(x1)   (replicate padding, cross-correlation)
//   D = mean (xh - x)^2;  dxh = 2 (xh - x) / (3HW);  dx1 = dxh + conv2^T(dxh);  dt = dx1 + conv1^T(dx1)
// Shared-memory tiles of t and x1 are replicate-padded (positions outside the image hold the
// clamped value), so the forward stencils and the weight-gradient correlations need no clamps.
// The transposed convolutions gather, per axis, the 3 (source, tap) pairs whose clamped index
// lands on the target: interior q <- (q+1, 0), (q, 1), (q-1, 2); q = 0 <- (0,0), (0,1), (1,0);
// q = n-1 <- (n-1,1), (n-1,2), (n-2,2); n = 1 <- (0,0), (0,1), (0,2).
#include "cc_kernels.h"

namespace cc {
namespace {

constexpr int kTH = kConvTH, kTW = kConvTW;
constexpr int kThreads = 256;
constexpr int R4H = kTH + 8, R4W = kTW + 8;  // t   (halo 4)
constexpr int R3H = kTH + 6, R3W = kTW + 6;  // x1  (halo 3)
constexpr int R2H = kTH + 4, R2W = kTW + 4;  // dxh (halo 2)
constexpr int R1H = kTH + 2, R1W = kTW + 2;  // dx1 (halo 1)
constexpr int kSlices = 8;                   // weight-gradient row slices of 2 rows


__device__ __forceinline__ void conv_pairs(int q, int n, int (&src)[3], int (&tap)[3]) {
    if (n == 1) {
        src[0] = 0; tap[0] = 0; src[1] = 0; tap[1] = 1; src[2] = 0; tap[2] = 2;
    } else if (q == 0) {
        src[0] = 0; tap[0] = 0; src[1] = 0; tap[1] = 1; src[2] = 1; tap[2] = 0;
    } else if (q == n - 1) {
        src[0] = n - 1; tap[0] = 1; src[1] = n - 1; tap[1] = 2; src[2] = n - 2; tap[2] = 2;
    } else {
        src[0] = q + 1; tap[0] = 0; src[1] = q; tap[1] = 1; src[2] = q - 1; tap[2] = 2;
    }
}

template <int PASS>
__device__ __forceinline__ void conv_body(const ConvArgs& a, int cta, int ncta) {
    constexpr bool BWD = pass_bwd(PASS);
    __shared__ float sWc[2][84];
    __shared__ float sT[3][R4H][R4W];
    __shared__ float sX1[3][R3H][R3W];
    __shared__ float sD[3][R2H][R2W];
    __shared__ float sD1[3][R1H][R1W];
    __shared__ double sSe[kThreads / 32];
    const int tid = threadIdx.x;
    for (int j = tid; j < 84; j += kThreads) {
        sWc[0][j] = j < 81 ? a.params[po::cv1_w + j] : a.params[po::cv1_b + j - 81];
        sWc[1][j] = j < 81 ? a.params[po::cv2_w + j] : a.params[po::cv2_b + j - 81];
    }
    // weight-gradient task: tid < 144 -> (conv c, out o, in i, slice); 144 <= tid < 192 -> bias (c, o, slice)
    float gacc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) gacc[q] = 0.f;
    double se = 0.0;
    const int H = a.H, W = a.W;
    for (int tile = cta; tile < a.n_tiles; tile += ncta) {
        const int ty0 = (tile / a.tiles_x) * kTH, tx0 = (tile % a.tiles_x) * kTW;
        __syncthreads();
        {
            // the t tile (clamped reads, i.e. replicate-padded) and the image on the halo-2 region
            // (into sD, replaced by dxh below) arrive by asynchronous copies in flight together
            constexpr int NT = 3 * R4H * R4W, NI = 3 * R2H * R2W;
            for (int e = tid; e < NT; e += kThreads) {
                const int c = e / (R4H * R4W), rem = e - c * (R4H * R4W);
                const int ry = rem / R4W, rx = rem - ry * R4W;
                const int gy = clampi(ty0 - 4 + ry, 0, H - 1), gx = clampi(tx0 - 4 + rx, 0, W - 1);
                cp_async4(&sT[c][ry][rx], a.t + (int64_t)c * a.HW + (int64_t)gy * W + gx);
            }
            for (int e = tid; e < NI; e += kThreads) {
                const int c = e / (R2H * R2W), rem = e - c * (R2H * R2W);
                const int ry = rem / R2W, rx = rem - ry * R2W;
                const int gy = clampi(ty0 - 2 + ry, 0, H - 1), gx = clampi(tx0 - 2 + rx, 0, W - 1);
                cp_async4(&sD[c][ry][rx], a.img + (int64_t)c * a.HW + (int64_t)gy * W + gx);
            }
            cp_async_wait_all();
        }
        __syncthreads();
        // x1 at the real positions of the halo-3 region
        for (int e = tid; e < R3H * R3W; e += kThreads) {
            const int ry = e / R3W, rx = e - ry * R3W;
            const int gy = ty0 - 3 + ry, gx = tx0 - 3 + rx;
            if (gy < 0 || gy >= H || gx < 0 || gx >= W) continue;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                float acc = sT[o][ry + 1][rx + 1] + sWc[0][81 + o];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
                            acc = fmaf(sWc[0][((o * 3 + i) * 3 + ky) * 3 + kx], sT[i][ry + ky][rx + kx], acc);
                sX1[o][ry][rx] = acc;
            }
        }
        __syncthreads();
        // replicate-pad x1 outside the image
        for (int e = tid; e < R3H * R3W; e += kThreads) {
            const int ry = e / R3W, rx = e - ry * R3W;
            const int gy = ty0 - 3 + ry, gx = tx0 - 3 + rx;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) continue;
            const int sy = clampi(gy, 0, H - 1) - (ty0 - 3), sx = clampi(gx, 0, W - 1) - (tx0 - 3);
#pragma unroll
            for (int o = 0; o < 3; ++o) sX1[o][ry][rx] = sX1[o][sy][sx];
        }
        __syncthreads();
        // xh, distortion and dxh at the real positions of the halo-2 region
        for (int e = tid; e < R2H * R2W; e += kThreads) {
            const int ry = e / R2W, rx = e - ry * R2W;
            const int gy = ty0 - 2 + ry, gx = tx0 - 2 + rx;
            if (gy < 0 || gy >= H || gx < 0 || gx >= W) continue;
            const bool core = ry >= 2 && ry < 2 + kTH && rx >= 2 && rx < 2 + kTW;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                float acc = sX1[o][ry + 1][rx + 1] + sWc[1][81 + o];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
                            acc = fmaf(sWc[1][((o * 3 + i) * 3 + ky) * 3 + kx], sX1[i][ry + ky][rx + kx], acc);
                const int64_t gi = (int64_t)o * a.HW + (int64_t)gy * W + gx;
                const float diff = acc - sD[o][ry][rx];
                if (core) {
                    se += (double)diff * diff;
                    if (a.xhat) a.xhat[gi] = acc;
                }
                sD[o][ry][rx] = diff * a.gscale;
            }
        }
        if (!BWD) continue;
        __syncthreads();
        // dx1 = dxh + conv2^T(dxh) at the real positions of the halo-1 region
        for (int e = tid; e < R1H * R1W; e += kThreads) {
            const int ry = e / R1W, rx = e - ry * R1W;
            const int gy = ty0 - 1 + ry, gx = tx0 - 1 + rx;
            if (gy < 0 || gy >= H || gx < 0 || gx >= W) continue;
            int sy[3], ky[3], sx[3], kx[3];
            conv_pairs(gy, H, sy, ky);
            conv_pairs(gx, W, sx, kx);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                sy[p] -= ty0 - 2;
                sx[p] -= tx0 - 2;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float acc = sD[i][ry + 1][rx + 1];
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int o = 0; o < 3; ++o)
                            acc = fmaf(sWc[1][((o * 3 + i) * 3 + ky[p]) * 3 + kx[q]], sD[o][sy[p]][sx[q]], acc);
                sD1[i][ry][rx] = acc;
            }
        }
        __syncthreads();
        // dt = dx1 + conv1^T(dx1) on the core
        for (int e = tid; e < kTH * kTW; e += kThreads) {
            const int ry = e / kTW, rx = e - ry * kTW;
            const int gy = ty0 + ry, gx = tx0 + rx;
            if (gy >= H || gx >= W) continue;
            int sy[3], ky[3], sx[3], kx[3];
            conv_pairs(gy, H, sy, ky);
            conv_pairs(gx, W, sx, kx);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                sy[p] -= ty0 - 1;
                sx[p] -= tx0 - 1;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float acc = sD1[i][ry + 1][rx + 1];
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int o = 0; o < 3; ++o)
                            acc = fmaf(sWc[0][((o * 3 + i) * 3 + ky[p]) * 3 + kx[q]], sD1[o][sy[p]][sx[q]], acc);
                a.dt[(int64_t)i * a.HW + (int64_t)gy * W + gx] = acc;
            }
        }
        // parameter gradients over the core (no shared-memory writes above since the last barrier)
        const int ry_end = min(kTH, H - ty0), rx_end = min(kTW, W - tx0);
        if (tid < 144) {
            const int slice = tid & 7, task = tid >> 3;  // task 0..17
            const int c = task / 9, o = (task / 3) % 3, i = task % 3;
            for (int ry = 2 * slice; ry < min(2 * slice + 2, ry_end); ++ry) {
                for (int rx = 0; rx < rx_end; ++rx) {
                    if (c == 1) {  // conv2: dxh (origin ty0-2) x padded x1 (origin ty0-3)
                        const float gv = sD[o][ry + 2][rx + 2];
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx) gacc[ky * 3 + kx] = fmaf(gv, sX1[i][ry + 2 + ky][rx + 2 + kx], gacc[ky * 3 + kx]);
                    } else {       // conv1: dx1 (origin ty0-1) x padded t (origin ty0-4)
                        const float gv = sD1[o][ry + 1][rx + 1];
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx) gacc[ky * 3 + kx] = fmaf(gv, sT[i][ry + 3 + ky][rx + 3 + kx], gacc[ky * 3 + kx]);
                    }
                }
            }
        } else if (tid < 192) {
            const int slice = tid & 7, task = (tid - 144) >> 3;  // 0..5
            const int c = task / 3, o = task % 3;
            for (int ry = 2 * slice; ry < min(2 * slice + 2, ry_end); ++ry)
                for (int rx = 0; rx < rx_end; ++rx) gacc[0] += c == 1 ? sD[o][ry + 2][rx + 2] : sD1[o][ry + 1][rx + 1];
        }
    }
    __syncthreads();
    {
        double v = warp_sum_d(se);
        if ((tid & 31) == 0) sSe[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < kThreads / 32; ++q) s += sSe[q];
            a.se_part[cta] = s;
        }
    }
    if (!BWD) return;
    // reduce the row slices of each task in a fixed order; the x1 tile is free now
    float* sG = &sX1[0][0][0];  // [192][9]
#pragma unroll
    for (int q = 0; q < 9; ++q)
        if (tid < 192) sG[tid * 9 + q] = gacc[q];
    __syncthreads();
    float* gp = a.gpart + (int64_t)cta * po::conv_block;
    if (tid < 18 * 9) {
        const int task = tid / 9, q = tid % 9;
        const int c = task / 9, o = (task / 3) % 3, i = task % 3;
        float s = 0.f;
        for (int sl = 0; sl < kSlices; ++sl) s += sG[(task * 8 + sl) * 9 + q];
        gp[(c == 0 ? 0 : 84) + (o * 3 + i) * 9 + q] = s;
    } else if (tid < 18 * 9 + 6) {
        const int task = tid - 162, c = task / 3, o = task % 3;
        float s = 0.f;
        for (int sl = 0; sl < kSlices; ++sl) s += sG[(144 + task * 8 + sl) * 9];
        gp[(c == 0 ? 81 : 165) + o] = s;
    }
}

template <int PASS>
__global__ void __launch_bounds__(kThreads, 2) k_conv(ConvArgs a) {
    __shared__ ConvArgs sa;
    param_fetch(a, sa);
    conv_body<PASS>(sa, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kThreads, 2) k_conv_b(Batch<ConvArgs> b) {
    __shared__ ConvArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    conv_body<PASS>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

}  // namespace

int conv_tiles(int H, int W) { return ((H + kTH - 1) / kTH) * ((W + kTW - 1) / kTW); }

ConvArgs conv_args(const Work& w, const float* params, const float* image, float grad_scale, float* xhat_out) {
    ConvArgs a;
    a.pad_ = 0;
    a.H = w.g.H;
    a.W = w.g.W;
    a.HW = w.HW;
    a.t = w.t;
    a.img = image;
    a.params = params;
    a.gscale = grad_scale;
    a.dt = w.dt;
    a.xhat = xhat_out;
    a.gpart = w.gpart_conv;
    a.se_part = w.se_part;
    a.tiles_x = (w.g.W + kTW - 1) / kTW;
    a.n_tiles = conv_tiles(w.g.H, w.g.W);
    return a;
}

void launch_conv(const Work& w, const float* params, const float* image, int pass, float grad_scale,
                 float* xhat_out, cudaStream_t s) {
    const ConvArgs a = conv_args(w, params, image, grad_scale, xhat_out);
    if (pass_bwd(pass))
        k_conv<PASS_FWD_BWD><<<w.n_cta_conv, kThreads, 0, s>>>(a);
    else
        k_conv<PASS_FWD><<<w.n_cta_conv, kThreads, 0, s>>>(a);
}

void launch_conv_b(const Batch<ConvArgs>& b, cudaStream_t s) { k_conv_b<PASS_FWD_BWD><<<b.total_ctas, kThreads, 0, s>>>(b); }

}  // namespace cc
