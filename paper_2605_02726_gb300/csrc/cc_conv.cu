// Residual 3x3 convolutions of the synthesis (Sec. III-B, Table II: two 3 -> 3 post-filters),
// the distortion (Eq. 10) and their adjoint, on 22x32 pixel tiles with recomputed halos.
//   x1 = t + b1 + conv1(t),  xh = x1 + b2 + conv2(x1)   (replicate padding, cross-correlation)
//   D = mean (xh - x)^2;  dxh = 2 (xh - x) / (3HW);  dx1 = dxh + conv2^T(dxh);  dt = dx1 + conv1^T(dx1)
//
// All tiles of a CTA live in one frame of 30 x 40 cells whose origin is (ty0 - 4, tx0 - 4): t on
// the whole frame (halo 4), x1 on halo 3, the image and then dxh on halo 2, dx1 on halo 1, dt on
// the core.  Tiles of t and x1 are replicate-padded (cells outside the image hold the clamped
// value), so the forward stencils and the weight-gradient correlations need no clamps.
//
// Each thread computes a vertical strip of 2 cells at one column, all 3 channels, from a 4 x 3
// register window per input channel (162 FMAs per 36 shared loads and 27 broadcast weight loads);
// lanes take consecutive columns, so the loads are free of bank conflicts.  The transposed
// convolutions are plain correlations with the flipped kernel inside the image; cells on the image
// border gather, per axis, the 3 (source, tap) pairs whose clamped index lands on the target:
// interior q <- (q+1, 0), (q, 1), (q-1, 2); q = 0 <- (0,0), (0,1), (1,0);
// q = n-1 <- (n-1,1), (n-1,2), (n-2,2); n = 1 <- (0,0), (0,1), (0,2).
// Weight gradients: warp w owns the (conv, out, in) tasks w, w + 8, w + 16 with 9 + 1 accumulators
// each, lane = core column, a sliding 3-row window down the core; summed over the lanes at the end.
#include "cc_kernels.h"

namespace cc {
namespace {

// Core 22 x 32: at 512x768 that is 576 tiles, at most two per CTA at two CTAs per SM (16 x 32 tiles
// gave 768, three rounds for 160 CTAs and two for the rest), and 12% fewer stencil cells per CTA
// for the halos recomputed.  The four frame buffers (52 KB) are in dynamic shared memory.
constexpr int kTH = kConvTH, kTW = kConvTW;
constexpr int kThreads = 256;
constexpr int SW = kTW + 8;               // 40 frame columns
constexpr int T_R0 = 0, T_NR = kTH + 8;  // frame rows held by each buffer: t 0..kTH+7
constexpr int X_R0 = 1, X_NR = kTH + 6;  // x1 1..kTH+6
constexpr int D_R0 = 2, D_NR = kTH + 4;  // image / dxh 2..kTH+5
constexpr int E_R0 = 3, E_NR = kTH + 2;  // dx1 3..kTH+4
constexpr int kFrameFloats = 3 * (T_NR + X_NR + D_NR + E_NR) * SW;
static_assert(kTH % 2 == 0, "two-row strips");
constexpr int kTasks = 18;               // (conv, out, in) weight-gradient tasks

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

struct ConvW {
    float4 f[2][27];  // forward:    f[c][(i*3+ky)*3+kx] = (W[0][i][ky][kx], W[1][..], W[2][..], 0)
    float4 t[2][27];  // transposed: t[c][(o*3+ky)*3+kx] = (W[o][0][ky][kx], W[o][1][..], W[o][2][..], 0)
    float b[2][4];
};

// x_out = x_in + b + conv(x_in) at frame rows (ir, ir + 1) of IN (buffer rows), column c.
template <int NR>
__device__ __forceinline__ void fwd_strip(const float (*IN)[NR][SW], int ir, int c, const float4* wf,
                                          const float* b, float (&acc)[3][2]) {
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[o][j] = IN[o][ir + j][c] + b[o];
#pragma unroll 1
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            float v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = IN[i][ir - 1 + m][c - 1 + kx];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const float4 w = wf[(i * 3 + ky) * 3 + kx];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    acc[0][j] = fmaf(w.x, v[j + ky], acc[0][j]);
                    acc[1][j] = fmaf(w.y, v[j + ky], acc[1][j]);
                    acc[2][j] = fmaf(w.z, v[j + ky], acc[2][j]);
                }
            }
        }
}

// d_out = d_in + conv^T(d_in) at buffer rows (sr, sr + 1) of S, column c, all sources inside the
// image: source (y + 1 - ky, x + 1 - kx) with tap (ky, kx).
template <int NR>
__device__ __forceinline__ void adj_strip(const float (*S)[NR][SW], int sr, int c, const float4* wt, float (&acc)[3][2]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = S[i][sr + j][c];
#pragma unroll 1
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            float v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = S[o][sr - 1 + m][c + 1 - kx];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const float4 w = wt[(o * 3 + ky) * 3 + kx];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    acc[0][j] = fmaf(w.x, v[j + 2 - ky], acc[0][j]);
                    acc[1][j] = fmaf(w.y, v[j + 2 - ky], acc[1][j]);
                    acc[2][j] = fmaf(w.z, v[j + 2 - ky], acc[2][j]);
                }
            }
        }
}

// the same at one cell (global gy, gx; buffer row sr, column c) on or next to the image border
template <int NR>
__device__ __forceinline__ void adj_cell_border(const float (*S)[NR][SW], int sr, int c, int gy, int gx, int H,
                                                int W, const float4* wt, float (&out)[3]) {
    int sy[3], ky[3], sx[3], kx[3];
    conv_pairs(gy, H, sy, ky);
    conv_pairs(gx, W, sx, kx);
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = S[i][sr][c];
#pragma unroll 1
    for (int p = 0; p < 3; ++p) {
        // row pair p without a dynamically indexed array
        const int syp = p == 0 ? sy[0] : (p == 1 ? sy[1] : sy[2]);
        const int kyp = p == 0 ? ky[0] : (p == 1 ? ky[1] : ky[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int br = sr + syp - gy, bc = c + sx[q] - gx;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                const float4 w = wt[(o * 3 + kyp) * 3 + kx[q]];
                const float v = S[o][br][bc];
                out[0] = fmaf(w.x, v, out[0]);
                out[1] = fmaf(w.y, v, out[1]);
                out[2] = fmaf(w.z, v, out[2]);
            }
        }
    }
}

template <int PASS>
__device__ __forceinline__ void conv_body(const ConvArgs& a, int cta, int ncta) {
    constexpr bool BWD = pass_bwd(PASS);
    __shared__ ConvW sW;
    extern __shared__ __align__(16) float sFrame[];  // kFrameFloats
    float (*sT)[T_NR][SW] = reinterpret_cast<float (*)[T_NR][SW]>(sFrame);
    float (*sX)[X_NR][SW] = reinterpret_cast<float (*)[X_NR][SW]>(sFrame + 3 * T_NR * SW);
    float (*sD)[D_NR][SW] = reinterpret_cast<float (*)[D_NR][SW]>(sFrame + 3 * (T_NR + X_NR) * SW);
    float (*sE)[E_NR][SW] = reinterpret_cast<float (*)[E_NR][SW]>(sFrame + 3 * (T_NR + X_NR + D_NR) * SW);
    __shared__ double sSe[kThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int j = tid; j < 2 * 81; j += kThreads) {
        const int c = j / 81, e = j - c * 81;  // e = ((o*3+i)*3+ky)*3+kx
        const int o = e / 27, i = (e / 9) % 3, k = e % 9;
        const float w = a.params[(c ? po::cv2_w : po::cv1_w) + e];
        reinterpret_cast<float*>(&sW.f[c][i * 9 + k])[o] = w;
        reinterpret_cast<float*>(&sW.t[c][o * 9 + k])[i] = w;
    }
    if (tid < 2 * 27) {
        const int c = tid / 27, k = tid % 27;
        sW.f[c][k].w = 0.f;
        sW.t[c][k].w = 0.f;
    }
    if (tid < 8) {
        const int c = tid >> 2, o = tid & 3;
        sW.b[c][o] = o < 3 ? a.params[(c ? po::cv2_b : po::cv1_b) + o] : 0.f;
    }
    float gacc[3][9], bacc[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        bacc[s] = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q) gacc[s][q] = 0.f;
    }
    double se = 0.0;
    const int H = a.H, W = a.W;
    for (int tile = cta; tile < a.n_tiles; tile += ncta) {
        const int ty0 = (tile / a.tiles_x) * kTH, tx0 = (tile % a.tiles_x) * kTW;
        const int fy0 = ty0 - 4, fx0 = tx0 - 4;  // global coordinates of frame cell (0, 0)
        __syncthreads();
        {
            // t on the whole frame and the image on halo 2, clamped (replicate) reads in flight together
            for (int e = tid; e < 3 * T_NR * SW; e += kThreads) {
                const int c = e / (T_NR * SW), rem = e - c * (T_NR * SW);
                const int r = rem / SW, x = rem - r * SW;
                const int gy = clampi(fy0 + r, 0, H - 1), gx = clampi(fx0 + x, 0, W - 1);
                cp_async4(&sT[c][r][x], a.t + (int64_t)c * a.HW + (int64_t)gy * W + gx);
            }
            constexpr int DW = kTW + 4;
            for (int e = tid; e < 3 * D_NR * DW; e += kThreads) {
                const int c = e / (D_NR * DW), rem = e - c * (D_NR * DW);
                const int r = rem / DW, x = 2 + (rem - r * DW);
                const int gy = clampi(fy0 + D_R0 + r, 0, H - 1), gx = clampi(fx0 + x, 0, W - 1);
                cp_async4(&sD[c][r][x], a.img + (int64_t)c * a.HW + (int64_t)gy * W + gx);
            }
            cp_async_wait_all();
        }
        __syncthreads();
        // x1 on halo 3: frame rows 1..kTH+6, columns 1..kTW+6
        {
            constexpr int NC = kTW + 6, NT = (X_NR / 2) * NC;
            for (int task = tid; task < NT; task += kThreads) {
                const int rb = task / NC, c = 1 + (task - rb * NC), fr = X_R0 + 2 * rb;
                float acc[3][2];
                fwd_strip<T_NR>(sT, fr - T_R0, c, sW.f[0], sW.b[0], acc);
#pragma unroll
                for (int o = 0; o < 3; ++o)
#pragma unroll
                    for (int j = 0; j < 2; ++j) sX[o][fr - X_R0 + j][c] = acc[o][j];
            }
        }
        __syncthreads();
        if (fy0 + X_R0 < 0 || fx0 + 1 < 0 || fy0 + X_R0 + X_NR > H || fx0 + 1 + kTW + 6 > W) {
            // replicate-pad x1 outside the image (tiles on the image border)
            constexpr int NC = kTW + 6;
            for (int e = tid; e < X_NR * NC; e += kThreads) {
                const int r = e / NC, c = 1 + (e - r * NC);
                const int gy = fy0 + X_R0 + r, gx = fx0 + c;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) continue;
                const int sr = clampi(gy, 0, H - 1) - fy0 - X_R0, sc = clampi(gx, 0, W - 1) - fx0;
#pragma unroll
                for (int o = 0; o < 3; ++o) sX[o][r][c] = sX[o][sr][sc];
            }
            __syncthreads();
        }
        // xh, distortion and dxh on halo 2: frame rows 2..kTH+5, columns 2..kTW+5
        {
            constexpr int NC = kTW + 4, NT = (D_NR / 2) * NC;
            float sef = 0.f;
            for (int task = tid; task < NT; task += kThreads) {
                const int rb = task / NC, c = 2 + (task - rb * NC), fr = D_R0 + 2 * rb;
                float acc[3][2];
                fwd_strip<X_NR>(sX, fr - X_R0, c, sW.f[1], sW.b[1], acc);
                const int gx = fx0 + c;
                const bool core_x = c >= 4 && c < 4 + kTW && gx < W;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int gy = fy0 + fr + j;
                    const bool core = core_x && fr + j >= 4 && fr + j < 4 + kTH && gy < H;
#pragma unroll
                    for (int o = 0; o < 3; ++o) {
                        float& cell = sD[o][fr - D_R0 + j][c];
                        const float diff = acc[o][j] - cell;
                        if (core) {
                            sef = fmaf(diff, diff, sef);
                            if (a.xhat) a.xhat[(int64_t)o * a.HW + (int64_t)gy * W + gx] = acc[o][j];
                        }
                        cell = diff * a.gscale;
                    }
                }
            }
            se += (double)sef;
        }
        if (!BWD) continue;
        __syncthreads();
        // dx1 = dxh + conv2^T(dxh) on halo 1: frame rows 3..kTH+4, columns 3..kTW+4
        {
            constexpr int NC = kTW + 2, NT = (E_NR / 2) * NC;
            for (int task = tid; task < NT; task += kThreads) {
                const int rb = task / NC, c = 3 + (task - rb * NC), fr = E_R0 + 2 * rb;
                const int gy = fy0 + fr, gx = fx0 + c;
                float acc[3][2];
                if (gy >= 1 && gy + 1 <= H - 2 && gx >= 1 && gx <= W - 2) {
                    adj_strip<D_NR>(sD, fr - D_R0, c, sW.t[1], acc);
                } else {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        float out[3] = {0.f, 0.f, 0.f};
                        if (gy + j >= 0 && gy + j < H && gx >= 0 && gx < W)
                            adj_cell_border<D_NR>(sD, fr - D_R0 + j, c, gy + j, gx, H, W, sW.t[1], out);
#pragma unroll
                        for (int i = 0; i < 3; ++i) acc[i][j] = out[i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) sE[i][fr - E_R0 + j][c] = acc[i][j];
            }
        }
        __syncthreads();
        // dt = dx1 + conv1^T(dx1) on the core: frame rows 4..kTH+3, columns 4..kTW+3
        {
            constexpr int NC = kTW, NT = (kTH / 2) * NC;
            for (int task = tid; task < NT; task += kThreads) {
                const int rb = task / NC, c = 4 + (task - rb * NC), fr = 4 + 2 * rb;
                const int gy = fy0 + fr, gx = fx0 + c;
                if (gx >= W || gy >= H) continue;
                float acc[3][2];
                if (gy >= 1 && gy + 1 <= H - 2 && gx >= 1 && gx <= W - 2) {
                    adj_strip<E_NR>(sE, fr - E_R0, c, sW.t[0], acc);
                } else {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        float out[3] = {0.f, 0.f, 0.f};
                        if (gy + j < H) adj_cell_border<E_NR>(sE, fr - E_R0 + j, c, gy + j, gx, H, W, sW.t[0], out);
#pragma unroll
                        for (int i = 0; i < 3; ++i) acc[i][j] = out[i];
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (gy + j < H)
#pragma unroll
                        for (int i = 0; i < 3; ++i) a.dt[(int64_t)i * a.HW + (int64_t)(gy + j) * W + gx] = acc[i][j];
            }
        }
        // parameter gradients over the core (the buffers read here are not written since the last barrier)
        {
            const int c = 4 + lane;
            const bool colok = tx0 + lane < W;
            const int ny = min(kTH, H - ty0);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int task = wid + 8 * s;
                if (task >= kTasks) break;
                const int cv = task / 9, o = (task / 3) % 3, i = task % 3;
                // G row y = core row y; IN row y = core row y (rows -1 .. kTH valid)
                const float* G = cv ? &sD[o][4 - D_R0][0] : &sE[o][4 - E_R0][0];
                const float* IN = cv ? &sX[i][4 - X_R0][0] : &sT[i][4 - T_R0][0];
                float w0[3], w1[3];
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    w0[kx] = IN[-SW + c - 1 + kx];
                    w1[kx] = IN[c - 1 + kx];
                }
#pragma unroll
                for (int y = 0; y < kTH; ++y) {
                    float w2[3];
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) w2[kx] = IN[(y + 1) * SW + c - 1 + kx];
                    const float g = (colok && y < ny) ? G[y * SW + c] : 0.f;
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        gacc[s][kx] = fmaf(g, w0[kx], gacc[s][kx]);
                        gacc[s][3 + kx] = fmaf(g, w1[kx], gacc[s][3 + kx]);
                        gacc[s][6 + kx] = fmaf(g, w2[kx], gacc[s][6 + kx]);
                    }
                    bacc[s] += g;
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        w0[kx] = w1[kx];
                        w1[kx] = w2[kx];
                    }
                }
            }
        }
    }
    __syncthreads();
    {
        double v = warp_sum_d(se);
        if (lane == 0) sSe[wid] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < kThreads / 32; ++q) s += sSe[q];
            a.se_part[cta] = s;
        }
    }
    if (!BWD) return;
    float* gp = a.gpart + (int64_t)cta * po::conv_block;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int task = wid + 8 * s;
        if (task >= kTasks) break;
        const int cv = task / 9, o = (task / 3) % 3, i = task % 3;
        const int base = cv ? po::cv2_w - po::cv1_w : 0;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float v = warp_sum(gacc[s][q]);
            if (lane == 0) gp[base + (o * 3 + i) * 9 + q] = v;
        }
        const float bv = warp_sum(bacc[s]);
        if (lane == 0 && i == 0) gp[base + 81 + o] = bv;
    }
}

template <int PASS>
__global__ void __launch_bounds__(kThreads, 2) k_conv(const __grid_constant__ ConvArgs a) {
    pdl_enter();
    conv_body<PASS>(a, blockIdx.x, gridDim.x);
}
template <int PASS>
__global__ void __launch_bounds__(kThreads, 2) k_conv_b(Batch<ConvArgs> b) {
    __shared__ ConvArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    conv_body<PASS>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

}  // namespace

void conv_init_attributes() {
    const int sm = kFrameFloats * (int)sizeof(float);
    cudaFuncSetAttribute(k_conv<PASS_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_conv<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_conv_b<PASS_FWD_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

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
    constexpr size_t sm = kFrameFloats * sizeof(float);
    if (pass_bwd(pass))
        launch_pdl(k_conv<PASS_FWD_BWD>, w.n_cta_conv, kThreads, sm, s, a);
    else
        launch_pdl(k_conv<PASS_FWD>, w.n_cta_conv, kThreads, sm, s, a);
}

void launch_conv_b(const Batch<ConvArgs>& b, cudaStream_t s) {
    launch_pdl(k_conv_b<PASS_FWD_BWD>, b.total_ctas, kThreads, kFrameFloats * sizeof(float), s, b);
}

}  // namespace cc
