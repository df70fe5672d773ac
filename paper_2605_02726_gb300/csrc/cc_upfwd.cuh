// Forward upsampling stage body (Sec. III-B, Eq. 7), shared by the per-stage kernel and the
// entropy-model launch, whose first CTA runs the coarse stages.
#pragma once

#include "cc_kernels.h"

namespace cc {
namespace {

// ---------------------------------------------------------------------------------------------
// Upsampling stage s (grid s -> grid s-1), forward, stages 6..2.  Output up[m], m = s-1, holds
// the channels of grids m+1..6: channel 0 comes from y~^(m+1), channel j >= 1 from up[m+1][j-1].
// Separable 4x4 polyphase taps with replicate (clamped) indices, cropped to the grid size.
// ---------------------------------------------------------------------------------------------

// (32-bit indices: a stage has at most 5 channels of half the image, < 2^31 elements)
__device__ __forceinline__ void up_fwd_body(const UpFwdArgs& a, int cta, int ncta) {
    const int plane = a.ht * a.wt, total = a.nch * plane;
    const float tp[4] = {__ldg(a.taps), __ldg(a.taps + 1), __ldg(a.taps + 2), __ldg(a.taps + 3)};
    for (int e = cta * (int)blockDim.x + (int)threadIdx.x; e < total; e += ncta * (int)blockDim.x) {
        const int row = e / a.wt, x = e - row * a.wt;  // row of the stacked channels
        const int j = row / a.ht, y = row - j * a.ht;
        const float* S = j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * a.hs * a.ws;
        const int fy = poly_first(y), fx = poly_first(x);
        float wy[4], wx[4];
        poly_w(y, tp, wy);
        poly_w(x, tp, wx);
        float acc = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float* srow = S + clampi(fy + p, 0, a.hs - 1) * a.ws;
            float rs = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) rs = fmaf(wx[q], __ldg(srow + clampi(fx + q, 0, a.ws - 1)), rs);
            acc = fmaf(wy[p], rs, acc);
        }
        a.dst[e] = acc;
    }
}

// A whole forward stage in one CTA (the coarse stages): the input channels are staged in shared
// memory `sm` (capacity `cap` floats) by asynchronous copies when they fit, else read from global
// memory (the previous stage wrote them in the same CTA); warps take output rows, lanes x, and a
// lane computes four outputs of its row at once (x, x + 32, x + 64, x + 96), so that one warp per
// SM sub-partition still has independent chains to interleave.  The arithmetic is the
// per-element expression of up_fwd_body, so the values are the same bits.  Ends with a barrier:
// dst is then visible to the whole CTA and `sm` free.
__device__ __forceinline__ void up_fwd_stage_cta(const UpFwdArgs& a, float* sm, int cap) {
    const float tp[4] = {a.taps[0], a.taps[1], a.taps[2], a.taps[3]};
    const int nin = a.hs * a.ws;
    const bool staged = a.nch * nin <= cap;
    if (staged) {
        for (int j = 0; j < a.nch; ++j) {
            const float* src = j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * nin;
            for (int e = threadIdx.x; e < nin; e += blockDim.x) cp_async4(sm + j * nin + e, src + e);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int row = threadIdx.x >> 5; row < a.nch * a.ht; row += nwarps) {
        const int j = row / a.ht, y = row - j * a.ht;
        const float* S = staged ? sm + j * nin : (j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * nin);
        const int fy = poly_first(y);
        float wy[4];
        poly_w(y, tp, wy);
        const float* r[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) r[p] = S + clampi(fy + p, 0, a.hs - 1) * a.ws;
        float* drow = a.dst + ((int64_t)j * a.ht + y) * a.wt;
        for (int x0 = lane; x0 < a.wt; x0 += 128) {
            float acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int x = x0 + 32 * u < a.wt ? x0 + 32 * u : x0;  // (out-of-row lanes recompute x0)
                const int fx = poly_first(x);
                float wx[4];
                poly_w(x, tp, wx);
                acc[u] = 0.f;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float rs = 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) rs = fmaf(wx[q], r[p][clampi(fx + q, 0, a.ws - 1)], rs);
                    acc[u] = fmaf(wy[p], rs, acc[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (x0 + 32 * u < a.wt) drow[x0 + 32 * u] = acc[u];
        }
    }
    __syncthreads();
}
}  // namespace
}  // namespace cc
