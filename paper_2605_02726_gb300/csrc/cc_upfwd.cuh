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
// memory `sm` (capacity `cap` floats) when they fit, else read from global memory with coherent
// loads (the previous stage wrote them in the same kernel); warps take output rows, lanes x.  The
// arithmetic is the per-element expression of up_fwd_body, so the values are the same bits.  Ends
// with a barrier: dst is then visible to the whole CTA and `sm` free.
__device__ __forceinline__ void up_fwd_stage_cta(const UpFwdArgs& a, float* sm, int cap) {
    const float tp[4] = {a.taps[0], a.taps[1], a.taps[2], a.taps[3]};
    const int nin = a.hs * a.ws;
    const bool staged = a.nch * nin <= cap;
    if (staged) {
        for (int j = 0; j < a.nch; ++j) {
            const float* src = j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * nin;
            for (int e = threadIdx.x; e < nin; e += blockDim.x) sm[j * nin + e] = src[e];
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int row = threadIdx.x >> 5; row < a.nch * a.ht; row += nwarps) {
        const int j = row / a.ht, y = row - j * a.ht;
        const float* S = staged ? sm + j * nin : (j == 0 ? a.src0 : a.srcup + (int64_t)(j - 1) * nin);
        const int fy = poly_first(y);
        float wy[4];
        poly_w(y, tp, wy);
        float* drow = a.dst + ((int64_t)j * a.ht + y) * a.wt;
        for (int x = lane; x < a.wt; x += 32) {
            const int fx = poly_first(x);
            float wx[4];
            poly_w(x, tp, wx);
            float acc = 0.f;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float* r = S + clampi(fy + p, 0, a.hs - 1) * a.ws;
                float rs = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) rs = fmaf(wx[q], r[clampi(fx + q, 0, a.ws - 1)], rs);
                acc = fmaf(wy[p], rs, acc);
            }
            drow[x] = acc;
        }
    }
    __syncthreads();
}
}  // namespace
}  // namespace cc
