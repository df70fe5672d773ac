// Host-side launch wrappers of the encoder-step kernels (internal to the library).
#pragma once

#include "cc_common.cuh"

namespace cc {

enum Pass : int {
    PASS_FWD = 0,        // forward only (rate, reconstruction, distortion)
    PASS_FWD_STORE = 1,  // forward, keep the activations the adjoint needs
    PASS_FWD_BWD = 2,    // forward recomputed and adjoint in the same kernel
    PASS_BWD_LOAD = 3,   // adjoint from stored activations
};
__host__ __device__ constexpr bool pass_bwd(int p) { return p >= PASS_FWD_BWD; }

constexpr int kRelaxNoise = 0, kRelaxHard = 1, kRelaxIdentity = 2;

struct Hp {
    float lambda, lr, beta1, beta2, eps;
    uint64_t seed;
};

constexpr int kArmThreads = 128;   // latents per ARM round
constexpr int kSynThreads = 128;   // pixels per synthesis round
constexpr int kConvTH = 16, kConvTW = 32;  // conv tile (pixels)
constexpr int kUpThreads = 256;
constexpr int kUpMaxCta = 1024;    // per-stage cap on CTAs of an upsampling-adjoint pass

// Per-job device buffers carved from the caller's workspace (layout in cc_api.cu).
struct Work {
    Geom g;
    int64_t N;         // latents
    int64_t HW;
    float* yt;         // relaxed latents [N]
    float* dS;         // context-gradient planes [16][N]
    float* dR[3];      // IFCE-input gradient planes: grid k has ifce_nin(k) planes of h_k*w_k
    float* dYd;        // direct rate gradient [N]
    float* dYsyn;      // gradient reaching each grid through upsampling + synthesis [N]
    float* dIf;        // IFCE gradient of grids 3..6 summed per grid-3 cell [4][h_3*w_3]
    float* up[kL];     // up[m], m = 1..5: channels of grids m+1..6 upsampled to grid m
    float* dup[kL];    // adjoints of up[m], m = 1..5
    float* t;          // synthesis output before the residual convs [3][HW]
    float* dt;         // its adjoint [3][HW]
    float* dz;         // adjoint of the dense latents of grids 1..6 at full resolution [6][HW]
    float* tmp;        // upsampling-adjoint intermediate (largest stage)
    float* act_arm;    // stored ARM activations [34][N] (optional)
    float* act_syn;    // stored synthesis pre-activations [40][HW] (optional)
    float* gpart_arm;  // per-CTA partial gradients [n_cta_arm][756]
    float* gpart_syn;  // [n_cta_syn][467]
    float* gpart_conv; // [n_cta_conv][168]
    float* gpart_up;   // [6 stages][kUpMaxCta][4]
    double* rate_part; // [n_cta_arm]
    double* se_part;   // [n_cta_conv]
    float* grad_params;// [1415] reduced parameter gradient
    int64_t* base_step;// step at the start of an encode call
    int n_cta_arm, n_cta_syn, n_cta_conv;
    int n_cta_up[kL];  // CTAs of the upsampling-adjoint kernel of stage s = 1..6
};

int num_sms();
// Records a printf-style message for coolchic_last_error() and returns `code`.
int set_error(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// a1 relaxation: yt = y + u(seed, step, i) | rint(y) | y.  step from step_dev when non-null.
void launch_relax(const Work& w, const float* y, const int64_t* step_dev, int64_t step_host,
                  uint64_t seed, int relax, cudaStream_t s);
// a2-a3 and a9: entropy model over all latents.
void launch_arm(const Work& w, const float* params, int pass, float grad_scale, cudaStream_t s);
// a4: upsampling stages 6..2 (stage 1 is fused into the synthesis kernels).
void launch_up_forward(const Work& w, const float* params, cudaStream_t s);
// a5-a7: synthesis MLP, residual convs, distortion and their adjoints.
void launch_syn_forward(const Work& w, const float* params, int pass, cudaStream_t s);
void launch_conv(const Work& w, const float* params, const float* image, int pass, float grad_scale,
                 float* xhat_out, cudaStream_t s);
void launch_syn_backward(const Work& w, const float* params, int pass, cudaStream_t s);
// a8: upsampling adjoint, stages 1..6.
void launch_up_adjoint(const Work& w, const float* params, cudaStream_t s);
// a9 gather + a11: latent gradient assembly, then either Adam on the latents or a copy-out.
void launch_gather(const Work& w, const float* params, int relax, float* grad_out, float* y,
                   float* m, float* v, const Hp& hp, const int64_t* step_dev, cudaStream_t s);
// a10 + a11: fixed-order reduction of the per-CTA parameter gradients, then Adam or a copy-out.
void launch_param_reduce(const Work& w, float* params, float* m, float* v, float* grad_out,
                         float out_scale, const Hp& hp, const int64_t* step_dev, cudaStream_t s);
// loss record (FP64, 3 doubles: loss, rate, mse) in rd_out[*step_dev - *base_step] (slot 0 when
// step_dev is null), optional step increment.
void launch_finish(const Work& w, const Hp& hp, int have_arm, int have_conv, double* rd_out,
                   int64_t* step_dev, int mark_base, int increment, cudaStream_t s);
void launch_mark_base(const Work& w, const int64_t* step_dev, cudaStream_t s);

// sizes that the workspace layout depends on
size_t arm_smem_bytes(int pass);
int arm_grid(int64_t N);
size_t syn_bwd_smem_bytes();
int conv_tiles(int H, int W);
int up_adj_grid(int64_t pairs);
void arm_init_attributes();
void synth_init_attributes();

// decoder
void decode_init_tables();
void launch_decode(const Geom& g, const int32_t* q, const float* params, float* yq, uint32_t* prob,
                   int32_t* mu_q, int32_t* logb_q, cudaStream_t s);
void launch_clamp01(float* x, int64_t n, cudaStream_t s);

}  // namespace cc
