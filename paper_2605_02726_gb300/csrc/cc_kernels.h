// Host-side launch wrappers of the encoder-step kernels (internal to the library).
#pragma once

#include "../../include/coolchic.h"
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
    int noise_mode;                              // 0 additive uniform, 1 soft-round schedule
    float sigma0, sigma1, temp0, temp1, lr_min;  // mode 1
    int64_t n_main;                              // mode 1: first step of the hard-round stage
    int nn_opt;                                  // network parameters: 0 Adam, 1 SOAP
    float sb1, sb2, sbs;                         // SOAP: moment betas, preconditioner beta
    int sfreq;                                   // SOAP: eigenbasis refresh every sfreq steps
};
Hp hp_from(const cc_hparams_t* h);
int validate_hparams(const cc_hparams_t* h);  // CC_OK or an error code with the message set

// Training proxy at step t (Sec. IV-C/D, Table I): noise scale, temperature, learning rate and
// whether t is in the hard-round stage (mode 1 only).
struct ProxyAt {
    float sigma, temp, lr;
    bool hard;
};
__device__ __forceinline__ ProxyAt proxy_at(const Hp& hp, int64_t t) {
    ProxyAt p{0.f, 1.f, hp.lr, false};
    if (hp.noise_mode == 1) {
        p.hard = t >= hp.n_main;
        const float f = p.hard ? 1.f : (float)t / (float)hp.n_main;
        p.sigma = hp.sigma0 + (hp.sigma1 - hp.sigma0) * f;
        p.temp = hp.temp0 + (hp.temp1 - hp.temp0) * f;
        p.lr = p.hard ? hp.lr_min : hp.lr_min + 0.5f * (hp.lr - hp.lr_min) * (1.f + cospif(f));
    }
    return p;
}
// y~ of latent i at step t under the training proxy, and dy~/dy: the additive uniform proxy
// (mode 0), Eq. 13 (mode 1, main stage), rint (mode 1, hard-round stage)
__device__ __forceinline__ float relax_latent(const Hp& hp, const ProxyAt& p, float y, int64_t t, int64_t i,
                                              float& jac) {
    if (hp.noise_mode == 0) {
        jac = 1.f;
        return y + counter_uniform(hp.seed, t, i);
    }
    if (p.hard) {
        jac = 0.f;
        return rintf(y);
    }
    float d1, d2;
    const float s1 = softround(y, p.temp, d1);
    const float v = softround(fmaf(p.sigma, counter_gauss(hp.seed, t, i), s1), p.temp, d2);
    jac = d2 * d1;
    return v;
}

constexpr int kArmThreads = 128;   // latents per ARM round
constexpr int kSynThreads = 128;   // pixels per synthesis round
constexpr int kConvTH = 22, kConvTW = 32;  // conv tile (pixels)
constexpr int kUpThreads = 256;
constexpr int kUpMaxCta = 1024;    // per-stage cap on CTAs of an upsampling-adjoint pass
constexpr int kUpTX = 64;          // input columns of an upsampling-adjoint tile
constexpr int kUpTYMax = 16;       // tallest upsampling-adjoint tile (input rows)
constexpr int kUpAdjThreads = 288; // 2 x (2 kUpTX + 6) column tasks of the adjoint's pass A, in 9 warps

// Per-job device buffers carved from the caller's workspace (layout in cc_api.cu).
struct Work {
    Geom g;
    int64_t N;         // latents
    int64_t HW;
    float* yt;         // relaxed latents [N]
    float* dS;         // context-gradient planes [16][N]
    float* dR[3];      // IFCE-input gradient planes: grid k has ifce_nin(k) (+ nh) planes of h_k*w_k
    float* dYd;        // direct rate gradient [N]
    float* dYsyn;      // gradient reaching each grid through upsampling + synthesis [N]
    float* dIf;        // IFCE gradient of grids 3..6 (then the hyperlatent grids) per grid-3 cell [4 + nh][h_3*w_3]
    float* up[kL];     // up[m], m = 1..5: channels of grids m+1..6 upsampled to grid m
    float* dup[kL];    // adjoints of up[m], m = 1..5
    float* t;          // synthesis output before the residual convs [3][HW]
    float* dt;         // its adjoint [3][HW]
    float* dz;         // adjoint of the dense latents of grids 1..6 at full resolution [6][HW]
    float* zden;       // dense latents of grids 1..6 at full resolution [6][HW], written by the
                       // synthesis forward for its adjoint (null: not kept)
    float* act_arm;    // stored ARM activations [34][N] (optional)
    float* act_syn;    // stored synthesis pre-activations [40][HW] (optional)
    float* gpart_arm;  // per-CTA partial gradients [n_cta_arm][756, or 792 with hyperlatents]
    float* gpart_syn;  // [n_cta_syn][467]
    float* gpart_conv; // [n_cta_conv][168]
    float* gpart_up;   // [6 stages][kUpMaxCta][4]
    double* rate_part; // [n_cta_arm]
    double* se_part;   // [n_cta_conv]
    float* grad_params;// [1415] reduced parameter gradient
    int64_t* base_step;// step at the start of an encode call
    int64_t* step_snap;// encoder iterations: the step as the iteration's forward launches saw it
    int* status;       // bit 0: a bounded wait in the entropy model ran out (cleared by blocking calls)
    float* io_image;   // device copy of a host image [3][HW] (workspace flag bit 1, else null)
    double* io_record; // one loss record (loss, rate, mse) read back to the host (flag bit 1)
    int n_cta_arm, n_cta_syn, n_cta_conv;
    int discard_dead;  // encoder iterations: drop the L2 lines of synthesis scratch after its last read
    int ifce_early;    // encoder iterations: the IFCE cell sums run in the first forward upsampling launch
    int n_cta_up[kL];  // CTAs of the upsampling-adjoint kernel of stage s = 1..6
};

// ---------------------------------------------------------------------------------------------
// Multi-job launches.  Every kernel body takes its arguments, its CTA index within the job and
// the job's CTA count.  A single-job launch passes the arguments by value; a multi-job launch
// reads an array of per-job arguments and the first CTA of each job (njobs + 1 entries) from
// device memory, so that one launch serves many images of different sizes.
// ---------------------------------------------------------------------------------------------
template <typename A>
struct Batch {
    const A* args;         // [njobs], device
    const int* cta_begin;  // [njobs + 1], device
    int njobs;
    int total_ctas;
};

// The job whose CTA range [cb[j], cb[j+1]) holds this CTA: the number of job starts cb[1..nj-1] at
// or below blockIdx.x (cb is increasing), counted by the first warp 32 starts per round trip.
// Reads only the static table, so it may run before the dependent-launch wait.
__device__ __forceinline__ int batch_job(const int* __restrict__ cb, int nj) {
    __shared__ int s_job;
    if (threadIdx.x < 32) {
        int j = 0;
        for (int base = 1; base < nj; base += 32) {
            const int q = base + (int)threadIdx.x;
            const unsigned past = __ballot_sync(0xffffffffu, q < nj && (int)blockIdx.x >= __ldg(cb + q));
            j += __popc(past);
            if (past != 0xffffffffu) break;
        }
        if (threadIdx.x == 0) s_job = j;
    }
    __syncthreads();
    return s_job;
}

// Programmatic dependent launch: the kernels of an iteration are launched with programmatic stream
// serialization, so a kernel's CTAs may be scheduled while its predecessor in the stream finishes.
// Every such kernel lets its own successor start as soon as all of its CTAs are running
// (launch_dependents) and reads nothing that earlier kernels wrote before griddepcontrol.wait,
// which returns once the predecessor has completed and its writes are visible.  Both happen in
// the argument fetches below; only kernel parameters and the static argument tables are read
// before the wait.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline void launch_pdl(void (*kern)(P...), int grid, int block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// Copies job j's arguments into shared memory (all threads), then synchronises and waits for the
// predecessor kernel.
template <typename A>
__device__ __forceinline__ void batch_fetch(const A* __restrict__ args, int j, A& sa) {
    static_assert(sizeof(A) % 4 == 0, "argument structs are copied as 32-bit words");
    pdl_trigger();
    const int* src = reinterpret_cast<const int*>(args + j);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    pdl_wait();
}

// Arguments of a single-job launch.  The kernel parameter is declared __grid_constant__ (taking
// its address makes no copy).  Kernels whose bodies read it at compile-time offsets only use it
// where it is, in the parameter space (pdl_enter); kernels that index it with a runtime grid number
// (the grid tables) first copy it to shared memory (param_fetch: the first warp copies, the CTA
// synchronises).  A copy in every thread of every CTA, as the predicated per-word form needs, cost
// more than the arguments' use.
__device__ __forceinline__ void pdl_enter() {
    pdl_trigger();
    pdl_wait();
}
template <typename A>
__device__ __forceinline__ void param_fetch(const A& a, A& sa) {  // a: the __grid_constant__ parameter
    static_assert(sizeof(A) % 4 == 0, "argument structs are copied as 32-bit words");
    pdl_trigger();
    if (threadIdx.x < 32) {
        const int* src = reinterpret_cast<const int*>(&a);
        int* dst = reinterpret_cast<int*>(&sa);
        for (int w = threadIdx.x; w < (int)(sizeof(A) / 4); w += 32) dst[w] = src[w];
    }
    __syncthreads();
    pdl_wait();
}

// Copies params[lo, lo + n) to shared memory `sm` by asynchronous copies (every thread's copies
// in flight at once: one round trip for the CTA instead of one per loop pass), then a barrier.
// The result indexes the copy with absolute parameter offsets (valid for [lo, lo + n) only).
__device__ __forceinline__ const float* stage_params(const float* P, int lo, int n, float* sm) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) cp_async4(sm + j, P + lo + j);
    cp_async_wait_all();
    __syncthreads();
    return sm - lo;
}

// Argument structs of the kernels (filled by the launchers and by the batch planner).
struct RelaxArgs {
    const float* y;
    float* yt;
    int64_t N;
    const int64_t* step_dev;  // step from here when non-null, else step_host
    int64_t step_host;
    Hp hp;                    // seed and training proxy
    int relax;
    int pad_;
};
struct UpFwdArgs {
    const float* src0;   // y~ of grid m+1
    const float* srcup;  // up[m+1] (channels 1..), may be null when nch == 1
    float* dst;          // up[m]
    const float* taps;   // 4 taps of this stage (device)
    int hs, ws, ht, wt, nch, pad_;
};
// The forward upsampling outputs up[m] for m >= kUpArmLo (stages 6..4, grids of 1/16 the image
// and smaller) are computed by the first CTA of the entropy-model launch, which needs none of
// them and whose other CTAs take all the latents; the per-stage kernels compute the rest.
constexpr int kUpArmLo = 3;
constexpr int kUpArmStages = kL - 1 - kUpArmLo;  // up[5], up[4], up[3]
struct ArmArgs {
    UpFwdArgs upc[kUpArmStages];  // m = kL-2 down to kUpArmLo
    int upc_on, pad2_;
    Geom g;
    int64_t N;
    const float* yt;
    const float* params;
    float gscale;  // dLoss / dbits
    int pad_;
    float* dS;
    float* dR0;
    float* dR1;
    float* dR2;
    float* dYd;
    float* act;         // [34][N]: a1 (16), a2 (16), mu, s
    float* gpart;       // [n_cta][756, or 792 with hyperlatents]
    double* rate_part;  // [n_cta]
    int* status;        // bit 0 set when a wait on the MMA completion ran out
    int inject_stall;   // failure-detection tests: the first MMA group is never committed
    int pad3_;
};
// Failure-detection test hook (coolchic_test_inject_stall): launches made while it is set withhold
// the entropy model's first MMA commit, so that its bounded waits run out.
int test_inject_stall();
// Workspace ranges that are dead when a kernel starts (kernels before it have read them for the
// last time this iteration; the next iteration writes them before reading): the kernel drops their
// L2 lines with discard.global.L2, so they are neither written back to DRAM nor left to displace
// data that is still live (the context-gradient planes, which the gather reads after the synthesis
// chain).  Slots with n = 0 are unused; every range starts on a 256-byte boundary and its last line
// lies within its own padding.  Set only for encoder iterations (coolchic_encode_step, batches);
// COOLCHIC_DISCARD=0 turns it off.
bool discard_enabled();
struct DeadRanges {
    float* p[4];
    int64_t n[4];  // floats
};
__device__ __forceinline__ void discard_dead(const DeadRanges& d, int cta, int ncta) {
    const int64_t t0 = (int64_t)cta * blockDim.x + threadIdx.x, nt = (int64_t)ncta * blockDim.x;
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
        if (d.n[r] <= 0) continue;
        const char* b = reinterpret_cast<const char*>(d.p[r]);
        const int64_t lines = (d.n[r] * 4 + 127) / 128;
        for (int64_t l = t0; l < lines; l += nt) asm volatile("discard.global.L2 [%0], 128;" ::"l"(b + l * 128) : "memory");
    }
}

struct SynArgs {
    Geom g;
    int64_t HW;
    const float* yt;
    const float* up1;
    const float* params;
    float* t;         // [3][HW]
    const float* dt;  // [3][HW]
    float* act;       // [40][HW]
    float* dYsyn0;    // grid-0 part of dYsyn [HW]
    float* dz;        // [6][HW]
    float* zden;      // [6][HW] dense latents of grids 1..6: written by the forward, read by the adjoint
    float* gpart;     // [n_cta][467]
    DeadRanges dead;  // the adjoint: t (read last by the convolutions)
};
struct ConvArgs {
    int H, W;
    int64_t HW;
    const float* t;
    const float* img;
    const float* params;
    float* dt;
    float* xhat;      // optional
    float* gpart;     // [n_cta][168]
    double* se_part;  // [n_cta]
    float gscale;     // 2 / (3 HW) times the caller's outer scale
    int tiles_x, n_tiles, pad_;
};
struct UpAdjArgs {
    const float* D;      // [nch][ht][wt]
    const float* src0;   // S_s channel 0 = y~ of grid s
    const float* srcup;  // S_s channels 1.. = up[s]
    float* out0;         // dYsyn of grid s
    float* outup;        // dup[s]
    float* gpart;        // [n_cta][4]
    const float* taps;
    int hs, ws, ht, wt, nch;
    int ty;              // tile height in input rows (2..kUpTYMax)
    DeadRanges dead;     // stage 1: the dense latents and dt (read last by the synthesis adjoint); stage 2: dz
};
struct IfceArgs {
    Geom g;
    const float* dR0;
    const float* dR1;
    const float* dR2;
    float* Q;
};
struct GatherArgs {
    Geom g;
    const float* dYd;
    const float* dS;
    const float* dR0;
    const float* dR1;
    const float* dIf;
    const float* dYsyn;
    float* grad_out;  // non-null: write the gradient instead of taking an Adam step
    float* y;
    float* m;
    float* v;
    const int64_t* step_dev;  // step from here when non-null, else step_host
    int64_t step_host;
    float* yt_next;   // non-null (with Adam): also write the next step's relaxed latents
    Hp hp;
    int zero_grad;    // hard rounding: no latent gradient
    int proxy;        // latents relaxed by the training proxy: chain rule through dy~/dy
};
struct ReduceArgs {
    float* gsoap;  // SOAP (hp.nn_opt == 1): the reduced gradient of the SOAP blocks goes here
    int hyper;     // the job has hyperlatent grids: 1451 parameters, ARM partial rows of 792
    int pad_h_;
    const float* garm;
    const float* gup;  // [6][kUpMaxCta][4]
    const float* gsyn;
    const float* gconv;
    float* params;
    float* m;
    float* v;
    float* grad_out;  // non-null: write the gradient (times out_scale) instead of Adam
    const int64_t* step_dev;
    Hp hp;
    int n_arm, n_syn, n_conv;
    int nup[kL - 1];
    float out_scale;
};
struct FinishArgs {
    const double* rate_part;
    const double* se_part;
    double* rd;         // record base (3 doubles per slot), may be null
    int64_t* step_dev;  // slot = *step_dev - *base_step when both non-null, else 0
    int64_t* base_step;
    double inv_hw, inv_3hw, lambda;
    int n_rate, n_se, rd_stride, mark_base, increment, pad_;
};

// The network-parameter blocks that SOAP preconditions (two-dimensional weights).
constexpr int kSoapBlocks = 12;
__host__ __device__ constexpr bool soap_param(int p) {
    return (p >= po::arm_w1 && p < po::arm_b1) || (p >= po::arm_w2 && p < po::arm_b2) ||
           (p >= po::arm_w3 && p < po::arm_b3) || (p >= po::arm_ws && p < po::arm_bs) ||
           (p >= po::if_w0 && p < po::if_b0) || (p >= po::if_w1 && p < po::if_b1) ||
           (p >= po::if_w2 && p < po::if_b2) || (p >= po::syn_w1 && p < po::syn_b1) ||
           (p >= po::syn_w2 && p < po::syn_b2) || (p >= po::syn_ws && p < po::syn_bs) ||
           (p >= po::cv1_w && p < po::cv1_b) || (p >= po::cv2_w && p < po::cv2_b);
}
struct SoapArgs {
    const float* grad;  // reduced gradient (workspace)
    float* params;
    float* m;
    float* v;
    float* soap;        // L, R, Q_L, Q_R of every block
    const int64_t* step_dev;
    Hp hp;
};
int64_t soap_state_floats();
SoapArgs soap_args(const Work& w, float* params, float* m, float* v, float* soap, const Hp& hp,
                   const int64_t* step_dev);
// SOAP step of the two-dimensional network blocks (after the parameter reduction)
void launch_soap(const Work& w, float* params, float* m, float* v, float* soap, const Hp& hp,
                 const int64_t* step_dev, cudaStream_t s);
void launch_soap_b(const Batch<SoapArgs>& b, cudaStream_t s);

int num_sms();
// Records a printf-style message for coolchic_last_error() and returns `code`.
int set_error(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// a1 relaxation: yt = y + u(seed, step, i) | rint(y) | y.  step from step_dev when non-null.
void launch_relax(const Work& w, const float* y, const int64_t* step_dev, int64_t step_host,
                  const Hp& hp, int relax, cudaStream_t s);
// a2-a3 and a9: entropy model over all latents.
void launch_arm(const Work& w, const float* params, int pass, float grad_scale, cudaStream_t s);
// a4: upsampling stages m_hi+1 .. 2, output up[m_hi] .. up[1] (stage 1 is fused into the
// synthesis kernels; after an entropy-model launch m_hi = kUpArmLo - 1, for decoding kL - 2).
void launch_up_forward(const Work& w, const float* params, int m_hi, cudaStream_t s);
// a5-a7: synthesis MLP, residual convs, distortion and their adjoints.
void launch_syn_forward(const Work& w, const float* params, int pass, cudaStream_t s);
void launch_conv(const Work& w, const float* params, const float* image, int pass, float grad_scale,
                 float* xhat_out, cudaStream_t s);
void launch_syn_backward(const Work& w, const float* params, int pass, cudaStream_t s);
// a8: upsampling adjoint, stages 1..6.
void launch_up_adjoint(const Work& w, const float* params, cudaStream_t s);
// a9 gather + a11: latent gradient assembly, then either Adam on the latents or a copy-out.
// relax_next: the Adam update also writes the next step's relaxed latents (y~ of step + 1), so
// that the next iteration needs no relaxation launch.
void launch_gather(const Work& w, const float* params, int relax, float* grad_out, float* y,
                   float* m, float* v, const Hp& hp, const int64_t* step_dev, int64_t step_host,
                   cudaStream_t s, bool relax_next = false);
// a10 + a11: fixed-order reduction of the per-CTA parameter gradients, then Adam or a copy-out.
void launch_param_reduce(const Work& w, float* params, float* m, float* v, float* grad_out,
                         float out_scale, const Hp& hp, const int64_t* step_dev, cudaStream_t s);
// loss record (FP64, 3 doubles: loss, rate, mse) in rd_out[*step_dev - *base_step] (slot 0 when
// step_dev is null), optional step increment.
void launch_finish(const Work& w, const Hp& hp, int have_arm, int have_conv, double* rd_out,
                   int64_t* step_dev, int mark_base, int increment, cudaStream_t s);
void launch_mark_base(const Work& w, const int64_t* step_dev, cudaStream_t s);
// the seeded initial state (coolchic_init_state)
struct InitArgs {
    float *y, *params, *m_lat, *v_lat, *m_par, *v_par;
    int64_t* step;
    int64_t N;
    uint64_t seed;
    int nh;  // hyperlatent grids (0 or kNH)
    int pad_;
};
void launch_init_state(const InitArgs& a, cudaStream_t s);

// sizes that the workspace layout depends on
size_t arm_smem_bytes(int pass, bool hyper);
int arm_grid(int64_t N, bool hyper);
int conv_tiles(int H, int W);
int up_adj_ctas(int nch, int hs, int ws);
void arm_init_attributes();
void synth_init_attributes();
void syn_init_attributes();
void conv_init_attributes();

// argument builders, CTA counts and multi-job launches (batched encode)
RelaxArgs relax_args(const Work& w, const float* y, const int64_t* step_dev, int64_t step_host, const Hp& hp,
                     int relax);
ArmArgs arm_args(const Work& w, const float* params, float grad_scale);
UpFwdArgs up_fwd_args(const Work& w, const float* params, int m);
SynArgs syn_args(const Work& w, const float* params);
ConvArgs conv_args(const Work& w, const float* params, const float* image, float grad_scale, float* xhat_out);
UpAdjArgs up_adj_args(const Work& w, const float* params, int st);
IfceArgs ifce_args(const Work& w);
GatherArgs gather_args(const Work& w, int relax, float* grad_out, float* y, float* m, float* v, const Hp& hp,
                       const int64_t* step_dev, int64_t step_host, bool relax_next = false);
ReduceArgs reduce_args(const Work& w, float* params, float* m, float* v, float* grad_out, float out_scale,
                       const Hp& hp, const int64_t* step_dev);
FinishArgs finish_args(const Work& w, const Hp& hp, int have_arm, int have_conv, double* rd, int rd_stride,
                       int64_t* step_dev, int mark_base, int increment);
int relax_ctas(const Work& w);
int up_fwd_ctas(const Work& w, int m);
int syn_fwd_ctas(const Work& w);
int ifce_ctas(const Work& w);
// encoder iterations: the parameter reduction, the loss record with the step increment (the finish,
// reading w.rate_part and w.se_part; rd_out as in launch_finish) and the latent gather (with Adam)
// in one launch.  The reduction and the gather read the step from w.step_snap, which the
// iteration's launch_up_fwd_ifce wrote, so that the finish may increment *step_dev beside them.
void launch_gather_reduce(const Work& w, float* y, float* m_lat, float* v_lat, float* params, float* m_par,
                          float* v_par, const Hp& hp, int64_t* step_dev, double* rd_out, cudaStream_t s,
                          bool relax_next);
// the first forward upsampling stage after the entropy model (output up[m]) and the IFCE cell sums
// in one launch (encoder iterations); its first thread also copies *step_dev to w.step_snap
void launch_up_fwd_ifce(const Work& w, const float* params, int m, const int64_t* step_dev, cudaStream_t s);
int gather_ctas(const Work& w);
int reduce_ctas();
void launch_relax_b(const Batch<RelaxArgs>& b, cudaStream_t s);
void launch_arm_b(const Batch<ArmArgs>& b, int pass, bool hyper, cudaStream_t s);  // hyper: the kernel form of jobs with hyperlatent grids
void launch_up_fwd_b(const Batch<UpFwdArgs>& b, cudaStream_t s);
void launch_syn_fwd_b(const Batch<SynArgs>& b, cudaStream_t s);
void launch_conv_b(const Batch<ConvArgs>& b, cudaStream_t s);
void launch_syn_bwd_b(const Batch<SynArgs>& b, cudaStream_t s);
void launch_up_adj_b(const Batch<UpAdjArgs>& b, cudaStream_t s);
void launch_ifce_b(const Batch<IfceArgs>& b, cudaStream_t s);
void launch_gather_b(const Batch<GatherArgs>& b, cudaStream_t s);
void launch_reduce_b(const Batch<ReduceArgs>& b, cudaStream_t s);
void launch_finish_b(const Batch<FinishArgs>& b, cudaStream_t s);
void launch_mark_base_b(const Batch<FinishArgs>& b, cudaStream_t s);
// workspace layout of one job (cc_api.cu); returns the bytes needed, fills *w when base != null
size_t layout_job(const cc_arch_t* arch, int flags, char* base, Work* w);
int device_setup_checked();

// decoder
void decode_init_tables();
void launch_decode(const Geom& g, const int32_t* q, const float* params, float* yq, uint32_t* prob,
                   int32_t* mu_q, int32_t* logb_q, cudaStream_t s);
void launch_clamp01(float* x, int64_t n, cudaStream_t s);

}  // namespace cc
