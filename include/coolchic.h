/*
 * coolchic.h -- C ABI of the GB300 (sm_103a) Cool-chic encoder-step library.
 *
 * The library runs the per-iteration encoder step of an overfitted image codec: forward and
 * backward pass over every pixel and latent, then Adam (Cool-chic 5.0, Sec. IV-A, Eq. 10), plus
 * the rate-distortion evaluation and the decoder (Sec. III).  Every step runs in hand-written CUDA
 * kernels; the library never allocates device memory per call and never falls back to the CPU.
 *
 * Conventions (all entry points):
 *   - Pointers marked [device] must point to device memory of the current CUDA device; [host]
 *     pointers to host memory.  The caller owns every buffer.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *     stream-ordered and asynchronous unless marked "blocking".
 *   - Return value: CC_OK (0) or a negative CC_ERR_* code.  On error, coolchic_last_error()
 *     returns a thread-local message.  Argument checks run before any launch; a failed check
 *     launches nothing.
 *   - Floating point is FP32 on the device; loss reductions are finished in FP64.
 *
 * Architecture (fixed by this library; see cc_arch_t): C = 3 channels, L = 7 latent grids of one
 * channel (grid k is ceil(H/2^k) x ceil(W/2^k), Sec. III-A1, Eq. 1), ARM over 16 causal
 * neighbours + 4 inter-feature values from an IFCE on grids 0..2 (Sec. III-A2, Eq. 5), two hidden
 * layers of 16 with ReLU and a linear stabilizer (Eq. 9), outputs (mu, log b); learned symmetric
 * 8-tap x2 upsampling per stage (Sec. III-B, Eq. 7); synthesis 7 -> 40 (GELU) -> 3 with a 7 -> 3
 * stabilizer, then two residual 3x3 convolutions 3 -> 3 (Eq. 8, Table II).
 *
 * Latent layout: one flat FP32 vector, grids concatenated k = 0..6, each row-major [h_k][w_k].
 * Image layout: planar CHW FP32, values in [0, 1].
 * Parameter layout: one flat FP32 vector of 1415 values; blocks in this order, matrices row-major
 * [out][in]:  arm.w1[16][20] arm.b1[16] arm.w2[16][16] arm.b2[16] arm.w3[2][16] arm.b3[2]
 *             arm.ws[2][20] arm.bs[2] ifce0.w[4][6] ifce0.b[4] ifce1.w[4][5] ifce1.b[4]
 *             ifce2.w[4][4] ifce2.b[4] up.taps[6][4] syn.w1[40][7] syn.b1[40] syn.w2[3][40]
 *             syn.b2[3] syn.ws[3][7] syn.bs[3] conv1.w[3][3][3][3] conv1.b[3] conv2.w[3][3][3][3]
 *             conv2.b[3].   Use coolchic_param_block() to enumerate them.
 */
#ifndef COOLCHIC_H
#define COOLCHIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_OK 0
#define CC_ERR_ARG (-1)         /* invalid argument (shape, pointer, value)          */
#define CC_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed       */
#define CC_ERR_WORKSPACE (-3)   /* workspace missing, too small or misaligned        */
#define CC_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up                */
#define CC_ERR_UNSUPPORTED (-5) /* architecture field other than the supported one   */

/* Decoder architecture.  Only H and W are free; every other field must hold the value in
 * brackets (coolchic_arch_init fills them), otherwise calls return CC_ERR_UNSUPPORTED. */
typedef struct {
    int32_t C;          /* [3] image channels                                     */
    int32_t H, W;       /* image height and width, 1 .. 16384                      */
    int32_t L;          /* [7] latent grids                                        */
    int32_t n_ctx;      /* [16] spatial context size                               */
    int32_t ifce_dim;   /* [4] inter-feature context width F                       */
    int32_t ifce_grids; /* [3] grids 0..ifce_grids-1 carry an IFCE                 */
    int32_t arm_hidden; /* [16]                                                    */
    int32_t arm_layers; /* [2]                                                     */
    int32_t syn_hidden; /* [40]                                                    */
    int32_t n_resconv;  /* [2]                                                     */
    int32_t up_taps;    /* [8]                                                     */
    int32_t stabilizer; /* [1]                                                     */
    int32_t hyper_grids;/* [0] or 3: hyperlatent grids (Sec. III-A3, Eq. 6; Table II: 1/16 to
                           1/64 for small images).  They follow the latent grids in the latent
                           vector (grid 7 + q has the shape of grid 4 + q), are coded by the same
                           ARM from their spatial context, and are read by the IFCEs of grids 0..2
                           as three more nearest-neighbour inputs; the upsampling and the
                           synthesis never see them.  The IFCE weights of those inputs follow
                           the 1415 parameters as the block ifce_h.w [3][4][3] (1451 in all). */
} cc_arch_t;

/* Encoder hyper-parameters.  lambda weighs the rate in bits per pixel (Eq. 10 with R divided by
 * H*W); Adam (Sec. IV-B) uses lr, beta1, beta2, eps for latents and parameters alike.
 * noise_mode selects the training proxy of the latents at step t:
 *   CC_NOISE_UNIFORM:   y~ = y + u, u ~ U[-1/2, 1/2) from a counter hash of (seed, t, i); lr fixed.
 *   CC_NOISE_SOFTROUND: the paper's proxy and schedule (Sec. IV-C/D, Eq. 13-14, Table I): for
 *     t < n_main, y~ = s_T(s_T(y) + sigma n) with n ~ N(0, 1) (Box-Muller on the same hash),
 *     sigma and T linear from (sigma0, temp0) to (sigma1, temp1) over the n_main steps and the
 *     learning rate cosine from lr to lr_min; for t >= n_main (hard-round stage) y~ = rint(y),
 *     the latents are frozen and the parameters use lr_min.  temp0, temp1 > 0. */
#define CC_NOISE_UNIFORM 0
#define CC_NOISE_SOFTROUND 1
typedef struct {
    float lambda, lr, beta1, beta2, eps;
    int32_t noise_mode;
    uint64_t seed;
    float sigma0, sigma1, temp0, temp1, lr_min; /* CC_NOISE_SOFTROUND only */
    int32_t nn_optimizer;                       /* CC_OPT_ADAM or CC_OPT_SOAP                */
    int64_t n_main;                             /* CC_NOISE_SOFTROUND only */
    float soap_beta1, soap_beta2, soap_shampoo_beta; /* CC_OPT_SOAP only, each in [0, 1)  */
    int32_t soap_freq;                          /* CC_OPT_SOAP only: eigenbasis refresh period >= 1 */
} cc_hparams_t;

/* Optimizer of the network parameters (the latents always use Adam, Sec. IV-B):
 *   CC_OPT_ADAM: Adam with beta1, beta2, eps, like the latents.
 *   CC_OPT_SOAP: SOAP (Vyas et al., cited by Sec. IV-B; the paper gives none of its settings) on the
 *     two-dimensional weight blocks (ARM W1, W2, W3, Ws; the three IFCE matrices; synthesis W1, W2,
 *     Ws; each residual convolution's kernel as [out][in * 9]) and Adam on the other parameters.
 *     For a block W (m x n) with gradient G, at SOAP step s = Adam count - 1:
 *       s = 0: L = (1 - bs) G G^T, R = (1 - bs) G^T G, Q_L, Q_R = their eigenvectors; W unchanged;
 *       s >= 1: G' = Q_L^T G Q_R, M = b1 M + (1 - b1) G, M' = Q_L^T M Q_R, V = b2 V + (1 - b2) G'^2,
 *         W -= lr Q_L [(M' / (1 - b1^s)) / (sqrt(V / (1 - b2^s)) + eps)] Q_R^T, then L, R take the
 *         new G (same beta bs) and, every soap_freq steps, Q_L, Q_R become their eigenvectors
 *         (full eigen-decomposition; columns by decreasing eigenvalue, the entry of largest
 *         magnitude of each positive).
 *     (b1, b2, bs) = (soap_beta1, soap_beta2, soap_shampoo_beta); lr is the proxy's learning rate.
 *     M and V are the block's slots of m_par and v_par (V in the rotated coordinates); L, R, Q_L,
 *     Q_R live in state->soap.  Within a repeated eigenvalue the eigenbasis is not unique, so two
 *     implementations agree on the step only where the preconditioners' eigenvalues are distinct. */
#define CC_OPT_ADAM 0
#define CC_OPT_SOAP 1

/* Encoder state, all [device], caller-owned: latents, params and their Adam moments (same
 * sizes), and the step counter (one int64; the number of Adam steps already taken, which also
 * keys the noise of the next iteration). */
typedef struct {
    float *latents, *params, *m_lat, *v_lat, *m_par, *v_par;
    int64_t* step;
    float* soap; /* CC_OPT_SOAP: coolchic_soap_state_floats() floats (zero before the first step); else NULL */
} cc_state_t;

/* Rate-distortion record: loss = mse + lambda * rate_bits / (H*W). */
typedef struct {
    double loss, rate_bits, mse;
} cc_rd_t;

/* Relaxation of the latents used by a forward pass (Sec. IV-C). */
#define CC_RELAX_NOISE 0    /* the training proxy of hp->noise_mode at step */
#define CC_RELAX_HARD 1     /* rint(y), round half to even (Eq. 12) */
#define CC_RELAX_IDENTITY 2 /* y as given                           */

/* Fill *arch with the supported architecture for an H x W image.  Returns CC_ERR_ARG for a
 * NULL pointer or a size outside 1..16384. */
int coolchic_arch_init(cc_arch_t* arch, int32_t H, int32_t W);

/* Number of latents (sum over grids of h_k * w_k, hyperlatent grids included) and of parameters
 * (1415, or 1451 with hyperlatent grids); -1 on a bad arch. */
int64_t coolchic_latent_count(const cc_arch_t* arch);
int64_t coolchic_param_count(const cc_arch_t* arch);

/* Parameter block `index` (0-based, in storage order): its name (static string), offset and
 * length in floats.  Returns CC_ERR_ARG past the last block.  Block 25, ifce_h.w, exists only
 * in the parameter vectors of architectures with hyperlatent grids. */
int coolchic_param_block(int32_t index, const char** name, int32_t* offset, int32_t* length);

/* Seeded initial encoder state, written on the device (the paper does not give its
 * initialisation; this is the library's reading, the distribution of the host generator of the
 * tests drawn from the counter hash of the relaxation noise instead):
 *   latents y_i = 0.01 n_i, n_i the Box-Muller standard normal of the hash at (seed, step -1, i);
 *   hidden-layer weights (ARM W1 and W2, the three IFCE matrices, synthesis W1)
 *   w_p = 2 u_p / sqrt(fan_in), u_p in [-1/2, 1/2) the uniform of the hash at (seed, step -2, p),
 *   p the flat parameter index;  upsampling taps the Keys cubic (a = -0.75) samples at every
 *   stage;  every other parameter, both Adam moments and *state->step zero.
 *   state [host struct of device pointers], every buffer written (sizes as in
 *   coolchic_latent_count / coolchic_param_count).
 * Asynchronous on `stream`.  CC_ERR_ARG for a bad arch or a NULL pointer. */
int coolchic_init_state(const cc_arch_t* arch, uint64_t seed, const cc_state_t* state, void* stream);

/* Floats of the SOAP state (CC_OPT_SOAP): for each two-dimensional block in storage order, L
 * [m][m], R [n][n], Q_L [m][m], Q_R [n][n] (13498 floats). */
int64_t coolchic_soap_state_floats(void);

/* Bytes of device workspace one job needs.  `flags` bit 0 (CC_WS_STORE_ACTIVATIONS): room for
 * stored forward activations (coolchic_forward with store_activations = 1).  Bit 1
 * (CC_WS_HOST_IO): room for the device copy of the image and of one loss record that
 * coolchic_encode_step_host uses.  A workspace sized with more flags serves every call that needs
 * fewer.  Returns 0 on a bad arch. */
#define CC_WS_STORE_ACTIVATIONS 1
#define CC_WS_HOST_IO 2
size_t coolchic_workspace_bytes(const cc_arch_t* arch, int32_t flags);

/* Number of kernel launches a coolchic_encode_step call of n_iters iterations makes (no
 * counterpart in the paper; for profiling and graph sizing): the first iteration relaxes the
 * latents in a launch of its own, later ones take them from the previous Adam update.  -1 on a
 * bad arch or n_iters < 0; needs no device. */
int64_t coolchic_kernel_launches(const cc_arch_t* arch, int32_t n_iters);

/* Encoder iterations (Sec. IV-A..B): for it = 0..n_iters-1, relax the latents with the noise of
 * step *state->step, run the forward pass and its adjoint over all latents and pixels, take one
 * Adam step on latents and parameters, increment *state->step.
 *   image      [device] CHW FP32, 3*H*W values.
 *   state      [host struct of device pointers], updated in place.
 *   rd_per_iter [device, nullable] n_iters records: loss, rate, mse measured before each update.
 *   workspace  [device] coolchic_workspace_bytes(arch, 0) bytes, 256-byte aligned; contents are
 *              scratch between calls.
 * Asynchronous on `stream`; may be captured in a CUDA graph.  A call of at most 4 iterations is
 * captured into a CUDA graph of the library's own on its first occurrence with given arguments
 * (all values and pointers), which later identical calls replay (at most 16 kept; not while
 * kernel timing records or the caller's stream is capturing; environment COOLCHIC_GRAPHS=0 turns
 * this off); longer calls launch eagerly.  Workspace buffers that an iteration has read for the
 * last time (the synthesis output before the convolutions, the kept dense latents and their
 * gradients) are dropped from L2 without being written back (discard.global.L2; environment
 * COOLCHIC_DISCARD=0 turns this off), so the workspace holds nothing readable between calls.
 * n_iters = 0 launches nothing. */
int coolchic_encode_step(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image,
                         const cc_state_t* state, int32_t n_iters, cc_rd_t* rd_per_iter,
                         void* workspace, size_t workspace_bytes, void* stream);

/* coolchic_encode_step for a caller whose image and result live in host memory (the call an
 * application makes end to end): the image is copied from `image_host` [host, 3*H*W FP32; pinned
 * memory makes the copy asynchronous] into the workspace, the n_iters >= 1 iterations run on
 * it, and the record (loss, rate, mse) of the last iteration lands in `rd_last_host` [host,
 * nullable].  The image copy runs on a stream of the library's, after the work enqueued on
 * `stream` before the call and beside the iteration's first kernels (which do not read the
 * image), and the synthesis forward waits for it; `image_host` must stay unchanged until the call's
 * work on `stream` is done.  A pinned `rd_last_host` is written by the last kernel directly,
 * any other host buffer by a copy on `stream`; either way, synchronise `stream` before reading
 * it.  The workspace must hold coolchic_workspace_bytes(arch, CC_WS_HOST_IO) bytes.  The
 * iterations are those of coolchic_encode_step (Sec. IV-A..B), with its graph replay of short
 * calls. */
int coolchic_encode_step_host(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image_host,
                              const cc_state_t* state, int32_t n_iters, cc_rd_t* rd_last_host,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Batched encoder iterations (no counterpart in the paper, which encodes one image at a time):
 * n_jobs images of any sizes, each with its own hyper-parameters, state and workspace (sized by
 * coolchic_workspace_bytes(arch, 0)), advance together; every kernel of the iteration is one
 * launch for all jobs.  The result of each job equals that of coolchic_encode_step on it, up to
 * the summation order of its parameter gradients (which the schedule changes).
 *
 * coolchic_batch_create (blocking, not capturable) validates the jobs, plans the launches and
 * uploads the plan to `table` [device, 256-byte aligned, coolchic_batch_table_bytes bytes, owned
 * by the caller and kept alive and unmodified until coolchic_batch_destroy].  `schedule`
 * (nullable: all 1) gives, per kernel class, the fraction (0, 1] of each job's single-image CTA
 * count used in the batch.  rd_capacity: records kept per coolchic_batch_step call (0: none).
 * coolchic_batch_step (asynchronous, capturable in a CUDA graph) runs n_iters iterations on every
 * job (n_iters <= rd_capacity when rd_capacity > 0); the records of the last call are at
 * coolchic_batch_records(): [device] rd_capacity x n_jobs cc_rd_t, slot [iteration][job]. */
typedef struct {
    float arm, syn, conv, other;
} cc_schedule_t;
typedef struct cc_batch cc_batch_t;
size_t coolchic_batch_table_bytes(int32_t n_jobs, int32_t rd_capacity);
int coolchic_batch_create(int32_t n_jobs, const cc_arch_t* archs, const cc_hparams_t* hps,
                          const float* const* images, const cc_state_t* states, void* const* workspaces,
                          const size_t* workspace_bytes, const cc_schedule_t* schedule,
                          int32_t rd_capacity, void* table, size_t table_bytes, cc_batch_t** batch);
/* coolchic_batch_create for a caller that keeps the GPU busy while it plans (a serving loop):
 * the plan is written to `host_staging` [host, pinned, coolchic_batch_table_bytes bytes] and
 * copied to `table` by a cudaMemcpyAsync on `stream`, so the call returns without waiting for
 * the device; host_staging and table must stay untouched until the stream has passed the copy,
 * and the batch's first step must be ordered after it (same stream).  Nothing here blocks. */
int coolchic_batch_create_async(int32_t n_jobs, const cc_arch_t* archs, const cc_hparams_t* hps,
                                const float* const* images, const cc_state_t* states, void* const* workspaces,
                                const size_t* workspace_bytes, const cc_schedule_t* schedule,
                                int32_t rd_capacity, void* table, size_t table_bytes, void* host_staging,
                                void* stream, cc_batch_t** batch);
int coolchic_batch_step(cc_batch_t* batch, int32_t n_iters, void* stream);
const cc_rd_t* coolchic_batch_records(const cc_batch_t* batch);
int coolchic_batch_destroy(cc_batch_t* batch);

/* Forward pass only (Eq. 10): rate of the relaxed latents (Eq. 3, Eq. 11), reconstruction and
 * distortion.  relax = CC_RELAX_*; CC_RELAX_NOISE applies the training proxy of hp->noise_mode at
 * `step` (the noise, and for CC_NOISE_SOFTROUND the schedule's sigma, T and stage).
 *   latents, params [device];  rd_out [device, nullable] one record;
 *   xhat_out [device, nullable] reconstructed CHW image (not clamped);
 *   store_activations: 1 keeps the activations the adjoint needs in the workspace (workspace
 *   sized with flags = 1) so that coolchic_backward can skip their recomputation. */
int coolchic_forward(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image,
                     const float* latents, const float* params, int64_t step, int32_t relax,
                     int32_t store_activations, cc_rd_t* rd_out, float* xhat_out, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Adjoint of coolchic_forward: gradients of the loss with respect to the latents and the
 * parameters, scaled by grad_scale (dLoss/dOutput of a caller's graph); under CC_RELAX_NOISE the
 * latent gradient includes dy~/dy of the training proxy (1, or the soft-rounding derivatives).
 *   use_stored: 1 reads the activations a preceding coolchic_forward(store_activations = 1) left
 *   in the same workspace with the same inputs; 0 recomputes them per tile.
 *   grad_latents [device] N floats, grad_params [device] 1415 floats, both overwritten.
 *   Under CC_RELAX_HARD the latent gradient is zero (rounding has no derivative). */
int coolchic_backward(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image,
                      const float* latents, const float* params, int64_t step, int32_t relax,
                      int32_t use_stored, float grad_scale, float* grad_latents,
                      float* grad_params, void* workspace, size_t workspace_bytes, void* stream);

/* Rate-distortion of the current state (Sec. IV-A, Eq. 10), blocking: relax = CC_RELAX_HARD
 * evaluates the quantised latents (Eq. 12), CC_RELAX_NOISE the training proxy at `step`.
 *   rd_out [host] one record. */
int coolchic_rate_distortion(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image,
                             const float* latents, const float* params, int64_t step,
                             int32_t relax, cc_rd_t* rd_out, void* workspace,
                             size_t workspace_bytes, void* stream);

/* Rate-distortion evaluation that allocates nothing (the paper has no counterpart; this is a
 * library service).  Same computation and result as coolchic_rate_distortion, blocking, but
 * without a workspace argument: for callers that cannot call cudaMalloc, such as a process whose
 * device memory is owned entirely by its own pool, or code running while another thread of the
 * process holds a stream in global-mode capture (where cudaMalloc is illegal).
 *   Scratch: a 32 MiB array compiled into the library, held on every GPU that loads it until exit.
 *   Images that need more (above about 1.4 million pixels; 1024 x 1024 fits) are rejected with
 *   CC_ERR_WORKSPACE.  The first call on a device looks up the array's device address (with that
 *   device current); make it before any stream capture begins.  Calls share the array, so calls
 *   that overlap on the GPU race; nothing needs clearing between calls (each call writes every
 *   byte it reads).  rd_out [host].  Calls no allocating routine. */
int coolchic_rate_distortion_noalloc(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image,
                                     const float* latents, const float* params, int64_t step,
                                     int32_t relax, cc_rd_t* rd_out, void* stream);

/* Decoder (Sec. III): from integer latents q (the hard-quantised grids) and the parameters,
 *   - the integer entropy model: a fixed-point ARM (weights rint(256 w), 8 fractional bits,
 *     64-bit accumulation, floor shifts) and an integer Laplace CDF with 16-bit total mass,
 *     giving prob_q16[i] = max(1, C(256 q + 128 - mu_q) - C(256 q - 128 - mu_q)), bit-exact and
 *     platform-independent (motivated by Sec. III-A2);
 *   - the reconstruction x^ = synthesis(upsampling(q)) in FP32, clamped to [0, 1].
 *   q [device] N int32; params [device]; image_out [device, nullable] 3*H*W FP32;
 *   prob_q16 [device, nullable] N uint32; mu_q, logb_q [device, nullable] N int32 each. */
int coolchic_decode_image(const cc_arch_t* arch, const int32_t* q, const float* params,
                          float* image_out, uint32_t* prob_q16, int32_t* mu_q, int32_t* logb_q,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Measurement hooks (no counterpart in the paper; used by benchmarks).  While enabled, every
 * launch of the kernel `kernel_id` (CC_KERNEL_*) made by this library is bracketed by two CUDA
 * events recorded on the launch stream, up to `max_launches` launches (the events are created
 * here, on the current device).  Not for use under stream capture.  coolchic_timing_collect()
 * synchronises on the recorded events and returns the summed duration in milliseconds and the
 * number of timed launches; coolchic_timing_disable() destroys the events.  Returns CC_ERR_ARG
 * for an unknown id, CC_ERR_CUDA if event creation fails. */
#define CC_KERNEL_ARM 0      /* entropy model forward + adjoint */
#define CC_KERNEL_SYN_BWD 1  /* synthesis adjoint               */
#define CC_KERNEL_CONV 2     /* residual convs + distortion     */
#define CC_KERNEL_SYN_FWD 3  /* synthesis forward               */
#define CC_KERNEL_UP_FWD 4   /* upsampling stages 3..2 (one bracket around their two launches;
                                stages 6..4 run inside the entropy-model launch) */
#define CC_KERNEL_UP_ADJ 5   /* upsampling adjoint stages 1..6 (one bracket around the six)  */
#define CC_KERNEL_GATHER 6   /* latent-gradient gather + latent Adam (in encoder iterations the
                                same launch also reduces the parameter gradients, takes the
                                parameters' Adam step and writes the loss record) */
int coolchic_timing_enable(int32_t kernel_id, int32_t max_launches);
int coolchic_timing_collect(double* total_ms, int64_t* launches);
int coolchic_timing_disable(void);

/* Throughput ceiling of one arithmetic pipe on the current device (no counterpart in the paper;
 * the denominators of the benchmark's roofline fractions).  Blocking.  Runs a kernel that fills
 * every SM with independent dependency chains of one instruction kind for at least 2 ms per
 * launch, times 3 launches with CUDA events on `stream` and returns the best rate in TFLOP/s:
 *   CC_PEAK_FP32_FMA  FP32 fused multiply-add (2 FLOP each) on the SIMT pipe;
 *   CC_PEAK_TF32_MMA  warp-level tensor-core mma.sync.m16n8k8 with TF32 operands and FP32
 *                     accumulation (2 x 16 x 8 x 8 FLOP each), the instruction the entropy
 *                     model and the synthesis adjoint issue.
 *   sink        [device] 4 writable bytes (never written in practice; keeps the work alive).
 *   tflops_out  [host] the measured rate; ms_out [host, nullable] the duration of that launch.
 * Returns CC_ERR_ARG for an unknown pipe or a NULL pointer, CC_ERR_CUDA if a launch fails. */
#define CC_PEAK_FP32_FMA 0
#define CC_PEAK_TF32_MMA 1
int coolchic_measure_peak(int32_t which, float* sink, double* tflops_out, double* ms_out, void* stream);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* coolchic_last_error(void);

/* Failure-detection test hook (no counterpart in the paper).  While `on` is non-zero, entropy-model
 * launches made from then on (not the replay of a graph captured before) withhold the commit of
 * their first tensor-core MMA group, so that every wait on its completion runs out after about a
 * second: the kernel then frees its Tensor Memory and ends, the loss record of the call is NaN, and
 * the blocking coolchic_rate_distortion returns CC_ERR_TIMEOUT; the context stays usable.  No fault,
 * trap or hang is involved.  Returns CC_OK. */
int coolchic_test_inject_stall(int32_t on);

/* Library version string. */
const char* coolchic_version(void);

#ifdef __cplusplus
}
#endif
#endif /* COOLCHIC_H */
