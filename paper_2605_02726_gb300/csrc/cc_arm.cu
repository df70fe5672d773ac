// Entropy model of the encoder step (Sec. III-A, Eqs. 2-5, 9, 11) and its adjoint, on the
// 5th-generation tensor cores.
//
// Per latent: the 16 causal neighbours of the relaxed latents (zero outside the grid), the IFCE of
// grids 0..2 on nearest-neighbour co-located coarser values, the ARM MLP 20 -> 16 -> 16 -> 2 with
// ReLU plus the linear stabilizer, log-scale clamped to [-5, 5], Laplace interval mass and rate
// -log2 max(P, 2^-16).  Adjoint: dL/dbits = lambda/(HW) gives dmu, dlogb, then the MLP adjoint
// gives dL/dc; context gradients are written as 16 planes dS[n][i] and gathered by their source
// latent later (fixed order, no atomics).
//
// Work unit: a tile of 128 consecutive latents, one per thread of a 128-thread group (a CTA is one
// per SM and holds four groups, three with hyperlatents).  The dense products of
// a tile run as tcgen05 MMAs with M = 128 (the tile's latents): the activation operand A in Tensor
// Memory (each thread stores its own row), the weights B in shared memory in the canonical
// K-major layout, the accumulator in Tensor Memory:
//   D1 = c  [128 x 24] . [W1 | b1 ; Ws]^T   (N = 32: 16 hidden pre-activations, 2 stabilizer outputs)
//   D2 = h1 [128 x 16] . W2^T               (N = 16)
//   adjoint:  DH1 = da2 [128 x 16] . W2      DC = [da1 | dmu | dlogb] [128 x 24] . [W1 ; Ws]
//             (N = 32, 20 used)
// Every product is split x = hi + lo (hi = the 10 explicit mantissa bits a TF32 operand carries,
// lo = x - hi) and accumulated as Ahi.Bhi + Alo.Bhi + Ahi.Blo, which keeps FP32-level accuracy.
// One thread of the group issues a tile's MMAs and commits them to the group's mbarrier; every
// thread of the group then reads its
// own row of the accumulator with tcgen05.ld and does the element-wise work (bias, ReLU, the
// 16 -> 2 output layer, the Laplace mass and its derivatives) in FP32 on its own latent.
//
// Parameter gradients are sums over latents of outer products, i.e. GEMMs with K = latents:
// each warp writes its 32 latents' factors transposed into a private [feature][latent] shared
// tile and runs 10 m16n8 output tiles of mma.sync (TF32, hi/lo) over K = 32: W1 and b1, W2, b2, Ws
// and b3 = bs, W3, the IFCE weights.  The accumulators stay in the group's spare Tensor Memory
// columns between work units (loaded for the gradient phase, stored after it), so that they hold
// no registers during the rest of the tile.  The tile holds 72 feature rows and is filled twice
// per work unit (the gradient factors with the context, then the same gradient factors with h1,
// h2 and the IFCE inputs), which keeps the shared memory of a CTA within its 227 KB.
// The warps' accumulators are added in a fixed order at the end: one partial gradient per CTA.
//
// Every wait on the mbarrier is bounded (about a second); a group whose wait runs out stops, waits
// (again bounded) for its MMAs in flight, the CTA frees its Tensor Memory and writes a NaN rate
// partial and sets the status word, so that the loss of the call is NaN instead of the GPU hanging.
//
// With hyperlatent grids (Sec. III-A3, Eq. 6; the HYPER instantiation), their latents are coded
// like the others (spatial context only), and the IFCEs of grids 0..2 take three more inputs, the
// co-located hyperlatents; their gradients go to IFCE-input planes nin..nin+2 of the grid, their
// weights' gradients to entries 756..791 of the CTA's partial row (an 11th gradient tile).
//
// The first CTA also computes the coarse forward upsampling stages 6..4 (it needs none of the
// entropy model's results, and the other CTAs take the latents first), so that they cost no launch.
#include "cc_kernels.h"
#include "cc_mma.cuh"
#include "cc_tc.cuh"
#include "cc_upfwd.cuh"

namespace cc {
namespace {

constexpr int kT = 128;  // threads of a group = latents per tile = MMA M
// One CTA per SM of kGroups groups of 128 threads (four warps, one per Tensor Memory lane
// quarter); each group works through its own tiles with its own 128 Tensor Memory columns and
// mbarrier, and the groups share the weights in shared memory.  (Several CTAs per SM each
// allocating Tensor Memory cost about 2.7 us per extra CTA at launch; one CTA allocates once.)
template <bool HY>
constexpr int kGroups = HY ? 3 : 4;  // (the hyperlatent form needs more registers per thread)
constexpr uint32_t kTmemCols = 512;
// Tensor Memory columns: the A operand's hi and lo copies (at most 24 columns each) at 0 and 32,
// the accumulator of the tile's products (each in turn, at most 32 columns) at 96, and in the
// columns left over (24..31, 56..87) the parameter-gradient tiles 0..9 of this thread, kept there
// between work units so that they hold no registers outside the gradient phase
constexpr uint32_t TM_AH = 0, TM_AL = 32, TM_D = 96;
constexpr int kTmTiles = 10;  // gradient tiles kept in Tensor Memory (an 11th stays in registers)
__device__ __forceinline__ uint32_t tm_acc_col(int pair) { return pair == 0 ? 24u : 56u + 8u * (pair - 1); }
constexpr long long kWaitLimit = 1ll << 31;                         // clock cycles (about 1 s)

// Shared memory (dynamic), byte offsets.  B operands (weights) are K-major [N][K], a hi and a lo
// copy each.
// B1 and B4 are N = 32 operands whose rows 24..31 (accumulator columns 24..31) are never used: only
// rows 0..23 are stored (leading byte offset 24 * 16), so the MMA reads rows 24..31 of a K chunk from
// rows 0..7 of the next one (of the next buffer, for the last chunk), and those columns hold
// whatever results; this keeps a CTA's shared memory small enough for four CTAs per SM.
constexpr int B1_N = 32, B1_K = 24;  // rows 0..15: W1 with b1 at k = 20; rows 16, 17: Ws; 18..23 zero
constexpr int B2_N = 16, B2_K = 16;  // W2
constexpr int B3_N = 16, B3_K = 16;  // W2^T
constexpr int B4_N = 32, B4_K = 24;  // [W1^T | Ws^T]: row f, k < 16: W1[k][f], k = 16, 17: Ws[k-16][f]
constexpr int B14_ROWS = 24;         // stored rows of B1 and B4
constexpr uint32_t B1_BYTES = B14_ROWS * B1_K * 4, B2_BYTES = B2_N * B2_K * 4, B3_BYTES = B3_N * B3_K * 4,
                   B4_BYTES = B14_ROWS * B4_K * 4;
constexpr int kSld = 36;                                  // staging row stride (32 latents + 4)
constexpr uint32_t SM_B1 = 0, SM_B2 = SM_B1 + 2 * B1_BYTES, SM_B3 = SM_B2 + 2 * B2_BYTES,
                   SM_B4 = SM_B3 + 2 * B3_BYTES, SM_ST = SM_B4 + 2 * B4_BYTES;
// misc floats: IFCE weights and biases in flat parameter order, W3 [2][16], b2, Ws [2][20], b3 + bs,
// then (hyperlatents) the IFCE weights of the hyperlatent inputs [k][o][q]
constexpr int MS_IF = 0, MS_W3 = 72, MS_B2 = 104, MS_WS = 120, MS_OB = 160, MS_IFH = 164;
// Layout of one instantiation: staging rows per warp (the IFCE inputs take one more 8-row block
// with hyperlatents), gradient tiles, shared memory
template <bool HY>
struct ArmLayout {
    static constexpr int st_rows = HY ? 80 : 72;
    static constexpr uint32_t st_bytes = st_rows * kSld * 4;
    static constexpr int warps = kGroups<HY> * kT / 32;
    static constexpr uint32_t misc = SM_ST + warps * st_bytes;
    static constexpr int ms_n = MS_IFH + (HY ? po::ifce_h_n : 0);
    static constexpr uint32_t total = misc + ms_n * 4;
    static constexpr int tiles = HY ? 11 : 10;
    static_assert(st_bytes % 16 == 0, "16-byte alignment of the staging tiles");
    static_assert(total + 2048 <= 227 * 1024, "shared memory of one CTA");
};
static_assert(SM_ST % 16 == 0, "16-byte alignment of the staging tiles");

// Staging rows of a warp's [feature][latent] tile, first fill (gradient side U, activation side V):
//   U: 0..15 da1, 16..31 da2, 32 dmu, 33 dlogb, 34 + 4k + o: IFCE output gradient o of grid k
//      (zero unless the latent is on grid k), 46, 47 zero
//   V: 48..71 c (features 0..19, 68 = one, 69..71 zero)
// second fill: 0..15 h2, 16..47 as before, 48..63 h1, then the IFCE inputs: 64..69 r0..r5,
// 70 one, 71 zero; with hyperlatents 64..69 r0..r5, 70..72 the three hyperlatent inputs, 73 one,
// 74..79 zero.
constexpr int R_DA1 = 0, R_DA2 = 16, R_U2 = 32, R_C = 48;
constexpr int R_H2 = 0, R_H1 = 48, R_R = 64;

// Parameter index of gradient tile T, row, column (-1: padding); with hyperlatents, an index
// past po::total stands for entry (index - po::total + 756) of the CTA's partial row.
//   tiles 0-2: da1 x c (rows: hidden unit, columns: context feature; c[20] = 1 gives b1)
//   tiles 3-4: da2 x h1;  tile 5: da2 x c[16..23] (column 4, c[20] = 1: b2)
//   tiles 6-7: c[0..15], c[16..23] x (dmu, dlogb, ...) (rows: context feature, columns: output;
//              the transposed form, so that these two-row products take two tiles, not three)
//   tile 8: h2 x (dmu, dlogb, ...);  tiles 9(-10): IFCE output gradients x IFCE inputs
template <bool HY>
__device__ int wgrad_index(int T, int row, int col) {
    if (T <= 2) {  // da1 x c
        const int f = T * 8 + col;
        return f < 20 ? po::arm_w1 + row * 20 + f : (f == 20 ? po::arm_b1 + row : -1);
    }
    if (T <= 4) return po::arm_w2 + row * 16 + (T - 3) * 8 + col;  // da2 x h1
    if (T == 5) return col == 4 ? po::arm_b2 + row : -1;            // da2 x one
    if (T <= 7) {                                                   // c x (dmu, dlogb)
        if (col >= 2 || (T == 7 && row >= 8)) return -1;
        const int f = (T - 6) * 16 + row;
        return f < 20 ? po::arm_ws + col * 20 + f : (f == 20 ? po::arm_b3 + col : -1);
    }
    if (T == 8) return col < 2 ? po::arm_w3 + col * 16 + row : -1;  // h2 x (dmu, dlogb)
    if (row < 2 || row >= 14) return -1;  // T == 9 (10): IFCE output gradients x IFCE inputs
    const int k = (row - 2) >> 2, o = (row - 2) & 3, nin = ifce_nin(k);
    const int j = (T - 9) * 8 + col;  // column of the IFCE-input block
    if (j < nin) return ifce_w_off(k) + o * nin + j;
    if (HY && j >= 6 && j < 6 + kNH) return po::ifce_h + (k * kF + o) * kNH + (j - 6);
    if (j == (HY ? 6 + kNH : 6)) return ifce_b_off(k) + o;
    return -1;
}

// The coarse forward upsampling stages of CTA 0, out of line.
__device__ __noinline__ void coarse_upsampling(const ArmArgs& a, float* sm, int cap) {
#pragma unroll 1
    for (int q = 0; q < kUpArmStages; ++q) up_fwd_stage_cta(a.upc[q], sm, cap);
}

// hi = the TF32 part of x, lo = x - hi (exact)
__device__ __forceinline__ void split_f(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

// This thread's row (K values, K a multiple of 8) of the A operand, hi and lo copies, into Tensor
// Memory (t_row: this warp's lanes, column 0); complete for the warp on return.
template <int K>
__device__ __forceinline__ void store_a(uint32_t t_row, const float* v) {
#pragma unroll
    for (int q = 0; q < K / 8; ++q) {
        float h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split_f(v[8 * q + e], h[e], l[e]);
        tmem_st8(t_row + TM_AH + 8 * q, h);
        tmem_st8(t_row + TM_AL + 8 * q, l);
    }
    tmem_wait_st();
}

// D = A . B^T over K (multiple of 8) for the three hi/lo passes, A from Tensor Memory; one
// thread.  The B descriptors are built once; a k-step advances their start-address field
// (address / 16, no carry out of it: shared memory stays below 256 KB).
template <int ROWS, int K>
__device__ __forceinline__ void mma_group(uint32_t tmem, uint32_t sB, uint32_t idesc) {
    constexpr uint32_t b_lbo = ROWS * 16, b_bytes = ROWS * K * 4;
    const uint64_t bh = umma_desc(sB, b_lbo, 128), bl = umma_desc(sB + b_bytes, b_lbo, 128);
#pragma unroll
    for (int ks = 0; ks < K / 8; ++ks) {
        const uint64_t bo = (uint64_t)(ks * 2 * b_lbo >> 4);
        umma_tf32_ts(tmem + TM_D, tmem + TM_AH + 8 * ks, bh + bo, idesc, ks > 0 ? 1u : 0u);
        umma_tf32_ts(tmem + TM_D, tmem + TM_AL + 8 * ks, bh + bo, idesc, 1u);
        umma_tf32_ts(tmem + TM_D, tmem + TM_AH + 8 * ks, bl + bo, idesc, 1u);
    }
}

// The gradient tiles 0..9 of this thread from / to Tensor Memory (two tiles per 8 columns).
template <int NT>
__device__ __forceinline__ void acc_from_tmem(uint32_t t_row, float (&acc)[NT][4]) {
    uint32_t r[kTmTiles * 4];
#pragma unroll
    for (int p = 0; p < kTmTiles / 2; ++p) {
        uint32_t q[8];
        tmem_ld8_nowait(t_row + tm_acc_col(p), q);
#pragma unroll
        for (int e = 0; e < 8; ++e) r[8 * p + e] = q[e];
    }
    tmem_wait_ld(r);
#pragma unroll
    for (int T = 0; T < kTmTiles; ++T)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[T][e] = __uint_as_float(r[4 * T + e]);
}
template <int NT>
__device__ __forceinline__ void acc_to_tmem(uint32_t t_row, const float (&acc)[NT][4]) {
#pragma unroll
    for (int p = 0; p < kTmTiles / 2; ++p) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = acc[2 * p + (e >> 2)][e & 3];
        tmem_st8(t_row + tm_acc_col(p), v);
    }
    tmem_wait_st();
}

template <int PASS, bool HY>
__device__ __forceinline__ void arm_body(const ArmArgs& a, int cta, int ncta) {
    constexpr bool BWD = pass_bwd(PASS);
    constexpr bool LOAD = PASS == PASS_BWD_LOAD;
    using LY = ArmLayout<HY>;
    constexpr int kTiles = LY::tiles;
    constexpr uint32_t ST_BYTES = LY::st_bytes;
    constexpr int kRR = HY ? 16 : 8;        // rows of the IFCE-input block
    constexpr int kOneCol = HY ? 6 + kNH : 6;  // its column of ones
    constexpr int NG = kGroups<HY>, NT = NG * kT, NW = NT / 32;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sMisc = reinterpret_cast<float*>(smem + LY::misc);
    __shared__ Geom g;
    __shared__ float rcp_w[kG];
    __shared__ __align__(8) uint64_t s_mbar[NG];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int grp = wid >> 2, gtid = tid & (kT - 1);  // group, thread (= latent row) in the group
    float* st = reinterpret_cast<float*>(smem + SM_ST + wid * ST_BYTES);  // this warp's staging tile

    if (tid == 0) g = a.g;
    if (tid < kG) rcp_w[tid] = a.g.w[tid] > 0 ? 1.f / (float)a.g.w[tid] : 0.f;
    const bool hyper = HY && a.g.nh > 0;  // this job has hyperlatent grids
    // parameters staged through the staging area (free until the coarse stages and the first tile)
    const float* P = stage_params(a.params, 0, po::arm_block, reinterpret_cast<float*>(smem + SM_ST));
    const float* Ph = nullptr;  // the hyperlatent IFCE weights, at their absolute offsets
    if (hyper)
        Ph = stage_params(a.params, po::ifce_h, po::ifce_h_n, reinterpret_cast<float*>(smem + SM_ST) + po::arm_block);
    // B operands: element (n, k) of each, hi and lo
    for (int e = tid; e < B14_ROWS * B1_K; e += NT) {
        const int n = e / B1_K, k = e - n * B1_K;
        float v = 0.f;
        if (n < 16) v = k < 20 ? P[po::arm_w1 + n * 20 + k] : (k == 20 ? P[po::arm_b1 + n] : 0.f);
        else if (n < 18 && k < 20) v = P[po::arm_ws + (n - 16) * 20 + k];
        float h, l;
        split_f(v, h, l);
        const uint32_t off = SM_B1 + kmajor_off(B14_ROWS, n, k);
        *reinterpret_cast<float*>(smem + off) = h;
        *reinterpret_cast<float*>(smem + off + B1_BYTES) = l;
    }
    for (int e = tid; e < 16 * 16; e += NT) {
        const int n = e >> 4, k = e & 15;
        float h, l;
        split_f(P[po::arm_w2 + n * 16 + k], h, l);  // B2[n][k] = W2[n][k]
        uint32_t off = SM_B2 + kmajor_off(B2_N, n, k);
        *reinterpret_cast<float*>(smem + off) = h;
        *reinterpret_cast<float*>(smem + off + B2_BYTES) = l;
        off = SM_B3 + kmajor_off(B3_N, k, n);  // B3[k][n] = W2[n][k]
        *reinterpret_cast<float*>(smem + off) = h;
        *reinterpret_cast<float*>(smem + off + B3_BYTES) = l;
    }
    for (int e = tid; e < B14_ROWS * B4_K; e += NT) {
        const int n = e / B4_K, k = e - n * B4_K;  // B4[f][o] = W1[o][f], B4[f][16 + o] = Ws[o][f]
        float v = 0.f;
        if (n < 20) v = k < 16 ? P[po::arm_w1 + k * 20 + n] : (k < 18 ? P[po::arm_ws + (k - 16) * 20 + n] : 0.f);
        float h, l;
        split_f(v, h, l);
        const uint32_t off = SM_B4 + kmajor_off(B14_ROWS, n, k);
        *reinterpret_cast<float*>(smem + off) = h;
        *reinterpret_cast<float*>(smem + off + B4_BYTES) = l;
    }
    for (int j = tid; j < LY::ms_n; j += NT) {
        float v;
        if (j < MS_W3) v = P[po::if_w0 + j];
        else if (j < MS_B2) v = P[po::arm_w3 + (j - MS_W3)];
        else if (j < MS_WS) v = P[po::arm_b2 + (j - MS_B2)];
        else if (j < MS_OB) v = P[po::arm_ws + (j - MS_WS)];
        else if (j < MS_IFH) v = j - MS_OB < 2 ? P[po::arm_b3 + (j - MS_OB)] + P[po::arm_bs + (j - MS_OB)] : 0.f;
        else v = hyper ? Ph[po::ifce_h + (j - MS_IFH)] : 0.f;
        sMisc[j] = v;
    }
    const uint32_t mbar = smem_u32(&s_mbar[grp]);
    if (tid < NG) {
        mbar_init(smem_u32(&s_mbar[tid]), 1);
        mbar_init_fence();
    }
    if (wid == 0) tmem_alloc(smem_u32(&s_tmem), kTmemCols);
    fence_async_smem();  // the B operands, for the tensor core
    tc_fence_before();
    __syncthreads();  // (the staged parameters are dead from here: the staging area is reused)
    tc_fence_after();
    const uint32_t tmem = s_tmem + (uint32_t)(grp * kT);  // this group's 128 columns
    const uint32_t t_row = tmem + ((uint32_t)((wid & 3) * 32) << 16);  // this warp's lanes
    const uint32_t sbase = smem_u32(smem);  // (B operand descriptors)
    uint32_t phase = 0;
    bool bad = false;

    // CTA 0 computes the coarse forward upsampling stages (it takes no tiles when there are other
    // CTAs), staged through the staging area; each stage ends with a barrier.
    //   Tiles, over the V = C * NG groups of the C CTAs: no group takes more than
    // Q = ceil(tiles / V); the groups of CTAs 1.. take tiles [0, U1) round-robin
    // (U1 = min(tiles, Q * (V - NG))) and the groups of CTA 0 only the rest.
    const int64_t N = a.N;
    const int n_tiles = (int)((N + kT - 1) / kT);
    int t_first = cta * NG + grp, t_step = ncta * NG, t_end = n_tiles;
    if (a.upc_on) {
        if (cta == 0) coarse_upsampling(a, reinterpret_cast<float*>(smem + SM_ST), (int)(NW * ST_BYTES / 4));
        if (ncta > 1) {
            const int64_t v = (int64_t)ncta * NG;
            const int64_t q_max = (n_tiles + v - 1) / v;
            const int u1 = (int)std::min<int64_t>(n_tiles, q_max * (v - NG));
            if (cta > 0) {
                t_first = (cta - 1) * NG + grp;
                t_step = (ncta - 1) * NG;
                t_end = u1;
            } else {
                t_first = u1 + grp;
                t_step = NG;
            }
        }
    }
    if (BWD) {  // constant staging rows (the ones that no fill overwrites)
        st[46 * kSld + lane] = 0.f;
        st[47 * kSld + lane] = 0.f;
    }
    // gradient tile 10 (hyperlatent IFCE weights) in registers, tiles 0..9 in Tensor Memory
    float acc_h[4] = {0.f, 0.f, 0.f, 0.f};
    if (BWD) {
        const float zero[kTmTiles][4] = {};
        acc_to_tmem(t_row, zero);
    }
    float rate_acc = 0.f;
    const float4* W3v = reinterpret_cast<const float4*>(sMisc + MS_W3);  // W3 [2][16] as 8 float4
    const float4* B2v = reinterpret_cast<const float4*>(sMisc + MS_B2);  // b2 as 4 float4

    // one MMA group's completion, as one decision of the whole warp
    auto wait_mma = [&]() {
        bool ok = mbar_wait_bounded(mbar, phase, kWaitLimit);
        phase ^= 1u;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) bad = true;
        tc_fence_after();
    };
    // barrier of the group before an MMA group: Tensor Memory stores and loads of its four warps
    // ordered before it; true when some thread of the group has given up
    auto pre_mma = [&]() {
        tc_fence_before();
        return group_sync_or(1 + grp, bad);
    };

    for (int tile = t_first; tile < t_end; tile += t_step) {
        const int64_t i0 = (int64_t)tile * kT + gtid;
        const bool valid = i0 < N;
        const int64_t i = valid ? i0 : N - 1;
        const int k = grid_of(g, i);
        const int li = (int)(i - g.off[k]);
        const int w = g.w[k];
        int r = __float2int_rz(__int2float_rn(li) * rcp_w[k]);
        r -= (r * w > li) ? 1 : 0;
        r += ((r + 1) * w <= li) ? 1 : 0;
        const int c = li - r * w;
        // ---- context: 16 neighbours, IFCE inputs and outputs, the constant one
        float cx[24];
        const float* yk = a.yt + g.off[k] + (int64_t)r * w + c;
#pragma unroll
        for (int n = 0; n < kNCtx; ++n) {
            const int dy = ctx_dy(n), dx = ctx_dx(n);
            cx[n] = (r + dy >= 0 && c + dx >= 0 && c + dx < w) ? __ldg(yk + dy * w + dx) : 0.f;
        }
        const int nin = ifce_nin(k);  // main-grid IFCE inputs (0 on grids 3.. and on hyperlatent grids)
        float rin[6 + (HY ? kNH : 0)];  // main inputs 0..5 (zero past nin), hyperlatent inputs 6..8
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            rin[j] = 0.f;
            if (j < nin) {
                const int gj = k + 1 + j;
                const int rr = min(r >> (j + 1), g.h[gj] - 1), cc = min(c >> (j + 1), g.w[gj] - 1);
                rin[j] = __ldg(a.yt + g.off[gj] + (int64_t)rr * g.w[gj] + cc);
            }
        }
        if constexpr (HY) {
#pragma unroll
            for (int q = 0; q < kNH; ++q) {
                rin[6 + q] = 0.f;
                if (hyper && nin > 0) {
                    const int gq = kL + q, sh = kHB + q - k;
                    const int rr = min(r >> sh, g.h[gq] - 1), cc = min(c >> sh, g.w[gq] - 1);
                    rin[6 + q] = __ldg(a.yt + g.off[gq] + (int64_t)rr * g.w[gq] + cc);
                }
            }
        }
        {
            const int kk = k < kNIfce ? k : 0;
            const int wo = ifce_w_off(kk) - po::if_w0, bo = ifce_b_off(kk) - po::if_w0;
#pragma unroll
            for (int o = 0; o < kF; ++o) {
                float f = 0.f;
                if (nin > 0) {
                    f = sMisc[MS_IF + bo + o];
#pragma unroll
                    for (int j = 0; j < 6; ++j)
                        if (j < nin) f = fmaf(sMisc[MS_IF + wo + o * nin + j], rin[j], f);
                    if constexpr (HY) {
#pragma unroll
                        for (int q = 0; q < kNH; ++q) f = fmaf(sMisc[MS_IFH + (kk * kF + o) * kNH + q], rin[6 + q], f);
                    }
                }
                cx[kNCtx + o] = f;
            }
        }
        cx[20] = 1.f;
        cx[21] = cx[22] = cx[23] = 0.f;
        if (BWD) {
#pragma unroll
            for (int f = 0; f < 24; ++f) st[(R_C + f) * kSld + lane] = cx[f];
        }

        float a1[16], a2[16], mu, s;
        if (LOAD) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                a1[j] = a.act[(int64_t)j * N + i];
                a2[j] = a.act[(int64_t)(16 + j) * N + i];
            }
            mu = a.act[(int64_t)32 * N + i];
            s = a.act[(int64_t)33 * N + i];
        } else {
            // ---- layer 1 and the stabilizer: D = c . [W1 | b1 ; Ws]^T
            store_a<24>(t_row, cx);
            if (pre_mma()) break;
            if (gtid == 0 && !a.inject_stall) {  // (the failure-detection test hook withholds it)
                tc_fence_after();
                mma_group<B14_ROWS, B1_K>(tmem, sbase + SM_B1, umma_idesc_tf32(kT, B1_N));
                umma_commit(mbar);
            }
            wait_mma();
            float d1[32] = {};
            if (!bad) tmem_ld32(t_row + TM_D, d1);
            float h1[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                a1[j] = d1[j];
                h1[j] = fmaxf(d1[j], 0.f);
            }
            const float stab_mu = d1[16], stab_s = d1[17];
            // ---- layer 2: D = h1 . W2^T
            store_a<16>(t_row, h1);
            if (pre_mma()) break;
            if (gtid == 0) {
                tc_fence_after();
                mma_group<B2_N, B2_K>(tmem, sbase + SM_B2, umma_idesc_tf32(kT, B2_N));
                umma_commit(mbar);
            }
            wait_mma();
            float d2[16] = {};
            if (!bad) tmem_ld16(t_row + TM_D, d2);
            mu = sMisc[MS_OB] + stab_mu;
            s = sMisc[MS_OB + 1] + stab_s;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 b = B2v[q], wm = W3v[q], wsv = W3v[4 + q];
                const float bb[4] = {b.x, b.y, b.z, b.w}, m4[4] = {wm.x, wm.y, wm.z, wm.w},
                            s4[4] = {wsv.x, wsv.y, wsv.z, wsv.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * q + e;
                    a2[j] = d2[j] + bb[e];
                    const float h = fmaxf(a2[j], 0.f);
                    mu = fmaf(m4[e], h, mu);
                    s = fmaf(s4[e], h, s);
                }
            }
            if (PASS == PASS_FWD_STORE && valid) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    a.act[(int64_t)j * N + i] = a1[j];
                    a.act[(int64_t)(16 + j) * N + i] = a2[j];
                }
                a.act[(int64_t)32 * N + i] = mu;
                a.act[(int64_t)33 * N + i] = s;
            }
        }
        // ---- Laplace mass and rate
        const float logb = fminf(fmaxf(s, kLogbMin), kLogbMax);
        const LapOut L = laplace_mass(__ldg(a.yt + i), mu, logb);
        if (valid) rate_acc += -log2f(fmaxf(L.p, kPMin));
        if (!BWD) continue;

        const float dp = (valid && L.p >= kPMin) ? -a.gscale / (L.p * 0.69314718055994531f) : 0.f;
        const float dyd = dp * L.dp_dy;
        const float dmu = -dyd;
        const float ds = (s >= kLogbMin && s <= kLogbMax) ? dp * L.dp_dlogb : 0.f;
        if (valid) a.dYd[i] = dyd;
        // dA2 = (dout . W3) masked by a2 > 0
        float da2[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float4 wm = W3v[j >> 2], wsv = W3v[4 + (j >> 2)];
            const float m1 = (j & 3) == 0 ? wm.x : (j & 3) == 1 ? wm.y : (j & 3) == 2 ? wm.z : wm.w;
            const float s1 = (j & 3) == 0 ? wsv.x : (j & 3) == 1 ? wsv.y : (j & 3) == 2 ? wsv.z : wsv.w;
            da2[j] = a2[j] > 0.f ? fmaf(m1, dmu, s1 * ds) : 0.f;
            st[(R_DA2 + j) * kSld + lane] = da2[j];
        }
        st[R_U2 * kSld + lane] = dmu;
        st[(R_U2 + 1) * kSld + lane] = ds;
        // ---- dA1 = (dA2 . W2) masked by a1 > 0: D = da2 . (W2^T)^T
        store_a<16>(t_row, da2);
        if (pre_mma()) break;
        if (gtid == 0) {
            tc_fence_after();
            mma_group<B3_N, B3_K>(tmem, sbase + SM_B3, umma_idesc_tf32(kT, B3_N));
            umma_commit(mbar);
        }
        wait_mma();
        float dh1[16] = {};
        if (!bad) tmem_ld16(t_row + TM_D, dh1);
        float da1[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            da1[j] = a1[j] > 0.f ? dh1[j] : 0.f;
            st[(R_DA1 + j) * kSld + lane] = da1[j];
        }
        // ---- dC = dA1 . W1 + dout . Ws: DC = [da1 | dmu | dlogb | 0] . [W1^T | Ws^T]^T
        {
            float ua[24];
#pragma unroll
            for (int j = 0; j < 16; ++j) ua[j] = da1[j];
            ua[16] = dmu;
            ua[17] = ds;
#pragma unroll
            for (int j = 18; j < 24; ++j) ua[j] = 0.f;
            store_a<24>(t_row, ua);
        }
        if (pre_mma()) break;
        if (gtid == 0) {
            tc_fence_after();
            mma_group<B14_ROWS, B4_K>(tmem, sbase + SM_B4, umma_idesc_tf32(kT, B4_N));
            umma_commit(mbar);
        }
        wait_mma();
        float dc[32] = {};
        if (!bad) tmem_ld32(t_row + TM_D, dc);
        if (valid) {
#pragma unroll
            for (int f = 0; f < kNCtx; ++f) a.dS[(int64_t)f * N + i] = dc[f];
        }
        // IFCE: input gradients dr_j = sum_o W_k[o][j] df[o]; output gradients staged by grid
#pragma unroll
        for (int kk = 0; kk < kNIfce; ++kk)
#pragma unroll
            for (int o = 0; o < kF; ++o) st[(R_U2 + 2 + 4 * kk + o) * kSld + lane] = k == kk ? dc[16 + o] : 0.f;
        if (nin > 0 && valid) {
            float* dR = k == 0 ? a.dR0 : (k == 1 ? a.dR1 : a.dR2);
            const int64_t nk = (int64_t)g.h[k] * g.w[k];
            const int wo = ifce_w_off(k) - po::if_w0;
#pragma unroll
            for (int j = 0; j < 6; ++j)
                if (j < nin) {
                    float v = 0.f;
#pragma unroll
                    for (int o = 0; o < kF; ++o) v = fmaf(sMisc[MS_IF + wo + o * nin + j], dc[16 + o], v);
                    dR[(int64_t)j * nk + li] = v;
                }
            if constexpr (HY) {
                if (hyper) {  // planes nin..nin+2: the hyperlatent inputs
#pragma unroll
                    for (int q = 0; q < kNH; ++q) {
                        float v = 0.f;
#pragma unroll
                        for (int o = 0; o < kF; ++o) v = fmaf(sMisc[MS_IFH + (k * kF + o) * kNH + q], dc[16 + o], v);
                        dR[(int64_t)(nin + q) * nk + li] = v;
                    }
                }
            }
        }
        __syncwarp();
        // ---- parameter-gradient tiles over K = 32 latents (four k-steps of 8), fragments by ldmatrix:
        // an A fragment (16 rows) is matrices (rows 0-7, k 0-3), (8-15, 0-3), (0-7, 4-7), (8-15, 4-7);
        // a pair of B fragments (8 rows each) is (rows of the first, k 0-3), (first, 4-7),
        // (second, 0-3), (second, 4-7).  The three hi/lo passes of every tile are issued pass by
        // pass, so that no MMA waits on the one just before it.
        {
            float acc[kTiles][4];
            acc_from_tmem(t_row, acc);
            if constexpr (HY) {
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[kTiles - 1][q] = acc_h[q];
            }
            const int mi = lane >> 3, ri = lane & 7;
            auto afrag = [&](const float* arow, int row0) {
                uint32_t rr[4];
                ldsm_x4(rr, arow + row0 * kSld);
                AFrag f;
#pragma unroll
                for (int q = 0; q < 4; ++q) split_u(rr[q], f.h[q], f.l[q]);
                return f;
            };
            auto bpair = [&](const float* brow, int row0a, int row0b, AFrag& fa, AFrag& fb) {  // (b0, b1) in h[0..1], l[0..1]
                uint32_t rr[4];
                ldsm_x4(rr, brow + ((mi >> 1) ? row0b : row0a) * kSld);
                split_u(rr[0], fa.h[0], fa.l[0]);
                split_u(rr[1], fa.h[1], fa.l[1]);
                split_u(rr[2], fb.h[0], fb.l[0]);
                split_u(rr[3], fb.h[1], fb.l[1]);
            };
            // two B fragments (rows r..r+7 and r+8..r+15) as one A fragment of rows r..r+15, and
            // the first eight rows of an A fragment as a B fragment (the register layouts coincide)
            auto stack_b = [](const AFrag& x, const AFrag& y) {
                AFrag f;
                f.h[0] = x.h[0], f.h[1] = y.h[0], f.h[2] = x.h[1], f.h[3] = y.h[1];
                f.l[0] = x.l[0], f.l[1] = y.l[0], f.l[2] = x.l[1], f.l[3] = y.l[1];
                return f;
            };
            auto a_as_b = [](const AFrag& u) {
                AFrag f = u;
                f.h[1] = u.h[2], f.l[1] = u.l[2];
                return f;
            };
            // first fill: the gradient factors x the context (tiles 0-2, 5, 6-7)
#pragma unroll 1
            for (int ks = 0; ks < 4; ++ks) {
                const int k0 = ks * 8;
                const float* arow = st + (ri + (mi & 1) * 8) * kSld + k0 + (mi >> 1) * 4;
                const float* brow = st + ri * kSld + k0 + (mi & 1) * 4;
                const AFrag U0 = afrag(arow, R_DA1), U1 = afrag(arow, R_DA2), U2 = afrag(arow, R_U2);
                AFrag V0, V1, V2, Vx;
                bpair(brow, R_C, R_C + 8, V0, V1);
                bpair(brow, R_C + 16, R_C + 16, V2, Vx);
                const AFrag C01 = stack_b(V0, V1), C2 = stack_b(V2, Vx), U2b = a_as_b(U2);
                const AFrag* TA[6] = {&U0, &U0, &U0, &U1, &C01, &C2};
                const AFrag* TB[6] = {&V0, &V1, &V2, &V2, &U2b, &U2b};
                constexpr int TT[6] = {0, 1, 2, 5, 6, 7};
#pragma unroll
                for (int q = 0; q < 6; ++q) mma1(acc[TT[q]], TA[q]->l, TB[q]->h[0], TB[q]->h[1]);
#pragma unroll
                for (int q = 0; q < 6; ++q) mma1(acc[TT[q]], TA[q]->h, TB[q]->l[0], TB[q]->l[1]);
#pragma unroll
                for (int q = 0; q < 6; ++q) mma1(acc[TT[q]], TA[q]->h, TB[q]->h[0], TB[q]->h[1]);
            }
            __syncwarp();
            // second fill: h2, h1 and the IFCE inputs in the rows of da1 and the context
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                st[(R_H2 + j) * kSld + lane] = fmaxf(a2[j], 0.f);
                st[(R_H1 + j) * kSld + lane] = fmaxf(a1[j], 0.f);
            }
#pragma unroll
            for (int j = 0; j < 6 + (HY ? kNH : 0); ++j) st[(R_R + j) * kSld + lane] = rin[j];
            st[(R_R + kOneCol) * kSld + lane] = 1.f;
#pragma unroll
            for (int j = kOneCol + 1; j < kRR; ++j) st[(R_R + j) * kSld + lane] = 0.f;
            __syncwarp();
            // the gradient factors x h1, h2, r (tiles 3-4, 8, 9(-10))
#pragma unroll 1
            for (int ks = 0; ks < 4; ++ks) {
                const int k0 = ks * 8;
                const float* arow = st + (ri + (mi & 1) * 8) * kSld + k0 + (mi >> 1) * 4;
                const float* brow = st + ri * kSld + k0 + (mi & 1) * 4;
                const AFrag U1 = afrag(arow, R_DA2), U2 = afrag(arow, R_U2);
                AFrag H1a, H1b, H2a, H2b, Rr, Rr2;
                bpair(brow, R_H1, R_H1 + 8, H1a, H1b);
                bpair(brow, R_H2, R_H2 + 8, H2a, H2b);
                bpair(brow, R_R, R_R + (HY ? 8 : 0), Rr, Rr2);
                constexpr int NT2 = HY ? 5 : 4;
                const AFrag H2 = stack_b(H2a, H2b), U2b = a_as_b(U2);
                const AFrag* TA[5] = {&U1, &U1, &H2, &U2, &U2};
                const AFrag* TB[5] = {&H1a, &H1b, &U2b, &Rr, &Rr2};
                constexpr int TT[5] = {3, 4, 8, 9, 10};
#pragma unroll
                for (int q = 0; q < NT2; ++q) mma1(acc[TT[q]], TA[q]->l, TB[q]->h[0], TB[q]->h[1]);
#pragma unroll
                for (int q = 0; q < NT2; ++q) mma1(acc[TT[q]], TA[q]->h, TB[q]->l[0], TB[q]->l[1]);
#pragma unroll
                for (int q = 0; q < NT2; ++q) mma1(acc[TT[q]], TA[q]->h, TB[q]->h[0], TB[q]->h[1]);
            }
            acc_to_tmem(t_row, acc);
            if constexpr (HY) {
#pragma unroll
                for (int q = 0; q < 4; ++q) acc_h[q] = acc[kTiles - 1][q];
            }
        }
        __syncwarp();
    }
    bad = __syncthreads_or(bad ? 1 : 0) != 0;

    // rate partial of this CTA (NaN when a wait ran out)
    {
        float v[1] = {rate_acc};
        __shared__ float scratch[NW];
        block_sum<1>(v, scratch);
        if (tid == 0) a.rate_part[cta] = bad ? (double)__int_as_float(0x7fc00000) : (double)v[0];
        if (tid == 0 && bad && a.status) atomicOr(a.status, 1);
    }
    if (bad) {  // let any MMA still in flight finish (bounded) before the Tensor Memory is freed
        mbar_wait_bounded(mbar, phase ^ 1u, kWaitLimit);
        tc_fence_after();
    }
    float acc[kTiles][4];
    if constexpr (BWD) {
        acc_from_tmem(t_row, acc);
        if constexpr (HY) {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[kTiles - 1][q] = acc_h[q];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (wid == 0) tmem_dealloc(s_tmem, kTmemCols);
    if constexpr (BWD) {
        // the warps' gradient tiles, added in warp order
        float* sAcc = reinterpret_cast<float*>(smem + SM_ST);  // [warp][T][lane][4]
#pragma unroll
        for (int T = 0; T < kTiles; ++T)
#pragma unroll
            for (int q = 0; q < 4; ++q) sAcc[((wid * kTiles + T) * 32 + lane) * 4 + q] = acc[T][q];
        __syncthreads();
        float* gp = a.gpart + (int64_t)cta * (hyper ? po::arm_block_h : po::arm_block);
        for (int e = tid; e < kTiles * 32 * 4; e += NT) {
            const int T = e >> 7, l = (e >> 2) & 31, q = e & 3;
            const int row = (l >> 2) + (q >= 2 ? 8 : 0), col = 2 * (l & 3) + (q & 1);
            int idx = wgrad_index<HY>(T, row, col);
            if (idx < 0) continue;
            if (idx >= po::total) {  // a hyperlatent IFCE weight
                if (!hyper) continue;
                idx = po::arm_block + (idx - po::ifce_h);
            }
            float sum = 0.f;
            for (int wv = 0; wv < NW; ++wv) sum += sAcc[((wv * kTiles + T) * 32 + l) * 4 + q];
            gp[idx] = sum;
            if (idx == po::arm_b3 || idx == po::arm_b3 + 1) gp[po::arm_bs + (idx - po::arm_b3)] = sum;
        }
    }
}

template <int PASS, bool HY>
__global__ void __launch_bounds__(kGroups<HY> * kT, 1) k_arm(const __grid_constant__ ArmArgs a) {
    __shared__ ArmArgs sa;
    param_fetch(a, sa);
    arm_body<PASS, HY>(sa, blockIdx.x, gridDim.x);
}
template <int PASS, bool HY>
__global__ void __launch_bounds__(kGroups<HY> * kT, 1) k_arm_b(Batch<ArmArgs> b) {
    __shared__ ArmArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    arm_body<PASS, HY>(sa, blockIdx.x - b.cta_begin[j], b.cta_begin[j + 1] - b.cta_begin[j]);
}

template <bool HY, typename F>
void for_passes(F f) {
    f(k_arm<PASS_FWD, HY>, k_arm_b<PASS_FWD, HY>);
    f(k_arm<PASS_FWD_STORE, HY>, k_arm_b<PASS_FWD_STORE, HY>);
    f(k_arm<PASS_FWD_BWD, HY>, k_arm_b<PASS_FWD_BWD, HY>);
    f(k_arm<PASS_BWD_LOAD, HY>, k_arm_b<PASS_BWD_LOAD, HY>);
}

}  // namespace

size_t arm_smem_bytes(int pass, bool hyper) {
    (void)pass;
    return hyper ? ArmLayout<true>::total : ArmLayout<false>::total;
}

int arm_grid(int64_t N, bool hyper) {
    const int64_t groups = hyper ? kGroups<true> : kGroups<false>;
    const int64_t ctas = ((N + kT - 1) / kT + groups - 1) / groups;
    const int64_t cap = num_sms();  // one CTA per SM
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
    a.status = w.status;
    a.inject_stall = test_inject_stall();
    a.pad3_ = 0;
    return a;
}

template <bool HY>
void launch_arm_t(const Work& w, const ArmArgs& a, int pass, cudaStream_t s) {
    const size_t sm = arm_smem_bytes(pass, HY);
    const int grid = w.n_cta_arm;
    switch (pass) {
        case PASS_FWD: launch_pdl(k_arm<PASS_FWD, HY>, grid, kGroups<HY> * kT, sm, s, a); break;
        case PASS_FWD_STORE: launch_pdl(k_arm<PASS_FWD_STORE, HY>, grid, kGroups<HY> * kT, sm, s, a); break;
        case PASS_FWD_BWD: launch_pdl(k_arm<PASS_FWD_BWD, HY>, grid, kGroups<HY> * kT, sm, s, a); break;
        default: launch_pdl(k_arm<PASS_BWD_LOAD, HY>, grid, kGroups<HY> * kT, sm, s, a); break;
    }
}

void launch_arm(const Work& w, const float* params, int pass, float grad_scale, cudaStream_t s) {
    ArmArgs a = arm_args(w, params, grad_scale);
    if (pass == PASS_BWD_LOAD) a.upc_on = 0;  // the upsampled grids are still in the workspace
    if (w.g.nh > 0)
        launch_arm_t<true>(w, a, pass, s);
    else
        launch_arm_t<false>(w, a, pass, s);
}

template <bool HY>
void launch_arm_b_t(const Batch<ArmArgs>& b, int pass, cudaStream_t s) {
    const size_t sm = arm_smem_bytes(pass, HY);
    switch (pass) {
        case PASS_FWD: launch_pdl(k_arm_b<PASS_FWD, HY>, b.total_ctas, kGroups<HY> * kT, sm, s, b); break;
        case PASS_FWD_STORE: launch_pdl(k_arm_b<PASS_FWD_STORE, HY>, b.total_ctas, kGroups<HY> * kT, sm, s, b); break;
        case PASS_FWD_BWD: launch_pdl(k_arm_b<PASS_FWD_BWD, HY>, b.total_ctas, kGroups<HY> * kT, sm, s, b); break;
        default: launch_pdl(k_arm_b<PASS_BWD_LOAD, HY>, b.total_ctas, kGroups<HY> * kT, sm, s, b); break;
    }
}

void launch_arm_b(const Batch<ArmArgs>& b, int pass, bool hyper, cudaStream_t s) {
    if (hyper)
        launch_arm_b_t<true>(b, pass, s);
    else
        launch_arm_b_t<false>(b, pass, s);
}

void arm_init_attributes() {
    for_passes<false>([](auto k1, auto kb) {
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)arm_smem_bytes(0, false));
        cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)arm_smem_bytes(0, false));
    });
    for_passes<true>([](auto k1, auto kb) {
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)arm_smem_bytes(0, true));
        cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)arm_smem_bytes(0, true));
    });
}

}  // namespace cc
