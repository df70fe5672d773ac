/*
 * Cool-chic 5.0 per-iteration encoder step -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file.  It exists so that tests, the smoke check and the CPU-baseline leg of
 * the benchmark can compare the CUDA path against a slow, obviously correct
 * restatement of the method.  It shares no code, header or table with the CUDA
 * library; every constant it needs is written out here.
 *
 * What it computes (paper section / equation in brackets):
 *   - latent grids  y^(k), k = 0..L-1, shape ceil(H/2^k) x ceil(W/2^k)      [Sec. III-A1, Eq. 1]
 *   - noise relaxation  y~ = y + u, u ~ U(-1/2, 1/2) from a counter hash    [Sec. IV-C; the workload's
 *     additive uniform proxy]
 *   - the paper's proxy  y~ = s_T(s_T(y) + sigma n), n ~ N(0, 1) by Box-Muller  [Sec. IV-C, Eq. 13-14]
 *     from the same counter hash, with the linear sigma / T and cosine learning-rate schedules of
 *     the main stage and the hard-round stage with frozen latents            [Sec. IV-D, Table I]
 *   - causal spatial context s_i and inter-feature context f_i = IFCE_k(r_i)  [Sec. III-A1/A2, Eqs. 4-5]
 *   - ARM MLP + linear stabilizer -> (mu, log b)                             [Eq. 4, Eq. 9, Sec. III-C]
 *   - Laplace interval probability and rate  -log2 p                         [Eq. 3, Eq. 11]
 *   - upsampling cascade  z = f_up(y)                                        [Sec. III-B, Eq. 7]
 *   - synthesis: 1x1 MLP + stabilizer, then two residual 3x3 convs           [Sec. III-B, Eq. 8, Eq. 9]
 *   - loss  D + lambda * R / (H W)                                           [Sec. IV-A, Eq. 10]
 *   - hand-written adjoint of all of the above (transposed forward loops)
 *   - Adam                                                                   [Sec. IV-B]
 *   - hard quantisation  Q = rint                                            [Sec. IV-C, Eq. 12]
 *   - integer decode ARM and integer Laplace CDF (16-bit probabilities)       [Sec. III-A2: integer,
 *     cross-platform decoding motivates it; the fixed-point format is this project's reading]
 *   - optional hyperlatent grids (`hyper` = 1)                                 [Sec. III-A3, Eq. 6]:
 *     three more grids at 1/16, 1/32, 1/64 of the image (b = 4, L_h = L = 7, Table II, small
 *     images), entropy coded by the same ARM (spatial context only, f = 0), read by the IFCEs of
 *     grids 0..2 as three more nearest-neighbour inputs, never by the upsampling or the synthesis.
 *     Their latents follow the main grids in the latent vector; the IFCE weights of the extra
 *     inputs follow the 1415 main parameters as one block [grid k = 0..2][output o][hyper grid q].
 *
 * Parity status: the spatial context pattern, the IFCE width F = 4, the upsampling filter form,
 * the initialisation and the integer decode format are readings of a paper that leaves them open;
 * they are pinned by invariants and by an independent float64 autograd composition in the tests,
 * not by values printed in the paper ("parity unpinned" for those readings).
 *
 * Loops are plain and in the order of the definitions.  OpenMP is used only across
 * independent rows; every reduction goes through per-row partial arrays summed serially,
 * so results do not depend on the thread count.
 */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------------------------------
 * Architecture (Table II read at the MOP/HOP scale chosen for this workload).
 * ---------------------------------------------------------------------------------------- */
#define NG 7          /* L: latent grids 1/1 .. 1/64 (Table II, small images)            */
#define NCTX 16       /* spatial causal context size                                      */
#define NF 4          /* IFCE output width                                                */
#define NIFCE 3       /* grids 1/1, 1/2, 1/4 carry an IFCE (Table II)                      */
#define AIN (NCTX + NF)
#define AH 16         /* ARM hidden width, two hidden layers                              */
#define NCH 3         /* image channels                                                   */
#define SH 40         /* synthesis hidden width                                           */
#define LOGB_MIN (-5.0)
#define LOGB_MAX (5.0)
#define P_MIN (1.0 / 65536.0)
#define NH 3          /* hyperlatent grids                                                */
#define HB 4          /* the largest hyperlatent grid is 1/2^HB of the image               */

/* Flat parameter vector, all matrices row-major [out][in]. */
enum {
    O_ARM_W1 = 0, O_ARM_B1 = 320, O_ARM_W2 = 336, O_ARM_B2 = 592,
    O_ARM_W3 = 608, O_ARM_B3 = 640, O_ARM_WS = 642, O_ARM_BS = 682,
    O_IF0_W = 684, O_IF0_B = 708, O_IF1_W = 712, O_IF1_B = 732, O_IF2_W = 736, O_IF2_B = 752,
    O_UP = 756,
    O_SYN_W1 = 780, O_SYN_B1 = 1060, O_SYN_W2 = 1100, O_SYN_B2 = 1220, O_SYN_WS = 1223, O_SYN_BS = 1244,
    O_CV1_W = 1247, O_CV1_B = 1328, O_CV2_W = 1331, O_CV2_B = 1412,
    N_PARAMS = 1415,
    O_IFH = N_PARAMS,                  /* IFCE weights of the hyperlatent inputs [NIFCE][NF][NH] */
    N_PARAMS_H = N_PARAMS + NIFCE * NF * NH
};
static const int IF_W[NIFCE] = {O_IF0_W, O_IF1_W, O_IF2_W};
static const int IF_B[NIFCE] = {O_IF0_B, O_IF1_B, O_IF2_B};

/* Causal offsets (dy, dx) of the 16 spatial context values, nearest first. */
static const int CTX_DY[NCTX] = {0, -1, -1, -1, 0, -2, -1, -1, -2, -2, -2, -2, 0, -3, -1, -1};
static const int CTX_DX[NCTX] = {-1, 0, -1, 1, -2, 0, -2, 2, -1, 1, -2, 2, -3, 0, -3, 3};

/* Grids 0..NG-1 are the latent grids; with hyperlatents (nh = NH) grids NG..NG+NH-1 are the
 * hyperlatent grids, grid NG + q with the shape of latent grid HB + q. */
typedef struct {
    int H, W, nh;
    int h[NG + NH], w[NG + NH];
    int64_t off[NG + NH + 1];
} geom_t;
#define NGT(g) (NG + (g)->nh)

static void geom_init(geom_t* g, int H, int W, int hyper) {
    g->H = H;
    g->W = W;
    g->nh = hyper ? NH : 0;
    g->off[0] = 0;
    for (int k = 0; k < NG + g->nh; ++k) {
        const int s = k < NG ? k : HB + (k - NG);
        g->h[k] = (H + (1 << s) - 1) >> s; /* ceil(H / 2^s) */
        g->w[k] = (W + (1 << s) - 1) >> s;
        g->off[k + 1] = g->off[k] + (int64_t)g->h[k] * g->w[k];
    }
}

int orc_param_count(int hyper) { return hyper ? N_PARAMS_H : N_PARAMS; }

int64_t orc_latent_count(int H, int W, int hyper) {
    geom_t g;
    geom_init(&g, H, W, hyper);
    return g.off[NGT(&g)];
}

void orc_grid_shape(int H, int W, int k, int* hk, int* wk) {
    geom_t g;
    geom_init(&g, H, W, k >= NG);
    *hk = g.h[k];
    *wk = g.w[k];
}

void orc_context_offsets(int* dy, int* dx) {
    for (int n = 0; n < NCTX; ++n) {
        dy[n] = CTX_DY[n];
        dx[n] = CTX_DX[n];
    }
}

/* ----------------------------------------------------------------------------------------
 * Counter-based uniform noise.  SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)
 * applied to  seed XOR ((t * 2^32 + i) * golden_gamma);  the top 24 bits give u in [-1/2, 1/2).
 * ---------------------------------------------------------------------------------------- */
uint64_t orc_splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t counter_hash(uint64_t seed, int64_t t, int64_t i) {
    uint64_t ctr = ((uint64_t)t << 32) + (uint64_t)i;
    return orc_splitmix64_mix(seed ^ (ctr * 0x9E3779B97F4A7C15ULL));
}

double orc_noise(uint64_t seed, int64_t t, int64_t i) {
    return (double)(counter_hash(seed, t, i) >> 40) * (1.0 / 16777216.0) - 0.5;
}

/* Standard normal n from the same hash by the Box-Muller transform (Box and Muller, 1958):
 * u1 = (bits 40..63 + 1/2) / 2^24 in (0, 1), u2 = bits 16..39 / 2^24 in [0, 1),
 * n = sqrt(-2 ln u1) cos(2 pi u2). */
double orc_gauss(uint64_t seed, int64_t t, int64_t i) {
    uint64_t h = counter_hash(seed, t, i);
    double u1 = ((double)(h >> 40) + 0.5) * (1.0 / 16777216.0);
    double u2 = (double)((h >> 16) & 0xFFFFFFULL) * (1.0 / 16777216.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Soft rounding, Eq. 14 (after Agustsson and Theis):
 *   s_T(x) = floor(x) + 1/2 + tanh(D / T) / (2 tanh(1 / (2T))),  D = x - floor(x) - 1/2,
 * and its derivative (1 - tanh^2(D / T)) / (2 T tanh(1 / (2T))). */
double orc_softround(double x, double T, double* deriv) {
    double fl = floor(x), d = x - fl - 0.5, th = tanh(d / T), den = 2.0 * tanh(0.5 / T);
    if (deriv) *deriv = (1.0 - th * th) / (T * den);
    return fl + 0.5 + th / den;
}

/* ----------------------------------------------------------------------------------------
 * Laplace interval probability, Eq. 3:  P = F(y + 1/2) - F(y - 1/2),  F the Laplace CDF with
 * location mu and scale b.  Evaluated on the side of mu that avoids cancellation.
 * Also returns dP/dy and dP/d(log b).
 * ---------------------------------------------------------------------------------------- */
static double lap_pdf(double z, double b) { return exp(-fabs(z) / b) / (2.0 * b); }

double orc_laplace_prob(double y, double mu, double b, double* dp_dy, double* dp_dlogb) {
    double lo = y - 0.5 - mu, hi = y + 0.5 - mu;
    double p;
    if (lo >= 0.0)
        p = -0.5 * exp(-lo / b) * expm1(-1.0 / b);
    else if (hi <= 0.0)
        p = -0.5 * exp(hi / b) * expm1(-1.0 / b);
    else
        p = 1.0 - 0.5 * exp(lo / b) - 0.5 * exp(-hi / b);
    double fh = lap_pdf(hi, b), fl = lap_pdf(lo, b);
    if (dp_dy) *dp_dy = fh - fl;
    /* dF(z)/db = -(z/b) f(z)  =>  dP/dlogb = b dP/db = -(hi f(hi) - lo f(lo)) */
    if (dp_dlogb) *dp_dlogb = -(hi * fh - lo * fl);
    return p;
}

/* ----------------------------------------------------------------------------------------
 * ARM on one context vector (Eq. 4 with the stabilizer of Eq. 9).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    double c[AIN];
    double a1[AH], h1[AH], a2[AH], h2[AH];
    double mu, s_raw, logb, b;
} arm_act_t;

static void arm_forward(const double* P, arm_act_t* A) {
    for (int o = 0; o < AH; ++o) {
        double acc = P[O_ARM_B1 + o];
        for (int i = 0; i < AIN; ++i) acc += P[O_ARM_W1 + o * AIN + i] * A->c[i];
        A->a1[o] = acc;
        A->h1[o] = acc > 0.0 ? acc : 0.0;
    }
    for (int o = 0; o < AH; ++o) {
        double acc = P[O_ARM_B2 + o];
        for (int i = 0; i < AH; ++i) acc += P[O_ARM_W2 + o * AH + i] * A->h1[i];
        A->a2[o] = acc;
        A->h2[o] = acc > 0.0 ? acc : 0.0;
    }
    double out[2];
    for (int o = 0; o < 2; ++o) {
        double acc = P[O_ARM_B3 + o] + P[O_ARM_BS + o];
        for (int i = 0; i < AH; ++i) acc += P[O_ARM_W3 + o * AH + i] * A->h2[i];
        for (int i = 0; i < AIN; ++i) acc += P[O_ARM_WS + o * AIN + i] * A->c[i];
        out[o] = acc;
    }
    A->mu = out[0];
    A->s_raw = out[1];
    A->logb = fmin(fmax(out[1], LOGB_MIN), LOGB_MAX);
    A->b = exp(A->logb);
}

/* Adjoint of arm_forward: given dL/dmu and dL/dlogb (after the clamp), accumulate parameter
 * gradients into G and return dL/dc. */
static void arm_backward(const double* P, const arm_act_t* A, double dmu, double dlogb, double* G,
                         double* dc) {
    double ds = (A->s_raw >= LOGB_MIN && A->s_raw <= LOGB_MAX) ? dlogb : 0.0;
    double dout[2] = {dmu, ds};
    double dh2[AH], da2[AH], dh1[AH], da1[AH];
    for (int i = 0; i < AIN; ++i) dc[i] = 0.0;
    for (int i = 0; i < AH; ++i) dh2[i] = 0.0;
    for (int o = 0; o < 2; ++o) {
        G[O_ARM_B3 + o] += dout[o];
        G[O_ARM_BS + o] += dout[o];
        for (int i = 0; i < AH; ++i) {
            G[O_ARM_W3 + o * AH + i] += dout[o] * A->h2[i];
            dh2[i] += P[O_ARM_W3 + o * AH + i] * dout[o];
        }
        for (int i = 0; i < AIN; ++i) {
            G[O_ARM_WS + o * AIN + i] += dout[o] * A->c[i];
            dc[i] += P[O_ARM_WS + o * AIN + i] * dout[o];
        }
    }
    for (int o = 0; o < AH; ++o) da2[o] = A->a2[o] > 0.0 ? dh2[o] : 0.0;
    for (int i = 0; i < AH; ++i) dh1[i] = 0.0;
    for (int o = 0; o < AH; ++o) {
        G[O_ARM_B2 + o] += da2[o];
        for (int i = 0; i < AH; ++i) {
            G[O_ARM_W2 + o * AH + i] += da2[o] * A->h1[i];
            dh1[i] += P[O_ARM_W2 + o * AH + i] * da2[o];
        }
    }
    for (int o = 0; o < AH; ++o) da1[o] = A->a1[o] > 0.0 ? dh1[o] : 0.0;
    for (int o = 0; o < AH; ++o) {
        G[O_ARM_B1 + o] += da1[o];
        for (int i = 0; i < AIN; ++i) {
            G[O_ARM_W1 + o * AIN + i] += da1[o] * A->c[i];
            dc[i] += P[O_ARM_W1 + o * AIN + i] * da1[o];
        }
    }
}

/* Number of coarser grids feeding the IFCE of grid k (0 when grid k has no IFCE). */
static int ifce_inputs(int k) { return (k < NIFCE && k < NG - 1) ? NG - k - 1 : 0; }

/* Builds c_i = concat(s_i, f_i) for latent (k, r, c) of the relaxed latents yt.  r_i holds the
 * nearest-neighbour co-located values of the coarser grids k+1..L-1 (Sec. III-A2), then, with
 * hyperlatents, those of the hyperlatent grids (Sec. III-A3); rvec has room for NG + NH values. */
static void build_context(const geom_t* g, const double* P, const double* yt, int k, int r, int c,
                          double* ctx, double* rvec) {
    const double* yk = yt + g->off[k];
    for (int n = 0; n < NCTX; ++n) {
        int rr = r + CTX_DY[n], cc = c + CTX_DX[n];
        ctx[n] = (rr >= 0 && rr < g->h[k] && cc >= 0 && cc < g->w[k]) ? yk[(int64_t)rr * g->w[k] + cc]
                                                                      : 0.0;
    }
    int nin = ifce_inputs(k);
    for (int j = 0; j < nin; ++j) {
        int gj = k + 1 + j, sh = gj - k;
        int rr = r >> sh, cc = c >> sh;
        if (rr > g->h[gj] - 1) rr = g->h[gj] - 1;
        if (cc > g->w[gj] - 1) cc = g->w[gj] - 1;
        rvec[j] = yt[g->off[gj] + (int64_t)rr * g->w[gj] + cc];
    }
    const int nh = nin > 0 ? g->nh : 0;
    for (int q = 0; q < nh; ++q) {
        int gq = NG + q, sh = HB + q - k;
        int rr = r >> sh, cc = c >> sh;
        if (rr > g->h[gq] - 1) rr = g->h[gq] - 1;
        if (cc > g->w[gq] - 1) cc = g->w[gq] - 1;
        rvec[nin + q] = yt[g->off[gq] + (int64_t)rr * g->w[gq] + cc];
    }
    for (int o = 0; o < NF; ++o) {
        double acc = 0.0;
        if (nin > 0) {
            acc = P[IF_B[k] + o];
            for (int j = 0; j < nin; ++j) acc += P[IF_W[k] + o * nin + j] * rvec[j];
            for (int q = 0; q < nh; ++q) acc += P[O_IFH + (k * NF + o) * NH + q] * rvec[nin + q];
        }
        ctx[NCTX + o] = acc;
    }
}

/* ----------------------------------------------------------------------------------------
 * Upsampling stage (Sec. III-B, Eq. 7): x2 separable symmetric 8-tap filter [a b c d d c b a]
 * as a transposed convolution with replicate padding; output cropped to (th, tw).
 * Polyphase form per axis, X indices clamped to [0, n-1]:
 *   out[2p]   = a X[p-2] + c X[p-1] + d X[p]   + b X[p+1]
 *   out[2p+1] = b X[p-1] + d X[p]   + c X[p+1] + a X[p+2]
 * Rows (the W axis) first, then columns.
 * ---------------------------------------------------------------------------------------- */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* tap index (0=a,1=b,2=c,3=d) and input offset of the 4 taps of output position o */
static void poly_taps(int o, int* tap, int* src) {
    int p = o >> 1;
    if ((o & 1) == 0) {
        tap[0] = 0; src[0] = p - 2;
        tap[1] = 2; src[1] = p - 1;
        tap[2] = 3; src[2] = p;
        tap[3] = 1; src[3] = p + 1;
    } else {
        tap[0] = 1; src[0] = p - 1;
        tap[1] = 3; src[1] = p;
        tap[2] = 2; src[2] = p + 1;
        tap[3] = 0; src[3] = p + 2;
    }
}

void orc_upsample(int sh, int sw, int th, int tw, const double* taps, const double* x, double* out) {
    double* tmp = (double*)malloc(sizeof(double) * (size_t)sh * tw);
    for (int r = 0; r < sh; ++r)
        for (int o = 0; o < tw; ++o) {
            int tap[4], src[4];
            poly_taps(o, tap, src);
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) acc += taps[tap[q]] * x[(int64_t)r * sw + clampi(src[q], 0, sw - 1)];
            tmp[(int64_t)r * tw + o] = acc;
        }
    for (int o = 0; o < th; ++o)
        for (int c = 0; c < tw; ++c) {
            int tap[4], src[4];
            poly_taps(o, tap, src);
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) acc += taps[tap[q]] * tmp[(int64_t)clampi(src[q], 0, sh - 1) * tw + c];
            out[(int64_t)o * tw + c] = acc;
        }
    free(tmp);
}

/* Adjoint of orc_upsample: scatter dout back to dx and accumulate the 4 tap gradients. */
static void upsample_adjoint(int sh, int sw, int th, int tw, const double* taps, const double* x,
                             const double* dout, double* dx, double* dtaps) {
    double* tmp = (double*)malloc(sizeof(double) * (size_t)sh * tw);
    double* dtmp = (double*)calloc((size_t)sh * tw, sizeof(double));
    for (int r = 0; r < sh; ++r)
        for (int o = 0; o < tw; ++o) {
            int tap[4], src[4];
            poly_taps(o, tap, src);
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) acc += taps[tap[q]] * x[(int64_t)r * sw + clampi(src[q], 0, sw - 1)];
            tmp[(int64_t)r * tw + o] = acc;
        }
    for (int o = 0; o < th; ++o)
        for (int c = 0; c < tw; ++c) {
            int tap[4], src[4];
            poly_taps(o, tap, src);
            double g = dout[(int64_t)o * tw + c];
            for (int q = 0; q < 4; ++q) {
                int64_t si = (int64_t)clampi(src[q], 0, sh - 1) * tw + c;
                dtaps[tap[q]] += g * tmp[si];
                dtmp[si] += g * taps[tap[q]];
            }
        }
    for (int r = 0; r < sh; ++r)
        for (int o = 0; o < tw; ++o) {
            int tap[4], src[4];
            poly_taps(o, tap, src);
            double g = dtmp[(int64_t)r * tw + o];
            for (int q = 0; q < 4; ++q) {
                int64_t si = (int64_t)r * sw + clampi(src[q], 0, sw - 1);
                dtaps[tap[q]] += g * x[si];
                dx[si] += g * taps[tap[q]];
            }
        }
    free(tmp);
    free(dtmp);
}

/* ----------------------------------------------------------------------------------------
 * 3x3 residual convolution, 3 -> 3 channels, replicate padding (cross-correlation):
 *   out[o][y][x] = in[o][y][x] + b[o] + sum_{i,ky,kx} W[o][i][ky][kx] in[i][y+ky-1][x+kx-1]
 * ---------------------------------------------------------------------------------------- */
void orc_conv3x3_res(int H, int W, const double* Wt, const double* b, const double* in, double* out) {
    int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int o = 0; o < NCH; ++o) {
                double acc = in[o * HW + (int64_t)y * W + x] + b[o];
                for (int i = 0; i < NCH; ++i)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            int yy = clampi(y + ky - 1, 0, H - 1), xx = clampi(x + kx - 1, 0, W - 1);
                            acc += Wt[((o * NCH + i) * 3 + ky) * 3 + kx] * in[i * HW + (int64_t)yy * W + xx];
                        }
                out[o * HW + (int64_t)y * W + x] = acc;
            }
}

/* Adjoint of orc_conv3x3_res: din += dout + conv^T(dout); dW, db accumulated. */
static void conv3x3_res_adjoint(int H, int W, const double* Wt, const double* in, const double* dout,
                                double* din, double* dW, double* db) {
    int64_t HW = (int64_t)H * W;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int o = 0; o < NCH; ++o) {
                double g = dout[o * HW + (int64_t)y * W + x];
                din[o * HW + (int64_t)y * W + x] += g;
                db[o] += g;
                for (int i = 0; i < NCH; ++i)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            int yy = clampi(y + ky - 1, 0, H - 1), xx = clampi(x + kx - 1, 0, W - 1);
                            int widx = ((o * NCH + i) * 3 + ky) * 3 + kx;
                            int64_t si = i * HW + (int64_t)yy * W + xx;
                            dW[widx] += g * in[si];
                            din[si] += g * Wt[widx];
                        }
            }
}

/* ----------------------------------------------------------------------------------------
 * Synthesis 1x1 MLP with stabilizer (Eq. 8, Eq. 9): t = W2 gelu(W1 z + b1) + b2 + Ws z + bs.
 * GELU in its exact erf form.
 * ---------------------------------------------------------------------------------------- */
static double gelu(double a) { return 0.5 * a * (1.0 + erf(a / sqrt(2.0))); }
static double gelu_grad(double a) {
    return 0.5 * (1.0 + erf(a / sqrt(2.0))) + a * exp(-0.5 * a * a) / sqrt(2.0 * M_PI);
}

static void synth_pixel(const double* P, const double* z, double* a, double* t) {
    for (int o = 0; o < SH; ++o) {
        double acc = P[O_SYN_B1 + o];
        for (int i = 0; i < NG; ++i) acc += P[O_SYN_W1 + o * NG + i] * z[i];
        a[o] = acc;
    }
    for (int o = 0; o < NCH; ++o) {
        double acc = P[O_SYN_B2 + o] + P[O_SYN_BS + o];
        for (int i = 0; i < SH; ++i) acc += P[O_SYN_W2 + o * SH + i] * gelu(a[i]);
        for (int i = 0; i < NG; ++i) acc += P[O_SYN_WS + o * NG + i] * z[i];
        t[o] = acc;
    }
}

/* ----------------------------------------------------------------------------------------
 * Whole forward and adjoint.
 * ---------------------------------------------------------------------------------------- */
enum { MODE_NOISE = 0, MODE_HARD = 1, MODE_IDENTITY = 2, MODE_SOFTROUND = 3 };

/* How the latents are relaxed: MODE_SOFTROUND uses sigma and temp (Eq. 13). */
typedef struct {
    int mode;
    uint64_t seed;
    int64_t t;
    double sigma, temp;
} relax_t;

typedef struct {
    geom_t g;
    double* yt;         /* relaxed latents, all grids                                 */
    double* up[NG];     /* up[m]: channels for grids m+1..L-1 upsampled to grid m      */
    double* z;          /* dense representation [L][H][W]                              */
    double* t;          /* synthesis output before the residual convs [3][H][W]       */
    double* x1;         /* after conv 1                                                */
    double* xh;         /* reconstruction                                              */
    double* mu;
    double* logb;
    double* bits;
} fwd_t;

static void fwd_free(fwd_t* F) {
    free(F->yt);
    for (int m = 0; m < NG; ++m) free(F->up[m]);
    free(F->z);
    free(F->t);
    free(F->x1);
    free(F->xh);
    free(F->mu);
    free(F->logb);
    free(F->bits);
}

/* channels of S_m = [y~^(m), up[m]] are grids m..L-1; return pointer to channel j (grid m+j). */
static const double* stage_channel(const fwd_t* F, int m, int j) {
    if (j == 0) return F->yt + F->g.off[m];
    return F->up[m] + (int64_t)(j - 1) * F->g.h[m] * F->g.w[m];
}

/* y~ of latent i and, when jac is non-null, dy~/dy */
static double relax_one(const relax_t* R, double y, int64_t i, double* jac) {
    double j = 1.0, v;
    if (R->mode == MODE_NOISE) {
        v = y + orc_noise(R->seed, R->t, i);
    } else if (R->mode == MODE_HARD) {
        v = rint(y);
        j = 0.0;
    } else if (R->mode == MODE_SOFTROUND) {
        double d1, d2;
        double s1 = orc_softround(y, R->temp, &d1);
        v = orc_softround(s1 + R->sigma * orc_gauss(R->seed, R->t, i), R->temp, &d2);
        j = d2 * d1;
    } else {
        v = y;
    }
    if (jac) *jac = j;
    return v;
}

static double run_forward(int H, int W, int hyper, const double* img, const double* y, const double* P,
                          const relax_t* R, double lambda, fwd_t* F, double* rate_out, double* mse_out) {
    geom_init(&F->g, H, W, hyper);
    const geom_t* g = &F->g;
    int64_t N = g->off[NGT(g)], HW = (int64_t)H * W;
    F->yt = (double*)malloc(sizeof(double) * N);
    F->mu = (double*)malloc(sizeof(double) * N);
    F->logb = (double*)malloc(sizeof(double) * N);
    F->bits = (double*)malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) F->yt[i] = relax_one(R, y[i], i, NULL);
    /* entropy model: Eqs. 2-5, 9, 11 (every grid, hyperlatent grids included) */
    for (int k = 0; k < NGT(g); ++k) {
#pragma omp parallel for schedule(static)
        for (int r = 0; r < g->h[k]; ++r)
            for (int c = 0; c < g->w[k]; ++c) {
                int64_t i = g->off[k] + (int64_t)r * g->w[k] + c;
                arm_act_t A;
                double rv[NG + NH];
                build_context(g, P, F->yt, k, r, c, A.c, rv);
                arm_forward(P, &A);
                double p = orc_laplace_prob(F->yt[i], A.mu, A.b, NULL, NULL);
                F->mu[i] = A.mu;
                F->logb[i] = A.logb;
                F->bits[i] = -log2(fmax(p, P_MIN));
            }
    }
    double rate = 0.0;
    for (int64_t i = 0; i < N; ++i) rate += F->bits[i];
    /* upsampling cascade: S_{L-1} = y~^(L-1); S_{m} = [y~^(m), U_{m+1}(S_{m+1})] */
    for (int m = 0; m < NG; ++m) F->up[m] = NULL;
    for (int m = NG - 2; m >= 0; --m) {
        int nch = NG - m - 1; /* channels of up[m] = channels of S_{m+1} */
        int64_t sz = (int64_t)g->h[m] * g->w[m];
        F->up[m] = (double*)malloc(sizeof(double) * nch * sz);
        const double* taps = P + O_UP + 4 * m; /* stage s = m + 1 */
        for (int j = 0; j < nch; ++j)
            orc_upsample(g->h[m + 1], g->w[m + 1], g->h[m], g->w[m], taps, stage_channel(F, m + 1, j),
                         F->up[m] + j * sz);
    }
    F->z = (double*)malloc(sizeof(double) * NG * HW);
    for (int j = 0; j < NG; ++j) memcpy(F->z + j * HW, stage_channel(F, 0, j), sizeof(double) * HW);
    /* synthesis */
    F->t = (double*)malloc(sizeof(double) * NCH * HW);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < HW; ++p) {
        double z[NG], a[SH], tt[NCH];
        for (int j = 0; j < NG; ++j) z[j] = F->z[j * HW + p];
        synth_pixel(P, z, a, tt);
        for (int o = 0; o < NCH; ++o) F->t[o * HW + p] = tt[o];
    }
    F->x1 = (double*)malloc(sizeof(double) * NCH * HW);
    F->xh = (double*)malloc(sizeof(double) * NCH * HW);
    orc_conv3x3_res(H, W, P + O_CV1_W, P + O_CV1_B, F->t, F->x1);
    orc_conv3x3_res(H, W, P + O_CV2_W, P + O_CV2_B, F->x1, F->xh);
    double se = 0.0;
    for (int64_t q = 0; q < NCH * HW; ++q) {
        double d = F->xh[q] - img[q];
        se += d * d;
    }
    double mse = se / (double)(NCH * HW);
    *rate_out = rate;
    *mse_out = mse;
    return mse + lambda * rate / (double)HW;
}

double orc_forward(int H, int W, int hyper, const double* img, const double* y, const double* P, int mode,
                   uint64_t seed, int64_t t, double sigma, double temp, double lambda, double* rate_out,
                   double* mse_out, double* mu_out, double* logb_out, double* bits_out, double* xhat_out) {
    fwd_t F;
    memset(&F, 0, sizeof(F));
    relax_t R = {mode, seed, t, sigma, temp};
    double loss = run_forward(H, W, hyper, img, y, P, &R, lambda, &F, rate_out, mse_out);
    int64_t N = F.g.off[NGT(&F.g)], HW = (int64_t)H * W;
    if (mu_out) memcpy(mu_out, F.mu, sizeof(double) * N);
    if (logb_out) memcpy(logb_out, F.logb, sizeof(double) * N);
    if (bits_out) memcpy(bits_out, F.bits, sizeof(double) * N);
    if (xhat_out) memcpy(xhat_out, F.xh, sizeof(double) * NCH * HW);
    fwd_free(&F);
    return loss;
}

/* Loss and its gradient with respect to the continuous latents y and the parameters:
 * dL/dy = dL/dy~ * dy~/dy (1 for the additive proxy, 0 under hard rounding, the product of the
 * two soft-rounding derivatives for Eq. 13). */
double orc_loss_grad(int H, int W, int hyper, const double* img, const double* y, const double* P, int mode,
                     uint64_t seed, int64_t t, double sigma, double temp, double lambda, double* rate_out,
                     double* mse_out, double* gy, double* gP) {
    fwd_t F;
    memset(&F, 0, sizeof(F));
    relax_t R = {mode, seed, t, sigma, temp};
    double loss = run_forward(H, W, hyper, img, y, P, &R, lambda, &F, rate_out, mse_out);
    const geom_t* g = &F.g;
    int64_t N = g->off[NGT(g)], HW = (int64_t)H * W;
    double* gyt = (double*)calloc(N, sizeof(double));
    for (int q = 0; q < orc_param_count(hyper); ++q) gP[q] = 0.0;

    /* distortion: D = mean (xh - x)^2 */
    double* dxh = (double*)malloc(sizeof(double) * NCH * HW);
    for (int64_t q = 0; q < NCH * HW; ++q) dxh[q] = 2.0 * (F.xh[q] - img[q]) / (double)(NCH * HW);
    double* dx1 = (double*)calloc(NCH * HW, sizeof(double));
    double* dt = (double*)calloc(NCH * HW, sizeof(double));
    conv3x3_res_adjoint(H, W, P + O_CV2_W, F.x1, dxh, dx1, gP + O_CV2_W, gP + O_CV2_B);
    conv3x3_res_adjoint(H, W, P + O_CV1_W, F.t, dx1, dt, gP + O_CV1_W, gP + O_CV1_B);

    /* synthesis adjoint; per-row partial parameter gradients summed serially afterwards */
    double* dz = (double*)calloc(NG * HW, sizeof(double));
    double* rowg = (double*)calloc((size_t)H * N_PARAMS, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int yy = 0; yy < H; ++yy) {
        double* Gr = rowg + (size_t)yy * N_PARAMS; /* this row's partial gradient */
        for (int xx = 0; xx < W; ++xx) {
            int64_t p = (int64_t)yy * W + xx;
            double z[NG], a[SH], tt[NCH], dtt[NCH], ga[SH];
            for (int j = 0; j < NG; ++j) z[j] = F.z[j * HW + p];
            synth_pixel(P, z, a, tt);
            for (int o = 0; o < NCH; ++o) dtt[o] = dt[o * HW + p];
            double dzp[NG] = {0};
            for (int i = 0; i < SH; ++i) ga[i] = 0.0;
            for (int o = 0; o < NCH; ++o) {
                Gr[O_SYN_B2 + o] += dtt[o];
                Gr[O_SYN_BS + o] += dtt[o];
                for (int i = 0; i < SH; ++i) {
                    Gr[O_SYN_W2 + o * SH + i] += dtt[o] * gelu(a[i]);
                    ga[i] += P[O_SYN_W2 + o * SH + i] * dtt[o];
                }
                for (int i = 0; i < NG; ++i) {
                    Gr[O_SYN_WS + o * NG + i] += dtt[o] * z[i];
                    dzp[i] += P[O_SYN_WS + o * NG + i] * dtt[o];
                }
            }
            for (int o = 0; o < SH; ++o) {
                double da = ga[o] * gelu_grad(a[o]);
                Gr[O_SYN_B1 + o] += da;
                for (int i = 0; i < NG; ++i) {
                    Gr[O_SYN_W1 + o * NG + i] += da * z[i];
                    dzp[i] += P[O_SYN_W1 + o * NG + i] * da;
                }
            }
            for (int j = 0; j < NG; ++j) dz[j * HW + p] = dzp[j];
        }
    }
    for (int yy = 0; yy < H; ++yy)
        for (int q = O_SYN_W1; q < O_CV1_W; ++q) gP[q] += rowg[(size_t)yy * N_PARAMS + q];
    free(rowg);

    /* upsampling adjoint: dS_0 = dz; for m = 1..L-1: dS_m = U_m^T(dup[m-1]) */
    double* dS = dz; /* channels of S_0 */
    for (int m = 0; m < NG; ++m) {
        int64_t sz = (int64_t)g->h[m] * g->w[m];
        int nch = NG - m; /* channels of S_m */
        for (int64_t q = 0; q < sz; ++q) gyt[g->off[m] + q] += dS[q];
        if (m == NG - 1) break;
        int64_t szn = (int64_t)g->h[m + 1] * g->w[m + 1];
        double* dSn = (double*)calloc((size_t)(nch - 1) * szn, sizeof(double));
        for (int j = 0; j < nch - 1; ++j)
            upsample_adjoint(g->h[m + 1], g->w[m + 1], g->h[m], g->w[m], P + O_UP + 4 * m,
                             stage_channel(&F, m + 1, j), dS + (int64_t)(j + 1) * sz, dSn + j * szn,
                             gP + O_UP + 4 * m);
        if (dS != dz) free(dS);
        dS = dSn;
    }
    if (dS != dz) free(dS);
    free(dz);

    /* entropy-model adjoint: per-latent contributions computed in parallel, scattered serially */
    double dbits = lambda / (double)HW;
    const int NARM = O_UP; /* ARM + IFCE parameter block */
    const int RV = NG + NH; /* room for the IFCE inputs of one latent */
    for (int k = 0; k < NGT(g); ++k) {
        int h = g->h[k], w = g->w[k];
        double* dcs = (double*)malloc(sizeof(double) * (size_t)h * w * AIN);
        double* rvs = (double*)malloc(sizeof(double) * (size_t)h * w * RV);
        double* ddir = (double*)malloc(sizeof(double) * (size_t)h * w);
        double* rowa = (double*)calloc((size_t)h * NARM, sizeof(double));
#pragma omp parallel for schedule(static)
        for (int r = 0; r < h; ++r) {
            double* Gr = rowa + (size_t)r * NARM;
            for (int c = 0; c < w; ++c) {
                int64_t li = (int64_t)r * w + c, i = g->off[k] + li;
                arm_act_t A;
                double* rv = rvs + li * RV;
                build_context(g, P, F.yt, k, r, c, A.c, rv);
                arm_forward(P, &A);
                double dpdy, dpdlb;
                double p = orc_laplace_prob(F.yt[i], A.mu, A.b, &dpdy, &dpdlb);
                double dp = (p >= P_MIN) ? -dbits / (p * log(2.0)) : 0.0;
                ddir[li] = dp * dpdy;
                arm_backward(P, &A, -dp * dpdy, dp * dpdlb, Gr, dcs + li * AIN);
            }
        }
        for (int r = 0; r < h; ++r)
            for (int q = 0; q < NARM; ++q) gP[q] += rowa[(size_t)r * NARM + q];
        int nin = ifce_inputs(k);
        for (int r = 0; r < h; ++r)
            for (int c = 0; c < w; ++c) {
                int64_t li = (int64_t)r * w + c;
                const double* dc = dcs + li * AIN;
                gyt[g->off[k] + li] += ddir[li];
                for (int n = 0; n < NCTX; ++n) {
                    int rr = r + CTX_DY[n], cc = c + CTX_DX[n];
                    if (rr >= 0 && rr < h && cc >= 0 && cc < w) gyt[g->off[k] + (int64_t)rr * w + cc] += dc[n];
                }
                if (nin > 0) {
                    const double* df = dc + NCTX;
                    for (int o = 0; o < NF; ++o) {
                        gP[IF_B[k] + o] += df[o];
                        for (int j = 0; j < nin; ++j) gP[IF_W[k] + o * nin + j] += df[o] * rvs[li * RV + j];
                        for (int q = 0; q < g->nh; ++q)
                            gP[O_IFH + (k * NF + o) * NH + q] += df[o] * rvs[li * RV + nin + q];
                    }
                    for (int q = 0; q < g->nh; ++q) {
                        int gq = NG + q, sh = HB + q - k;
                        int rr = r >> sh, cc = c >> sh;
                        if (rr > g->h[gq] - 1) rr = g->h[gq] - 1;
                        if (cc > g->w[gq] - 1) cc = g->w[gq] - 1;
                        double acc = 0.0;
                        for (int o = 0; o < NF; ++o) acc += P[O_IFH + (k * NF + o) * NH + q] * df[o];
                        gyt[g->off[gq] + (int64_t)rr * g->w[gq] + cc] += acc;
                    }
                    for (int j = 0; j < nin; ++j) {
                        int gj = k + 1 + j, sh = gj - k;
                        int rr = r >> sh, cc = c >> sh;
                        if (rr > g->h[gj] - 1) rr = g->h[gj] - 1;
                        if (cc > g->w[gj] - 1) cc = g->w[gj] - 1;
                        double acc = 0.0;
                        for (int o = 0; o < NF; ++o) acc += P[IF_W[k] + o * nin + j] * df[o];
                        gyt[g->off[gj] + (int64_t)rr * g->w[gj] + cc] += acc;
                    }
                }
            }
        free(dcs);
        free(rvs);
        free(ddir);
        free(rowa);
    }
    /* chain rule through the relaxation */
    for (int64_t i = 0; i < N; ++i) {
        double jac;
        relax_one(&R, y[i], i, &jac);
        gy[i] = gyt[i] * jac;
    }
    free(gyt);
    free(dxh);
    free(dx1);
    free(dt);
    fwd_free(&F);
    return loss;
}

/* ----------------------------------------------------------------------------------------
 * Adam (Kingma & Ba), bias-corrected, no weight decay.  t_new is the 1-based step count.
 * ---------------------------------------------------------------------------------------- */
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v, int64_t t_new, double lr,
              double b1, double b2, double eps) {
    double bc1 = 1.0 - pow(b1, (double)t_new), bc2 = 1.0 - pow(b2, (double)t_new);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* n_iters encoder iterations: loss+gradient at step t (noise keyed by t), then Adam on latents
 * and parameters.  Per-iteration loss, rate and mse (before the update) are reported. */
void orc_encode(int H, int W, int hyper, const double* img, double* y, double* P, double* m_y, double* v_y,
                double* m_p, double* v_p, int64_t* step, int n_iters, uint64_t seed, double lambda,
                double lr, double b1, double b2, double eps, double* loss_out, double* rate_out,
                double* mse_out) {
    int64_t N = orc_latent_count(H, W, hyper);
    const int NP = orc_param_count(hyper);
    double* gy = (double*)malloc(sizeof(double) * N);
    double gP[N_PARAMS_H];
    for (int it = 0; it < n_iters; ++it) {
        double rate, mse;
        double loss = orc_loss_grad(H, W, hyper, img, y, P, MODE_NOISE, seed, *step, 0.0, 1.0, lambda, &rate, &mse,
                                    gy, gP);
        if (loss_out) loss_out[it] = loss;
        if (rate_out) rate_out[it] = rate;
        if (mse_out) mse_out[it] = mse;
        *step += 1;
        orc_adam(N, y, gy, m_y, v_y, *step, lr, b1, b2, eps);
        orc_adam(NP, P, gP, m_p, v_p, *step, lr, b1, b2, eps);
    }
    free(gy);
}

/* The paper's encoder schedule (Sec. IV-C/D, Table I), n_iters iterations from *step:
 *   main stage, steps t < n_main, with f = t / n_main:  y~ = s_T(s_T(y) + sigma n),
 *     sigma = sigma0 + (sigma1 - sigma0) f,  T = temp0 + (temp1 - temp0) f,
 *     lr = lr_min + (lr_max - lr_min) (1 + cos(pi f)) / 2,  Adam on latents and parameters;
 *   hard-round stage, t >= n_main:  y~ = rint(y), latents frozen (no update, moments kept),
 *     Adam on the parameters at lr_min.
 * The Adam step count is t + 1 in both stages. */
void orc_encode_schedule(int H, int W, int hyper, const double* img, double* y, double* P, double* m_y, double* v_y,
                         double* m_p, double* v_p, int64_t* step, int n_iters, uint64_t seed, double lambda,
                         double lr_max, double lr_min, double sigma0, double sigma1, double temp0, double temp1,
                         int64_t n_main, double b1, double b2, double eps, double* loss_out, double* rate_out,
                         double* mse_out) {
    int64_t N = orc_latent_count(H, W, hyper);
    const int NP = orc_param_count(hyper);
    double* gy = (double*)malloc(sizeof(double) * N);
    double gP[N_PARAMS_H];
    for (int it = 0; it < n_iters; ++it) {
        const int64_t t = *step;
        const int main_stage = t < n_main;
        const double f = main_stage ? (double)t / (double)n_main : 1.0;
        const double sigma = sigma0 + (sigma1 - sigma0) * f, temp = temp0 + (temp1 - temp0) * f;
        const double lr = main_stage ? lr_min + 0.5 * (lr_max - lr_min) * (1.0 + cos(M_PI * f)) : lr_min;
        double rate, mse;
        double loss = orc_loss_grad(H, W, hyper, img, y, P, main_stage ? MODE_SOFTROUND : MODE_HARD, seed, t,
                                    sigma, temp, lambda, &rate, &mse, gy, gP);
        if (loss_out) loss_out[it] = loss;
        if (rate_out) rate_out[it] = rate;
        if (mse_out) mse_out[it] = mse;
        *step += 1;
        if (main_stage) orc_adam(N, y, gy, m_y, v_y, *step, lr, b1, b2, eps);
        orc_adam(NP, P, gP, m_p, v_p, *step, lr, b1, b2, eps);
    }
    free(gy);
}

/* ----------------------------------------------------------------------------------------
 * Integer decode-side entropy model (Sec. III-A2: integer, cross-platform decoding).
 * Fixed point with 8 fractional bits: weights and biases w_q = rint(256 w); the spatial context
 * enters as 256 * y^; each layer accumulates in 64-bit integers, adds the bias shifted to the
 * product scale, shifts right by 8 (floor) and applies ReLU.  The outputs mu_q, logb_q are on a
 * 1/256 grid; logb_q is clamped to [-1280, 1280].
 * Integer CDF with 16-bit total mass:  C(t) = 65536 - E(s, t) for t >= 0, E(s, -t) otherwise, where
 * E(s, u) ~ 2^15 exp(-u / (256 b_s)) = 2^15 2^(-v / 2^28) with v = u * K[s] and
 * K[s] = rint(2^20 log2(e) exp(-s/256)).  With n = v >> 28, hi = bits 18..27 of v, lo = bits 8..17:
 *   E = ((T_HI[hi] * T_LO[lo]) >> 15) >> n     (E = 0 once n >= 16),
 * T_HI[j] = rint(2^15 2^(-j/2^10)), T_LO[j] = rint(2^15 2^(-j/2^20)): a coarse x fine split of the
 * fractional exponent.  All tables are built here in FP64, independently of any other implementation.
 * P_q16 = max(1, C(256 y^ + 128 - mu_q) - C(256 y^ - 128 - mu_q)).
 * ---------------------------------------------------------------------------------------- */
#define LOGBQ_MIN (-1280)
#define LOGBQ_MAX (1280)
static int64_t K_TAB[LOGBQ_MAX - LOGBQ_MIN + 1];
static int64_t T_HI[1024], T_LO[1024];
static int tabs_ready = 0;

static void build_tables(void) {
    if (tabs_ready) return;
    for (int s = LOGBQ_MIN; s <= LOGBQ_MAX; ++s)
        K_TAB[s - LOGBQ_MIN] = (int64_t)rint(1048576.0 * (1.0 / log(2.0)) * exp(-(double)s / 256.0));
    for (int j = 0; j < 1024; ++j) {
        T_HI[j] = (int64_t)rint(32768.0 * exp2(-(double)j / 1024.0));
        T_LO[j] = (int64_t)rint(32768.0 * exp2(-(double)j / 1048576.0));
    }
    tabs_ready = 1;
}

int64_t orc_cdf_q16(int32_t s, int64_t t) {
    build_tables();
    int64_t u = t >= 0 ? t : -t;
    int64_t v = u * K_TAB[s - LOGBQ_MIN];
    int64_t n = v >> 28;
    int64_t e = 0;
    if (n < 16) e = ((T_HI[(v >> 18) & 1023] * T_LO[(v >> 8) & 1023]) >> 15) >> n;
    return t >= 0 ? 65536 - e : e;
}

/* which = 0: K[idx] (idx = s + 1280), 1: T_HI[idx], 2: T_LO[idx] */
int64_t orc_table_entry(int which, int idx) {
    build_tables();
    return which == 0 ? K_TAB[idx] : (which == 1 ? T_HI[idx] : T_LO[idx]);
}

static int64_t floor_shift8(int64_t v) { return v >> 8; } /* arithmetic shift = floor(v / 256) */
static int64_t q8(float w) { return (int64_t)rint((double)w * 256.0); }

/* Integer ARM for every latent of the hard-quantised grids q; writes mu_q, logb_q, P_q16. */
void orc_decode_probs(int H, int W, int hyper, const int32_t* q, const float* Pf, int32_t* mu_out,
                      int32_t* logb_out, uint32_t* prob_out) {
    build_tables();
    geom_t g;
    geom_init(&g, H, W, hyper);
    for (int k = 0; k < NGT(&g); ++k) {
        int nin = ifce_inputs(k);
        for (int r = 0; r < g.h[k]; ++r)
            for (int c = 0; c < g.w[k]; ++c) {
                int64_t i = g.off[k] + (int64_t)r * g.w[k] + c;
                int64_t ctx[AIN], h1[AH], h2[AH];
                for (int n = 0; n < NCTX; ++n) {
                    int rr = r + CTX_DY[n], cc = c + CTX_DX[n];
                    int64_t v = (rr >= 0 && rr < g.h[k] && cc >= 0 && cc < g.w[k])
                                    ? q[g.off[k] + (int64_t)rr * g.w[k] + cc]
                                    : 0;
                    ctx[n] = v * 256;
                }
                for (int o = 0; o < NF; ++o) {
                    int64_t acc = 0;
                    if (nin > 0) {
                        acc = q8(Pf[IF_B[k] + o]);
                        for (int j = 0; j < nin; ++j) {
                            int gj = k + 1 + j, sh = gj - k;
                            int rr = r >> sh, cc = c >> sh;
                            if (rr > g.h[gj] - 1) rr = g.h[gj] - 1;
                            if (cc > g.w[gj] - 1) cc = g.w[gj] - 1;
                            acc += q8(Pf[IF_W[k] + o * nin + j]) *
                                   (int64_t)q[g.off[gj] + (int64_t)rr * g.w[gj] + cc];
                        }
                        for (int hq = 0; hq < g.nh; ++hq) {
                            int gq = NG + hq, sh = HB + hq - k;
                            int rr = r >> sh, cc = c >> sh;
                            if (rr > g.h[gq] - 1) rr = g.h[gq] - 1;
                            if (cc > g.w[gq] - 1) cc = g.w[gq] - 1;
                            acc += q8(Pf[O_IFH + (k * NF + o) * NH + hq]) *
                                   (int64_t)q[g.off[gq] + (int64_t)rr * g.w[gq] + cc];
                        }
                    }
                    ctx[NCTX + o] = acc;
                }
                for (int o = 0; o < AH; ++o) {
                    int64_t acc = q8(Pf[O_ARM_B1 + o]) * 256;
                    for (int n = 0; n < AIN; ++n) acc += q8(Pf[O_ARM_W1 + o * AIN + n]) * ctx[n];
                    acc = floor_shift8(acc);
                    h1[o] = acc > 0 ? acc : 0;
                }
                for (int o = 0; o < AH; ++o) {
                    int64_t acc = q8(Pf[O_ARM_B2 + o]) * 256;
                    for (int n = 0; n < AH; ++n) acc += q8(Pf[O_ARM_W2 + o * AH + n]) * h1[n];
                    acc = floor_shift8(acc);
                    h2[o] = acc > 0 ? acc : 0;
                }
                int64_t out[2];
                for (int o = 0; o < 2; ++o) {
                    int64_t acc = (q8(Pf[O_ARM_B3 + o]) + q8(Pf[O_ARM_BS + o])) * 256;
                    for (int n = 0; n < AH; ++n) acc += q8(Pf[O_ARM_W3 + o * AH + n]) * h2[n];
                    for (int n = 0; n < AIN; ++n) acc += q8(Pf[O_ARM_WS + o * AIN + n]) * ctx[n];
                    out[o] = floor_shift8(acc);
                }
                int64_t mu = out[0];
                int64_t s = out[1] < LOGBQ_MIN ? LOGBQ_MIN : (out[1] > LOGBQ_MAX ? LOGBQ_MAX : out[1]);
                int64_t yq = (int64_t)q[i] * 256;
                int64_t cp = orc_cdf_q16((int32_t)s, yq + 128 - mu);
                int64_t cm = orc_cdf_q16((int32_t)s, yq - 128 - mu);
                int64_t pq = cp - cm;
                if (mu_out) mu_out[i] = (int32_t)mu;
                if (logb_out) logb_out[i] = (int32_t)s;
                if (prob_out) prob_out[i] = (uint32_t)(pq < 1 ? 1 : pq);
            }
    }
}

/* Decoder reconstruction from hard-quantised latents: upsampling + synthesis in FP64, x^ clamped
 * to [0, 1] (Sec. III-B). */
void orc_decode_image(int H, int W, int hyper, const int32_t* q, const float* Pf, double* img_out) {
    int64_t N = orc_latent_count(H, W, hyper);
    double* y = (double*)malloc(sizeof(double) * N);
    double P[N_PARAMS_H];
    for (int64_t i = 0; i < N; ++i) y[i] = (double)q[i];
    for (int j = 0; j < orc_param_count(hyper); ++j) P[j] = (double)Pf[j];
    double rate, mse;
    int64_t HW = (int64_t)H * W;
    double* zero = (double*)calloc(NCH * HW, sizeof(double));
    fwd_t F;
    memset(&F, 0, sizeof(F));
    relax_t R = {MODE_IDENTITY, 0, 0, 0.0, 1.0};
    run_forward(H, W, hyper, zero, y, P, &R, 0.0, &F, &rate, &mse);
    for (int64_t q2 = 0; q2 < NCH * HW; ++q2) img_out[q2] = fmin(fmax(F.xh[q2], 0.0), 1.0);
    fwd_free(&F);
    free(zero);
    free(y);
}

/* ----------------------------------------------------------------------------------------
 * SOAP for the neural-network parameters (Sec. IV-B: SOAP for the networks, Adam for the latents).
 * The paper names the optimizer (Vyas et al., "SOAP: Improving and Stabilizing Shampoo using Adam")
 * and fixes none of its settings; this restatement follows the SOAP paper's single-layer step.
 * For every two-dimensional weight block W (m x n; a residual convolution's kernel taken as
 * [out][in * 9]) with gradient G:
 *   step s = 0 (the first call): L = (1 - bs) G G^T, R = (1 - bs) G^T G, Q_L, Q_R = their
 *     eigenvectors; no parameter update;
 *   step s >= 1:  G' = Q_L^T G Q_R,  M = b1 M + (1 - b1) G,  M' = Q_L^T M Q_R,
 *     V = b2 V + (1 - b2) G' * G'  (element-wise, kept in the rotated coordinates),
 *     N' = (M' / (1 - b1^s)) / (sqrt(V / (1 - b2^s)) + eps),  W -= lr Q_L N' Q_R^T,
 *     then L = bs L + (1 - bs) G G^T, R = bs R + (1 - bs) G^T G, and every `freq` steps
 *     Q_L, Q_R = the eigenvectors of the new L, R.
 * Eigenvectors are the columns of Q, ordered by decreasing eigenvalue, each with its entry of
 * largest magnitude positive (unique when the eigenvalues are distinct).  They are computed by
 * the cyclic Jacobi method (Golub and Van Loan, Matrix Computations, the symmetric Schur 2 x 2
 * rotation applied pair by pair until the off-diagonal mass vanishes).  The SOAP paper refreshes
 * the eigenbasis with one power-iteration step and a QR decomposition; a full decomposition gives
 * the eigenbasis that iteration tracks.  One-dimensional blocks (biases, upsampling taps) and the
 * latents use Adam.  M and V of a block live in the parameter moment arrays at the block's offsets;
 * L, R, Q_L, Q_R in a separate state array, block after block, each row-major.
 * ---------------------------------------------------------------------------------------- */
#define N_SOAP 12
static const int SOAP_OFF[N_SOAP] = {O_ARM_W1, O_ARM_W2, O_ARM_W3, O_ARM_WS, O_IF0_W, O_IF1_W,
                                     O_IF2_W, O_SYN_W1, O_SYN_W2, O_SYN_WS, O_CV1_W, O_CV2_W};
static const int SOAP_M[N_SOAP] = {AH, AH, 2, 2, NF, NF, NF, SH, NCH, NCH, NCH, NCH};
static const int SOAP_N[N_SOAP] = {AIN, AH, AH, AIN, 6, 5, 4, NG, SH, NG, 27, 27};

int orc_soap_blocks(int* off, int* m, int* n) {
    for (int b = 0; b < N_SOAP; ++b) {
        if (off) off[b] = SOAP_OFF[b];
        if (m) m[b] = SOAP_M[b];
        if (n) n[b] = SOAP_N[b];
    }
    return N_SOAP;
}

int64_t orc_soap_state_count(void) {
    int64_t t = 0;
    for (int b = 0; b < N_SOAP; ++b) t += 2 * ((int64_t)SOAP_M[b] * SOAP_M[b] + (int64_t)SOAP_N[b] * SOAP_N[b]);
    return t;
}

/* Eigen-decomposition of the symmetric n x n matrix A (row-major): Q (row-major, eigenvectors
 * as columns) and lam, ordered by decreasing eigenvalue, canonical signs. */
void orc_sym_eig(int n, const double* A_in, double* Q, double* lam) {
    double* A = (double*)malloc(sizeof(double) * n * n);
    double* V = (double*)malloc(sizeof(double) * n * n);
    memcpy(A, A_in, sizeof(double) * n * n);
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    double norm = 0.0;
    for (int i = 0; i < n * n; ++i) norm += A[i] * A[i];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += 2.0 * A[p * n + q] * A[p * n + q];
        if (off <= 1e-30 * norm || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < n; ++k) {
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    /* order by decreasing eigenvalue (selection sort), canonical sign per column */
    int* idx = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 0; i < n; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (A[idx[j] * n + idx[j]] > A[idx[best] * n + idx[best]]) best = j;
        const int tmp = idx[i];
        idx[i] = idx[best];
        idx[best] = tmp;
    }
    for (int j = 0; j < n; ++j) {
        const int src = idx[j];
        if (lam) lam[j] = A[src * n + src];
        int imax = 0;
        for (int i = 1; i < n; ++i)
            if (fabs(V[i * n + src]) > fabs(V[imax * n + src])) imax = i;
        const double sg = V[imax * n + src] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < n; ++i) Q[i * n + j] = sg * V[i * n + src];
    }
    free(idx);
    free(V);
    free(A);
}

/* C = op(A) * op(B) for small row-major matrices; ta / tb: use the transpose. */
static void small_gemm(int m, int n, int k, const double* A, int ta, const double* B, int tb, double* C) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int q = 0; q < k; ++q) {
                const double a = ta ? A[q * m + i] : A[i * k + q];
                const double b = tb ? B[j * k + q] : B[q * n + j];
                acc += a * b;
            }
            C[i * n + j] = acc;
        }
}

/* One optimizer step of the network parameters at Adam count t_new (the SOAP step is t_new - 1):
 * SOAP on the two-dimensional blocks (b1s, b2s, bshamp, freq), Adam (b1, b2) on the rest, both
 * with learning rate lr and eps. */
void orc_soap_params(int hyper, double* P, const double* g, double* m, double* v, double* S, int64_t t_new,
                     double lr, double b1, double b2, double b1s, double b2s, double bshamp, int freq, double eps) {
    const int NP = orc_param_count(hyper);
    int is_soap[N_PARAMS_H];
    for (int i = 0; i < NP; ++i) is_soap[i] = 0;
    for (int b = 0; b < N_SOAP; ++b)
        for (int i = 0; i < SOAP_M[b] * SOAP_N[b]; ++i) is_soap[SOAP_OFF[b] + i] = 1;
    /* Adam on the one-dimensional blocks */
    {
        const double bc1 = 1.0 - pow(b1, (double)t_new), bc2 = 1.0 - pow(b2, (double)t_new);
        for (int i = 0; i < NP; ++i) {
            if (is_soap[i]) continue;
            m[i] = b1 * m[i] + (1.0 - b1) * g[i];
            v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
            P[i] -= lr * (m[i] / bc1) / (sqrt(v[i] / bc2) + eps);
        }
    }
    const int64_t s = t_new - 1;
    double* st = S;
    for (int b = 0; b < N_SOAP; ++b) {
        const int M_ = SOAP_M[b], N_ = SOAP_N[b], off = SOAP_OFF[b];
        double* L = st;
        double* R = L + M_ * M_;
        double* QL = R + N_ * N_;
        double* QR = QL + M_ * M_;
        st = QR + N_ * N_;
        const double* G = g + off;
        double* W = P + off;
        double* Mb = m + off;
        double* Vb = v + off;
        double* GGt = (double*)malloc(sizeof(double) * M_ * M_);
        double* GtG = (double*)malloc(sizeof(double) * N_ * N_);
        small_gemm(M_, M_, N_, G, 0, G, 1, GGt);
        small_gemm(N_, N_, M_, G, 1, G, 0, GtG);
        if (s == 0) {
            for (int i = 0; i < M_ * M_; ++i) L[i] = (1.0 - bshamp) * GGt[i];
            for (int i = 0; i < N_ * N_; ++i) R[i] = (1.0 - bshamp) * GtG[i];
            orc_sym_eig(M_, L, QL, NULL);
            orc_sym_eig(N_, R, QR, NULL);
        } else {
            double* T = (double*)malloc(sizeof(double) * M_ * N_);
            double* Gr = (double*)malloc(sizeof(double) * M_ * N_);
            double* Mr = (double*)malloc(sizeof(double) * M_ * N_);
            double* Nr = (double*)malloc(sizeof(double) * M_ * N_);
            /* G' = Q_L^T G Q_R */
            small_gemm(M_, N_, M_, QL, 1, G, 0, T);
            small_gemm(M_, N_, N_, T, 0, QR, 0, Gr);
            for (int i = 0; i < M_ * N_; ++i) Mb[i] = b1s * Mb[i] + (1.0 - b1s) * G[i];
            small_gemm(M_, N_, M_, QL, 1, Mb, 0, T);
            small_gemm(M_, N_, N_, T, 0, QR, 0, Mr);
            const double bc1 = 1.0 - pow(b1s, (double)s), bc2 = 1.0 - pow(b2s, (double)s);
            for (int i = 0; i < M_ * N_; ++i) {
                Vb[i] = b2s * Vb[i] + (1.0 - b2s) * Gr[i] * Gr[i];
                Nr[i] = (Mr[i] / bc1) / (sqrt(Vb[i] / bc2) + eps);
            }
            /* N = Q_L N' Q_R^T */
            small_gemm(M_, N_, M_, QL, 0, Nr, 0, T);
            small_gemm(M_, N_, N_, T, 0, QR, 1, Gr);
            for (int i = 0; i < M_ * N_; ++i) W[i] -= lr * Gr[i];
            for (int i = 0; i < M_ * M_; ++i) L[i] = bshamp * L[i] + (1.0 - bshamp) * GGt[i];
            for (int i = 0; i < N_ * N_; ++i) R[i] = bshamp * R[i] + (1.0 - bshamp) * GtG[i];
            if (freq > 0 && s % freq == 0) {
                orc_sym_eig(M_, L, QL, NULL);
                orc_sym_eig(N_, R, QR, NULL);
            }
            free(T);
            free(Gr);
            free(Mr);
            free(Nr);
        }
        free(GGt);
        free(GtG);
    }
}

/* n_iters encoder iterations with the uniform proxy (as orc_encode), Adam on the latents and
 * SOAP / Adam on the network parameters (orc_soap_params). */
void orc_encode_soap(int H, int W, int hyper, const double* img, double* y, double* P, double* m_y, double* v_y,
                     double* m_p, double* v_p, double* S, int64_t* step, int n_iters, uint64_t seed, double lambda,
                     double lr, double b1, double b2, double b1s, double b2s, double bshamp, int freq, double eps,
                     double* loss_out) {
    int64_t N = orc_latent_count(H, W, hyper);
    double* gy = (double*)malloc(sizeof(double) * N);
    double gP[N_PARAMS_H];
    for (int it = 0; it < n_iters; ++it) {
        double rate, mse;
        double loss = orc_loss_grad(H, W, hyper, img, y, P, MODE_NOISE, seed, *step, 0.0, 1.0, lambda, &rate, &mse,
                                    gy, gP);
        if (loss_out) loss_out[it] = loss;
        *step += 1;
        orc_adam(N, y, gy, m_y, v_y, *step, lr, b1, b2, eps);
        orc_soap_params(hyper, P, gP, m_p, v_p, S, *step, lr, b1, b2, b1s, b2s, bshamp, freq, eps);
    }
    free(gy);
}
