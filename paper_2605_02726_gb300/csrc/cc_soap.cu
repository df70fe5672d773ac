// SOAP step of the network parameters (Sec. IV-B: SOAP for the networks, Adam for the latents).
//
// The paper names the optimizer (Vyas et al., "SOAP: Improving and Stabilizing Shampoo using
// Adam") without its settings; the step below is that paper's single-layer update.  For every
// two-dimensional weight block W (m x n; a residual convolution's kernel taken as [out][in * 9])
// with gradient G (reduced by the parameter-reduction kernel into the workspace):
//   SOAP step s = 0 (Adam count 1): L = (1 - bs) G G^T, R = (1 - bs) G^T G, Q_L, Q_R = their
//     eigenvectors; the block does not move;
//   s >= 1:  G' = Q_L^T G Q_R,  M = b1 M + (1 - b1) G,  M' = Q_L^T M Q_R,  V = b2 V + (1 - b2) G'^2
//     (element-wise, in the rotated coordinates),  N' = (M' / (1 - b1^s)) / (sqrt(V / (1 - b2^s)) + eps),
//     W -= lr Q_L N' Q_R^T,  L = bs L + (1 - bs) G G^T,  R = bs R + (1 - bs) G^T G, and every `freq`
//     steps Q_L, Q_R = the eigenvectors of the new L, R.
// Eigenvectors are the columns of Q, by decreasing eigenvalue, each with its entry of largest
// magnitude positive.  They come from the cyclic Jacobi method in its parallel (round-robin)
// ordering: in each of the n - 1 rounds of a sweep, n / 2 disjoint index pairs are rotated at
// once (the symmetric Schur 2 x 2 rotation of Golub and Van Loan), columns then rows; sweeps stop
// once the off-diagonal mass is at the level of FP32 rounding (at most kJacobiSweeps).  A refresh
// after the first starts from the previous eigenbasis Q (Jacobi on Q^T L Q, accumulating onto Q):
// the preconditioner moves little between refreshes, so that matrix is nearly diagonal and one or
// two sweeps finish it, where a cold start takes six to twelve.  Either way the result is an
// eigenbasis of the new L to FP32 accuracy; where eigenvalues coincide (the null space of a
// rank-deficient L) the basis is not unique and depends on the start.
//
// One CTA per block; every matrix of a block (at most 40 x 40) lives in shared memory.  M and V
// are the block's slots of the parameter moment arrays; L, R, Q_L, Q_R are in the caller's SOAP
// state array, block after block, each row-major.
#include "cc_kernels.h"

namespace cc {
namespace {

constexpr int kSoapThreads = 512;
constexpr int kSoapMaxDim = 40;
constexpr int kJacobiSweeps = 12;

// shapes of the 2-D blocks, in flat parameter order
constexpr int kSoapM[kSoapBlocks] = {16, 16, 2, 2, 4, 4, 4, 40, 3, 3, 3, 3};
constexpr int kSoapN[kSoapBlocks] = {20, 16, 16, 20, 6, 5, 4, 7, 40, 7, 27, 27};
constexpr int soap_max(bool area) {
    int r = 0;
    for (int b = 0; b < kSoapBlocks; ++b) {
        const int v = area ? kSoapM[b] * kSoapN[b] : (kSoapM[b] > kSoapN[b] ? kSoapM[b] : kSoapN[b]);
        r = v > r ? v : r;
    }
    return r;
}
static_assert(soap_max(false) <= kSoapMaxDim, "a SOAP block side exceeds the shared-memory matrices");

struct SoapBlock {
    int off, m, n, state;  // parameter offset, shape, offset in the SOAP state array
};
__device__ __forceinline__ SoapBlock soap_block(int b) {
    const int off[kSoapBlocks] = {po::arm_w1, po::arm_w2, po::arm_w3, po::arm_ws, po::if_w0, po::if_w1,
                                  po::if_w2, po::syn_w1, po::syn_w2, po::syn_ws, po::cv1_w, po::cv2_w};
    const int mm[kSoapBlocks] = {kSoapM[0], kSoapM[1], kSoapM[2], kSoapM[3], kSoapM[4], kSoapM[5],
                                 kSoapM[6], kSoapM[7], kSoapM[8], kSoapM[9], kSoapM[10], kSoapM[11]};
    const int nn[kSoapBlocks] = {kSoapN[0], kSoapN[1], kSoapN[2], kSoapN[3], kSoapN[4], kSoapN[5],
                                 kSoapN[6], kSoapN[7], kSoapN[8], kSoapN[9], kSoapN[10], kSoapN[11]};
    SoapBlock s;
    s.state = 0;
    for (int q = 0; q < b; ++q) s.state += 2 * (mm[q] * mm[q] + nn[q] * nn[q]);
    s.off = off[b];
    s.m = mm[b];
    s.n = nn[b];
    return s;
}

// C = op(A) op(B) (row-major, shapes after op: m x k times k x n); whole CTA, then a barrier.
__device__ void sm_gemm(int m, int n, int k, const float* A, bool ta, const float* B, bool tb, float* C) {
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        float acc = 0.f;
        for (int q = 0; q < k; ++q) acc = fmaf(ta ? A[q * m + i] : A[i * k + q], tb ? B[j * k + q] : B[q * n + j], acc);
        C[e] = acc;
    }
    __syncthreads();
}

// Eigenvectors of the symmetric n x n matrix A (destroyed) into Q (columns, by decreasing
// eigenvalue, canonical signs).  warm: Q holds an orthogonal basis on entry and A has already been
// rotated into it (A = Q^T L Q); the rotations then accumulate onto Q; otherwise they start from the
// identity.  V, cs, sn, lam, rank, pq are scratch.  Whole CTA.
__device__ void sm_sym_eig(int n, float* A, float* Q, float* V, float* cs, float* sn, float* lam, int* rank,
                           bool warm, int* pq) {
    const int n2 = n + (n & 1);  // a padding index (no row, no column) when n is odd
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = warm ? Q[e] : ((e / n == e % n) ? 1.f : 0.f);
    __syncthreads();
    const int np = n2 / 2;
    // Threshold Jacobi: an off-diagonal entry at or below 1e-6 of the Frobenius norm of A (which the
    // rotations preserve; a few times the FP32 rounding that the rotations themselves leave behind) is
    // treated as zero, and the sweeps stop after one that rotates nothing.  The eigenvectors then
    // carry an error of about 1e-6 |A| / gap, against the 2^-23 |A| / gap of exact convergence.
    __shared__ float s_nrm[kSoapThreads / 32];
    __shared__ int s_rot;
    float skip;
    {
        float t = 0.f;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) t += A[e] * A[e];
        t = warp_sum(t);
        if ((threadIdx.x & 31) == 0) s_nrm[threadIdx.x >> 5] = t;
        __syncthreads();
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_nrm[w];
        skip = 1e-6f * sqrtf(tot);
    }
#pragma unroll 1
    for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < n2 - 1; ++r) {
            // round r of the circle method: index n2-1 stays, the others turn; the pairs go to pq
            for (int k = threadIdx.x; k < np; k += blockDim.x) {
                int p, q;
                if (k == 0) {
                    p = r;
                    q = n2 - 1;
                } else {
                    p = (r + k) % (n2 - 1);
                    q = (r - k + (n2 - 1)) % (n2 - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                pq[2 * k] = p;
                pq[2 * k + 1] = q;
                float c = 1.f, s = 0.f;
                if (q < n) {
                    const float apq = A[p * n + q];
                    if (fabsf(apq) > skip) {
                        s_rot = 1;
                        const float tau = (A[q * n + q] - A[p * n + p]) / (2.f * apq);
                        const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
                        c = rsqrtf(1.f + t * t);
                        s = t * c;
                    }
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // A <- J^T A J and V <- V J in one pass: thread (a, b) rotates the 2 x 2 block of A on
            // rows {p_a, q_a} and columns {p_b, q_b} (each entry read and written once); thread
            // (row, b) rotates columns p_b, q_b of V on that row.  (q >= n: the padding index of an
            // odd n, no row or column.)
            for (int e = threadIdx.x; e < np * np + n * np; e += blockDim.x) {
                if (e < np * np) {
                    const int ka = e / np, kb = e - ka * np;
                    const int pa = pq[2 * ka], qa = pq[2 * ka + 1], pb = pq[2 * kb], qb = pq[2 * kb + 1];
                    const float ca = cs[ka], sa = sn[ka], cb = cs[kb], sb = sn[kb];
                    const bool ra = qa < n, rb = qb < n;
                    const float x00 = A[pa * n + pb], x01 = rb ? A[pa * n + qb] : 0.f;
                    const float x10 = ra ? A[qa * n + pb] : 0.f, x11 = ra && rb ? A[qa * n + qb] : 0.f;
                    // columns: (x_p, x_q) <- (c x_p - s x_q, s x_p + c x_q), then the same on rows
                    const float y00 = cb * x00 - sb * x01, y01 = sb * x00 + cb * x01;
                    const float y10 = cb * x10 - sb * x11, y11 = sb * x10 + cb * x11;
                    A[pa * n + pb] = ca * y00 - sa * y10;
                    if (rb) A[pa * n + qb] = ca * y01 - sa * y11;
                    if (ra) A[qa * n + pb] = sa * y00 + ca * y10;
                    if (ra && rb) A[qa * n + qb] = sa * y01 + ca * y11;
                } else {
                    const int f = e - np * np, kb = f / n, row = f - kb * n;
                    const int p = pq[2 * kb], q = pq[2 * kb + 1];
                    if (q >= n) continue;
                    const float c = cs[kb], s = sn[kb];
                    const float vkp = V[row * n + p], vkq = V[row * n + q];
                    V[row * n + p] = c * vkp - s * vkq;
                    V[row * n + q] = s * vkp + c * vkq;
                }
            }
            __syncthreads();
        }
        const bool done = s_rot == 0;
        __syncthreads();  // (every thread has read the flag before it is reset)
        if (done) break;
    }
    // order by decreasing eigenvalue (ties by index), canonical sign
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = A[i * n + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int rk = 0;
        for (int j = 0; j < n; ++j) rk += (lam[j] > lam[i] || (lam[j] == lam[i] && j < i)) ? 1 : 0;
        rank[i] = rk;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int imax = 0;
        for (int r = 1; r < n; ++r)
            if (fabsf(V[r * n + i]) > fabsf(V[imax * n + i])) imax = r;
        const float sg = V[imax * n + i] < 0.f ? -1.f : 1.f;
        const int col = rank[i];
        for (int r = 0; r < n; ++r) Q[r * n + col] = sg * V[r * n + i];
    }
    __syncthreads();
}

__device__ __forceinline__ void soap_body(const SoapArgs& a, int b) {
    if (a.hp.nn_opt != 1) return;
    const SoapBlock B = soap_block(b);
    const int m = B.m, n = B.n, mn = m * n;
    constexpr int kMN = soap_max(true), kSq = kSoapMaxDim * kSoapMaxDim;  // largest block, largest L or R
    __shared__ float G[kMN], Wt[kMN], M[kMN], V[kMN], T[kMN], Gr[kMN], Mr[kMN];
    __shared__ float L[kSq], R[kSq], QL[kSq], QR[kSq], GG[kSq], S1[kSq];
    __shared__ float cs[kSoapMaxDim], sn[kSoapMaxDim], lam[kSoapMaxDim];
    __shared__ int rank[kSoapMaxDim], pq[kSoapMaxDim + 2];
    __shared__ int64_t s_step;
    if (threadIdx.x == 0) s_step = *a.step_dev;
    float* st = a.soap + B.state;
    float* gL = st;
    float* gR = gL + m * m;
    float* gQL = gR + n * n;
    float* gQR = gQL + m * m;
    for (int e = threadIdx.x; e < mn; e += blockDim.x) {
        G[e] = a.grad[B.off + e];
        Wt[e] = a.params[B.off + e];
        M[e] = a.m[B.off + e];
        V[e] = a.v[B.off + e];
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        L[e] = gL[e];
        QL[e] = gQL[e];
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        R[e] = gR[e];
        QR[e] = gQR[e];
    }
    __syncthreads();
    const int64_t s = s_step;  // Adam count s_step + 1, SOAP step s_step
    const float bs = a.hp.sbs;
    bool refresh = s == 0;
    if (s == 0) {
        sm_gemm(m, m, n, G, false, G, true, GG);
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) L[e] = (1.f - bs) * GG[e];
        sm_gemm(n, n, m, G, true, G, false, GG);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) R[e] = (1.f - bs) * GG[e];
        __syncthreads();
    } else {
        // G' = Q_L^T G Q_R;  M;  M' = Q_L^T M Q_R
        sm_gemm(m, n, m, QL, true, G, false, T);
        sm_gemm(m, n, n, T, false, QR, false, Gr);
        for (int e = threadIdx.x; e < mn; e += blockDim.x) M[e] = a.hp.sb1 * M[e] + (1.f - a.hp.sb1) * G[e];
        __syncthreads();
        sm_gemm(m, n, m, QL, true, M, false, T);
        sm_gemm(m, n, n, T, false, QR, false, Mr);
        float bc1, bc2;
        adam_bias_corrections(s, a.hp.sb1, a.hp.sb2, bc1, bc2);
        for (int e = threadIdx.x; e < mn; e += blockDim.x) {
            V[e] = a.hp.sb2 * V[e] + (1.f - a.hp.sb2) * Gr[e] * Gr[e];
            Mr[e] = (Mr[e] / bc1) / (sqrtf(V[e] / bc2) + a.hp.eps);  // N'
        }
        __syncthreads();
        // W -= lr Q_L N' Q_R^T
        sm_gemm(m, n, m, QL, false, Mr, false, T);
        sm_gemm(m, n, n, T, false, QR, true, Gr);
        const float lr = proxy_at(a.hp, s).lr;
        for (int e = threadIdx.x; e < mn; e += blockDim.x) Wt[e] -= lr * Gr[e];
        sm_gemm(m, m, n, G, false, G, true, GG);
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) L[e] = bs * L[e] + (1.f - bs) * GG[e];
        sm_gemm(n, n, m, G, true, G, false, GG);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) R[e] = bs * R[e] + (1.f - bs) * GG[e];
        __syncthreads();
        refresh = a.hp.sfreq > 0 && s % a.hp.sfreq == 0;
    }
    if (refresh) {
        // warm start (s > 0): rotate the new preconditioner into the previous eigenbasis first
        const bool warm = s > 0;
        if (warm) {
            sm_gemm(m, m, m, QL, true, L, false, GG);
            sm_gemm(m, m, m, GG, false, QL, false, S1);
        } else {
            for (int e = threadIdx.x; e < m * m; e += blockDim.x) S1[e] = L[e];
            __syncthreads();
        }
        sm_sym_eig(m, S1, QL, GG, cs, sn, lam, rank, warm, pq);
        if (warm) {
            sm_gemm(n, n, n, QR, true, R, false, GG);
            sm_gemm(n, n, n, GG, false, QR, false, S1);
        } else {
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) S1[e] = R[e];
            __syncthreads();
        }
        sm_sym_eig(n, S1, QR, GG, cs, sn, lam, rank, warm, pq);
    }
    for (int e = threadIdx.x; e < mn; e += blockDim.x) {
        a.params[B.off + e] = Wt[e];
        a.m[B.off + e] = M[e];
        a.v[B.off + e] = V[e];
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        gL[e] = L[e];
        gQL[e] = QL[e];
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        gR[e] = R[e];
        gQR[e] = QR[e];
    }
}

__global__ void __launch_bounds__(kSoapThreads) k_soap(const __grid_constant__ SoapArgs a) {
    pdl_enter();
    soap_body(a, blockIdx.x);
}
__global__ void __launch_bounds__(kSoapThreads) k_soap_b(Batch<SoapArgs> b) {
    __shared__ SoapArgs sa;
    const int j = batch_job(b.cta_begin, b.njobs);
    batch_fetch(b.args, j, sa);
    soap_body(sa, blockIdx.x - b.cta_begin[j]);
}

}  // namespace

int64_t soap_state_floats() {
    int64_t t = 0;
    for (int b = 0; b < kSoapBlocks; ++b) t += 2 * (kSoapM[b] * kSoapM[b] + kSoapN[b] * kSoapN[b]);
    return t;
}

SoapArgs soap_args(const Work& w, float* params, float* m, float* v, float* soap, const Hp& hp,
                   const int64_t* step_dev) {
    SoapArgs a;
    a.grad = w.grad_params;
    a.params = params;
    a.m = m;
    a.v = v;
    a.soap = soap;
    a.step_dev = step_dev;
    a.hp = hp;
    return a;
}

void launch_soap(const Work& w, float* params, float* m, float* v, float* soap, const Hp& hp,
                 const int64_t* step_dev, cudaStream_t s) {
    launch_pdl(k_soap, kSoapBlocks, kSoapThreads, 0, s, soap_args(w, params, m, v, soap, hp, step_dev));
}

void launch_soap_b(const Batch<SoapArgs>& b, cudaStream_t s) {
    launch_pdl(k_soap_b, b.total_ctas, kSoapThreads, 0, s, b);
}

}  // namespace cc
