// Learned re-rank depth (the engine's F1 extension to §4.3.2 Stage 3) for sm_103a.
//
//   k_features      per-query feature row (score histogram of C, traversal costs, sizes)
//   k_mlp_infer     MLP F -> H -> H -> O in the fixed FP32 order (+ depth quantisation)
//   k_select_score  the first d candidates by (V desc, id asc), written in ascending id
//   k_label_v/_s    depth labels from the plain search (training data)
//   k_gemm, ...     training: SIMT GEMMs, GELU forward/backward, MSE gradient, Adam
//
// GELU uses erf by Abramowitz & Stegun 7.1.28 (a polynomial, four squarings and a
// division), so inference is reproducible bit for bit from the parameters.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <random>
#include <vector>

#include "internal.cuh"

namespace {

constexpr float kA1 = 0.0705230784f, kA2 = 0.0422820123f, kA3 = 0.0092705272f, kA4 = 0.0001520143f,
                kA5 = 0.0002765672f, kA6 = 0.0000430638f;
constexpr float kInvSqrt2 = 0.70710678118654752f;

__device__ __forceinline__ float erf_as(float u) {
    float a = fabsf(u);
    float p = kA6;
    p = fmaf(p, a, kA5);
    p = fmaf(p, a, kA4);
    p = fmaf(p, a, kA3);
    p = fmaf(p, a, kA2);
    p = fmaf(p, a, kA1);
    p = fmaf(p, a, 1.0f);
    float p2 = p * p, p4 = p2 * p2, p8 = p4 * p4, p16 = p8 * p8;
    float e = 1.0f - 1.0f / p16;
    return u < 0.0f ? -e : e;
}

__device__ __forceinline__ float gelu_as(float z) {
    float u = z * kInvSqrt2;
    return (0.5f * z) * (1.0f + erf_as(u));
}

// derivative of gelu_as (training only)
__device__ __forceinline__ float gelu_as_grad(float z) {
    float u = z * kInvSqrt2, a = fabsf(u);
    float p = kA6;
    p = fmaf(p, a, kA5);
    p = fmaf(p, a, kA4);
    p = fmaf(p, a, kA3);
    p = fmaf(p, a, kA2);
    p = fmaf(p, a, kA1);
    p = fmaf(p, a, 1.0f);
    float dp = 6.0f * kA6;
    dp = fmaf(dp, a, 5.0f * kA5);
    dp = fmaf(dp, a, 4.0f * kA4);
    dp = fmaf(dp, a, 3.0f * kA3);
    dp = fmaf(dp, a, 2.0f * kA2);
    dp = fmaf(dp, a, kA1);
    float p2 = p * p, p4 = p2 * p2, p8 = p4 * p4, p16 = p8 * p8, p17 = p16 * p;
    float e = 1.0f - 1.0f / p16;
    float erf = u < 0.0f ? -e : e;
    float derf = 16.0f * dp / p17;
    return 0.5f * (1.0f + erf) + 0.5f * z * derf * kInvSqrt2;
}

// depth = ceil(2^(j/4)), j = ceil(4 (y + margin)) in FP32, clamped to [lo, hi]
__device__ long long depth_q(float y, float margin, long long lo, long long hi) {
    float t = 4.0f * (y + margin);
    if (!(t < 120.0f)) return hi;
    if (t < -120.0f) return lo;
    int j = (int)ceilf(t);
    int q = j >= 0 ? j / 4 : -((-j + 3) / 4);
    int r = j - 4 * q;
    double s2 = sqrt(2.0), s4 = sqrt(s2);
    double fr = r == 0 ? 1.0 : r == 1 ? s4 : r == 2 ? s2 : s2 * s4;
    double v = ceil(ldexp(fr, q));
    long long d = v > 9.0e18 ? hi : (long long)v;
    if (d < lo) d = lo;
    if (d > hi) d = hi;
    return d;
}

template <int NT>
__device__ __forceinline__ long long block_excl_scan_l(long long v, long long *ws, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < NT / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NT / 32) ws[lane] = t;
        if (lane == NT / 32 - 1) ws[NT / 32] = t;
    }
    __syncthreads();
    long long excl = x - v + (warp > 0 ? ws[warp - 1] : 0);
    *total = ws[NT / 32];
    __syncthreads();
    return excl;
}

template <int NT>
__device__ __forceinline__ long long block_sum_l(long long v, long long *ws) {
    long long tot;
    block_excl_scan_l<NT>(v, ws, &tot);
    return tot;
}

constexpr int LF_NT = 256;

// ------------------------------------------------------------- features
__global__ void __launch_bounds__(LF_NT) k_features(const int *__restrict__ cand, long long stride,
                                                    const long long *__restrict__ ncand,
                                                    const uint8_t *__restrict__ score, const float *__restrict__ cfirst,
                                                    const float *__restrict__ clast, int M, long long N, int kk, int tau,
                                                    const QParam *__restrict__ qp, float *__restrict__ feats) {
    __shared__ unsigned hist[64];
    const int q = blockIdx.x, F = 2 * M + 68;
    if (qp) {                           // per-query parameters
        kk = qp[q].k;
        tau = qp[q].tau;
    }
    long long n = ncand[q];
    if (n > stride) n = stride;
    for (int i = threadIdx.x; i < 64; i += LF_NT) hist[i] = 0;
    __syncthreads();
    const uint8_t *sq = score + (long long)q * stride;
    for (long long i = threadIdx.x; i < n; i += LF_NT) atomicAdd(&hist[sq[i] < 63 ? sq[i] : 63], 1u);
    __syncthreads();
    float *f = feats + (long long)q * F;
    const float den = (float)(n > 0 ? n : 1);
    for (int s = threadIdx.x; s < 64; s += LF_NT) f[s] = (float)hist[s] / den;
    if (threadIdx.x == 0) {
        const float *cf = cfirst + (long long)q * M, *cl = clast + (long long)q * M;
        float norm = 0.0f;
        for (int m = 0; m < M; ++m) norm = norm + cl[m];
        if (!(norm > 0.0f)) norm = 1.0f;
        for (int m = 0; m < M; ++m) {
            f[64 + m] = cf[m] / norm;
            f[64 + M + m] = cl[m] / norm;
        }
        long long v = n + 1;
        int lg = 0;
        while (v > 1) { v >>= 1; ++lg; }
        f[64 + 2 * M] = (float)n / (float)N;
        f[64 + 2 * M + 1] = (float)lg / 32.0f;
        f[64 + 2 * M + 2] = (float)kk / 256.0f;
        f[64 + 2 * M + 3] = (float)tau / (float)M;
    }
}

// ------------------------------------------------------- MLP inference
constexpr int MI_QPB = 8, MI_NT = 256;

// Y (or the two depths) of up to MI_QPB queries per block; every unit is an
// fmaf chain over its inputs in order, from its bias.  H <= MI_NT, O <= 8.
template <bool DEPTH>
__global__ void __launch_bounds__(MI_NT) k_mlp_infer(const float *__restrict__ P, int F, int H, int O,
                                                     const float *__restrict__ X, long long B, float *__restrict__ Y,
                                                     const long long *__restrict__ ncand, long long stride, int kk,
                                                     float mV, float mS, const QParam *__restrict__ qp,
                                                     long long *__restrict__ dV, long long *__restrict__ dS) {
    extern __shared__ float sm[];
    float *x = sm;                      // [QPB][F]
    float *h1 = x + MI_QPB * F;         // [QPB][H]
    float *h2 = h1 + MI_QPB * H;        // [QPB][H]
    __shared__ float y[MI_QPB][8];
    const long long q0 = (long long)blockIdx.x * MI_QPB;
    const int nb = (int)(B - q0 < MI_QPB ? B - q0 : MI_QPB);
    for (int e = threadIdx.x; e < nb * F; e += MI_NT) x[e] = X[q0 * F + e];
    __syncthreads();
    const float *W1 = P, *b1 = W1 + (long long)F * H, *W2 = b1 + H, *b2 = W2 + (long long)H * H, *W3 = b2 + H,
                *b3 = W3 + (long long)H * O;
    const int j = threadIdx.x;
    float z[MI_QPB];
    if (j < H) {
#pragma unroll
        for (int qi = 0; qi < MI_QPB; ++qi) z[qi] = b1[j];
        for (int i = 0; i < F; ++i) {
            float w = W1[(long long)i * H + j];
#pragma unroll
            for (int qi = 0; qi < MI_QPB; ++qi)
                if (qi < nb) z[qi] = fmaf(x[qi * F + i], w, z[qi]);
        }
#pragma unroll
        for (int qi = 0; qi < MI_QPB; ++qi)
            if (qi < nb) h1[qi * H + j] = gelu_as(z[qi]);
    }
    __syncthreads();
    if (j < H) {
#pragma unroll
        for (int qi = 0; qi < MI_QPB; ++qi) z[qi] = b2[j];
        for (int i = 0; i < H; ++i) {
            float w = W2[(long long)i * H + j];
#pragma unroll
            for (int qi = 0; qi < MI_QPB; ++qi)
                if (qi < nb) z[qi] = fmaf(h1[qi * H + i], w, z[qi]);
        }
#pragma unroll
        for (int qi = 0; qi < MI_QPB; ++qi)
            if (qi < nb) h2[qi * H + j] = gelu_as(z[qi]);
    }
    __syncthreads();
    if (threadIdx.x < nb * O) {
        int qi = threadIdx.x / O, o = threadIdx.x % O;
        float acc = b3[o];
        for (int jj = 0; jj < H; ++jj) acc = fmaf(h2[qi * H + jj], W3[(long long)jj * O + o], acc);
        y[qi][o] = acc;
        if (!DEPTH) Y[(q0 + qi) * O + o] = acc;
    }
    __syncthreads();
    if (DEPTH && threadIdx.x < nb) {
        long long q = q0 + threadIdx.x;
        if (qp) {                       // per-query parameters
            kk = qp[q].k;
            mV = qp[q].mV;
            mS = qp[q].mS;
        }
        long long n = ncand[q] < stride ? ncand[q] : stride;
        long long v = depth_q(y[threadIdx.x][0], mV, kk, n > kk ? n : kk);
        if (v > n) v = n;
        long long s = depth_q(y[threadIdx.x][1], mS, kk, v > kk ? v : kk);
        dV[q] = v;
        dS[q] = s;
    }
}

// ---------------------------------------------- selection by collision score
// The first depth[q] candidates by (V desc, id asc), written in ascending id.
__global__ void __launch_bounds__(LF_NT) k_select_score(const int *__restrict__ cand, long long stride,
                                                        const long long *__restrict__ ncand,
                                                        const uint8_t *__restrict__ score,
                                                        const long long *__restrict__ depth, int *__restrict__ out,
                                                        long long *__restrict__ nout) {
    __shared__ unsigned hist[256];
    __shared__ long long ws[LF_NT / 32 + 1];
    __shared__ int s_star;
    __shared__ long long s_need;
    const int q = blockIdx.x;
    long long n = ncand[q];
    if (n > stride) n = stride;
    long long d = depth[q];
    const int *cq = cand + (long long)q * stride;
    const uint8_t *sq = score + (long long)q * stride;
    int *oq = out + (long long)q * stride;
    if (d >= n) {
        for (long long i = threadIdx.x; i < n; i += LF_NT) oq[i] = cq[i];
        if (threadIdx.x == 0) nout[q] = n;
        return;
    }
    for (int i = threadIdx.x; i < 256; i += LF_NT) hist[i] = 0;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += LF_NT) atomicAdd(&hist[sq[i]], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        long long above = 0;
        int s = 255;
        for (; s > 0; --s) {
            if (above + hist[s] >= d) break;
            above += hist[s];
        }
        s_star = s;
        s_need = d - above;
    }
    __syncthreads();
    const int ss = s_star;
    const long long need = s_need;
    long long eq_seen = 0, sel_seen = 0;
    for (long long c0 = 0; c0 < n; c0 += LF_NT) {
        long long i = c0 + threadIdx.x;
        int v = i < n ? sq[i] : -1;
        long long eq_tot, sel_tot;
        long long eq_off = block_excl_scan_l<LF_NT>(v == ss ? 1 : 0, ws, &eq_tot);
        int sel = (i < n) && (v > ss || (v == ss && eq_seen + eq_off < need));
        long long sel_off = block_excl_scan_l<LF_NT>(sel, ws, &sel_tot);
        if (sel) oq[sel_seen + sel_off] = cq[i];
        eq_seen += eq_tot;
        sel_seen += sel_tot;
    }
    if (threadIdx.x == 0) nout[q] = sel_seen;
}

// ----------------------------------------------------------------- labels
__device__ long long find_sorted(const int *a, long long n, int x) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// depth_V* = 1 + max over the top-k ids r of #{c : V_c > V_r or (V_c = V_r and c < r)}
__global__ void __launch_bounds__(LF_NT) k_label_v(const int *__restrict__ cand, long long stride,
                                                   const long long *__restrict__ ncand,
                                                   const uint8_t *__restrict__ score, const long long *__restrict__ top,
                                                   int kk, long long *__restrict__ depthV) {
    __shared__ long long ws[LF_NT / 32 + 1];
    const int q = blockIdx.x;
    long long n = ncand[q] < stride ? ncand[q] : stride;
    const int *cq = cand + (long long)q * stride;
    const uint8_t *sq = score + (long long)q * stride;
    long long best = -1;
    for (int t = 0; t < kk; ++t) {
        long long r = top[(long long)q * kk + t];
        if (r < 0) continue;
        long long ir = find_sorted(cq, n, (int)r);
        if (ir >= n || cq[ir] != (int)r) continue;      // not a candidate (cannot happen: top-k comes from C)
        int vr = sq[ir];
        long long c = 0;
        for (long long i = threadIdx.x; i < n; i += LF_NT) {
            int v = sq[i];
            c += (v > vr) || (v == vr && cq[i] < r);
        }
        long long pos = block_sum_l<LF_NT>(c, ws);
        best = pos > best ? pos : best;
    }
    if (threadIdx.x == 0) depthV[q] = best >= 0 ? best + 1 : kk;
}

// depth_S* = 1 + max over the top-k ids r of #{c in P : (d_c, c) < (d_r, r)}
__global__ void __launch_bounds__(LF_NT) k_label_s(const int *__restrict__ Pl, long long stride,
                                                   const long long *__restrict__ nP, const float *__restrict__ dist,
                                                   const long long *__restrict__ top, int kk,
                                                   long long *__restrict__ depthS) {
    __shared__ long long ws[LF_NT / 32 + 1];
    const int q = blockIdx.x;
    long long n = nP[q] < stride ? nP[q] : stride;
    const int *pq = Pl + (long long)q * stride;
    const float *dq = dist + (long long)q * stride;
    long long best = -1;
    for (int t = 0; t < kk; ++t) {
        long long r = top[(long long)q * kk + t];
        if (r < 0) continue;
        long long ir = find_sorted(pq, n, (int)r);
        if (ir >= n || pq[ir] != (int)r) continue;      // not in the prefix (cannot happen by construction)
        float dr = dq[ir];
        long long c = 0;
        for (long long i = threadIdx.x; i < n; i += LF_NT) {
            float d = dq[i];
            c += (d < dr) || (d == dr && pq[i] < r);
        }
        long long pos = block_sum_l<LF_NT>(c, ws);
        best = pos > best ? pos : best;
    }
    if (threadIdx.x == 0) depthS[q] = best >= 0 ? best + 1 : kk;
}

__global__ void k_log2_targets(const long long *__restrict__ dV, const long long *__restrict__ dS, int nq,
                               long long *__restrict__ labels, float *__restrict__ targets) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    labels[2 * q] = dV[q];
    labels[2 * q + 1] = dS[q];
    if (targets) {
        targets[2 * q] = log2f((float)dV[q]);
        targets[2 * q + 1] = log2f((float)dS[q]);
    }
}

// --------------------------------------------------------------- training
constexpr int GT = 64, GK = 16;

// C[m][n] = sum_k opA(m, k) opB(k, n); opA = A^T when TA, opB = B^T when TB
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                              const float *__restrict__ Bm, int ldb, float *__restrict__ C, int ldc) {
    __shared__ float As[GK][GT + 1], Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int r = e / GK, c = e % GK;        // r: row of the tile (m or n), c: k
            int m = m0 + r, k = k0 + c;
            float a = 0.0f;
            if (m < M && k < K) a = TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k];
            As[c][r] = a;
            int n = n0 + r;
            float b = 0.0f;
            if (n < N && k < K) b = TB ? Bm[(long long)n * ldb + k] : Bm[(long long)k * ldb + n];
            Bs[c][r] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty + 16 * u]; b[u] = Bs[kk][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int m = m0 + ty + 16 * u, n = n0 + tx + 16 * v;
            if (m < M && n < N) C[(long long)m * ldc + n] = acc[u][v];
        }
}

// Z += b (per column); Hout = gelu(Z) when given
__global__ void k_bias_act(float *__restrict__ Z, const float *__restrict__ b, long long rows, int cols,
                           float *__restrict__ Hout) {
    long long tot = rows * cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        float z = Z[e] + b[e % cols];
        Z[e] = z;
        if (Hout) Hout[e] = gelu_as(z);
    }
}

__global__ void k_gelu_bwd(float *__restrict__ dZ, const float *__restrict__ Z, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dZ[e] *= gelu_as_grad(Z[e]);
}

__global__ void k_colsum(const float *__restrict__ A, long long rows, int cols, float *__restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (long long r = 0; r < rows; ++r) s += A[r * cols + c];
    out[c] = s;
}

__global__ void k_mse(const float *__restrict__ Y, const float *__restrict__ T, long long n, float *__restrict__ dY,
                      float *__restrict__ loss) {
    __shared__ float red[32];
    float s = 0.0f;
    const float sc = 2.0f / (float)n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float d = Y[e] - T[e];
        dY[e] = sc * d;
        s += d * d;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) atomicAdd(loss, t / (float)n);
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float gg = g[e];
        float mm = b1 * m[e] + (1.0f - b1) * gg;
        float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Xavier-uniform weights (bound sqrt(6 / (fan_in + fan_out))), zero biases
__global__ void k_mlp_init(float *__restrict__ P, int F, int H, int O, unsigned long long seed) {
    const long long sizes[6] = {(long long)F * H, H, (long long)H * H, H, (long long)H * O, O};
    const int fin[6] = {F, 0, H, 0, H, 0}, fout[6] = {H, 0, H, 0, O, 0};
    long long total = 0;
    for (int s = 0; s < 6; ++s) total += sizes[s];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long off = e;
        int s = 0;
        while (off >= sizes[s]) { off -= sizes[s]; ++s; }
        if (fin[s] == 0) { P[e] = 0.0f; continue; }
        unsigned long long r = splitmix64(seed ^ (unsigned long long)(e * 0x632BE59BD9B4E019ull));
        float u = (float)((r >> 40) * (1.0 / 16777216.0));   // [0, 1)
        float bound = sqrtf(6.0f / (float)(fin[s] + fout[s]));
        P[e] = (2.0f * u - 1.0f) * bound;
    }
}

__global__ void k_gather_f(const float *__restrict__ X, int cols, const long long *__restrict__ idx, long long B,
                           float *__restrict__ out) {
    long long tot = B * cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
        out[e] = X[idx[e / cols] * cols + e % cols];
}

unsigned g1(long long n, int nt) { return (unsigned)std::min<long long>((n + nt - 1) / nt, 152LL * 64); }

template <bool TA, bool TB>
void gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc, cudaStream_t st) {
    dim3 g((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm<TA, TB><<<g, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

struct MlpWork {
    float *Z1, *H1, *Z2, *H2, *Y, *dY, *dA, *dB;
};

// forward of a batch keeping the activations; then the MSE gradient and backward
crisp_status mlp_loss_grad(const float *P, int F, int H, int O, const float *X, const float *T, long long B,
                           float *G, float *loss, const MlpWork &w, cudaStream_t st) {
    const float *W1 = P, *b1 = W1 + (long long)F * H, *W2 = b1 + H, *b2 = W2 + (long long)H * H, *W3 = b2 + H,
                *b3 = W3 + (long long)H * O;
    float *gW1 = G, *gb1 = gW1 + (long long)F * H, *gW2 = gb1 + H, *gb2 = gW2 + (long long)H * H, *gW3 = gb2 + H,
          *gb3 = gW3 + (long long)H * O;
    int Bi = (int)B;
    gemm<false, false>(Bi, H, F, X, F, W1, H, w.Z1, H, st);
    k_bias_act<<<g1(B * H, 256), 256, 0, st>>>(w.Z1, b1, B, H, w.H1);
    gemm<false, false>(Bi, H, H, w.H1, H, W2, H, w.Z2, H, st);
    k_bias_act<<<g1(B * H, 256), 256, 0, st>>>(w.Z2, b2, B, H, w.H2);
    gemm<false, false>(Bi, O, H, w.H2, H, W3, O, w.Y, O, st);
    k_bias_act<<<g1(B * O, 256), 256, 0, st>>>(w.Y, b3, B, O, nullptr);
    CRISP_CK(cudaMemsetAsync(loss, 0, sizeof(float), st));
    k_mse<<<std::min<long long>(g1(B * O, 256), 64), 256, 0, st>>>(w.Y, T, B * O, w.dY, loss);
    // layer 3
    gemm<true, false>(H, O, Bi, w.H2, H, w.dY, O, gW3, O, st);
    k_colsum<<<(O + 127) / 128, 128, 0, st>>>(w.dY, B, O, gb3);
    gemm<false, true>(Bi, H, O, w.dY, O, W3, O, w.dA, H, st);
    k_gelu_bwd<<<g1(B * H, 256), 256, 0, st>>>(w.dA, w.Z2, B * H);
    // layer 2
    gemm<true, false>(H, H, Bi, w.H1, H, w.dA, H, gW2, H, st);
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(w.dA, B, H, gb2);
    gemm<false, true>(Bi, H, H, w.dA, H, W2, H, w.dB, H, st);
    k_gelu_bwd<<<g1(B * H, 256), 256, 0, st>>>(w.dB, w.Z1, B * H);
    // layer 1
    gemm<true, false>(F, H, Bi, X, F, w.dB, H, gW1, H, st);
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(w.dB, B, H, gb1);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

size_t mlp_work_floats(int H, int O, long long B) { return (size_t)B * (4 * H + 2 * O + 2 * H); }

MlpWork carve_work(float *base, int H, int O, long long B) {
    MlpWork w;
    w.Z1 = base;
    w.H1 = w.Z1 + B * H;
    w.Z2 = w.H1 + B * H;
    w.H2 = w.Z2 + B * H;
    w.Y = w.H2 + B * H;
    w.dY = w.Y + B * O;
    w.dA = w.dY + B * O;
    w.dB = w.dA + B * H;
    return w;
}

}  // namespace

// ================================================================== launchers
crisp_status crisp_run_features(const crisp_index *ix, const int32_t *cand, int64_t stride, const int64_t *ncand,
                                const uint8_t *score, const float *cfirst, const float *clast, int32_t nq, int32_t k,
                                int32_t tau, float *feats, cudaStream_t st, const QParam *qp) {
    if (nq <= 0) return CRISP_OK;
    k_features<<<nq, LF_NT, 0, st>>>(cand, (long long)stride, (const long long *)ncand, score, cfirst, clast, ix->M,
                                     (long long)ix->N, k, tau, qp, feats);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

static size_t infer_smem(int F, int H) { return sizeof(float) * (size_t)MI_QPB * (F + 2 * H); }

crisp_status crisp_run_mlp_depth(const crisp_index *ix, const float *feats, int32_t nq, const int64_t *ncand,
                                 int64_t stride, int32_t k, float mV, float mS, int64_t *dV, int64_t *dS,
                                 cudaStream_t st, const QParam *qp) {
    if (nq <= 0) return CRISP_OK;
    int F = 2 * ix->M + 68, H = ix->mlp_H;
    size_t smem = infer_smem(F, H);
    CRISP_CK(cudaFuncSetAttribute(k_mlp_infer<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_infer<true><<<(nq + MI_QPB - 1) / MI_QPB, MI_NT, smem, st>>>(
        ix->mlp, F, H, 2, feats, nq, nullptr, (const long long *)ncand, (long long)stride, k, mV, mS, qp,
        (long long *)dV, (long long *)dS);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_select_score(const int32_t *cand, int64_t stride, const int64_t *ncand, const uint8_t *score,
                                    const int64_t *depth, int32_t nq, int32_t *out, int64_t *nout, cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    k_select_score<<<nq, LF_NT, 0, st>>>(cand, (long long)stride, (const long long *)ncand, score,
                                         (const long long *)depth, out, (long long *)nout);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_labels_v(const int32_t *cand, int64_t stride, const int64_t *ncand, const uint8_t *score,
                                const int64_t *top, int32_t k, int32_t nq, int64_t *dV, cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    k_label_v<<<nq, LF_NT, 0, st>>>(cand, (long long)stride, (const long long *)ncand, score, (const long long *)top, k,
                                    (long long *)dV);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_labels_s(const int32_t *P, int64_t stride, const int64_t *nP, const float *dist,
                                const int64_t *top, int32_t k, int32_t nq, int64_t *dS, cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    k_label_s<<<nq, LF_NT, 0, st>>>(P, (long long)stride, (const long long *)nP, dist, (const long long *)top, k,
                                    (long long *)dS);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_log2_targets(const int64_t *dV, const int64_t *dS, int32_t nq, int64_t *labels, float *targets,
                                    cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    k_log2_targets<<<(nq + 255) / 256, 256, 0, st>>>((const long long *)dV, (const long long *)dS, nq,
                                                     (long long *)labels, targets);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

// ===================================================================== C ABI
extern "C" int64_t crisp_mlp_param_count(int32_t F, int32_t H, int32_t O) {
    return (int64_t)F * H + H + (int64_t)H * H + H + (int64_t)H * O + O;
}

static crisp_status check_mlp(int32_t F, int32_t H, int32_t O) {
    CRISP_REQUIRE(F >= 1 && H >= 1 && H <= MI_NT && O >= 1 && O <= 8, "MLP sizes: need F >= 1, 1 <= H <= 256, 1 <= O <= 8");
    return CRISP_OK;
}

extern "C" crisp_status crisp_mlp_init(float *params, int32_t F, int32_t H, int32_t O, uint64_t seed, void *stream) {
    crisp_status s = check_mlp(F, H, O);
    if (s) return s;
    CRISP_REQUIRE(params, "crisp_mlp_init: null params");
    long long n = crisp_mlp_param_count(F, H, O);
    k_mlp_init<<<g1(n, 256), 256, 0, as_stream(stream)>>>(params, F, H, O, (unsigned long long)seed);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

extern "C" crisp_status crisp_mlp_infer(const float *params, int32_t F, int32_t H, int32_t O, const float *X, int64_t B,
                                        float *Y, void *stream) {
    crisp_status s = check_mlp(F, H, O);
    if (s) return s;
    CRISP_REQUIRE(params && X && Y && B >= 0, "crisp_mlp_infer: bad arguments");
    if (B == 0) return CRISP_OK;
    size_t smem = infer_smem(F, H);
    CRISP_REQUIRE(smem <= 220 * 1024, "crisp_mlp_infer: F + 2H too large for shared memory");
    CRISP_CK(cudaFuncSetAttribute(k_mlp_infer<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_infer<false><<<(unsigned)((B + MI_QPB - 1) / MI_QPB), MI_NT, smem, as_stream(stream)>>>(
        params, F, H, O, X, (long long)B, Y, nullptr, 0, 0, 0.0f, 0.0f, nullptr, nullptr, nullptr);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

extern "C" crisp_status crisp_mlp_loss_grad(const float *params, int32_t F, int32_t H, int32_t O, const float *X,
                                            const float *T, int64_t B, float *grads, float *loss, void *stream) {
    crisp_status s = check_mlp(F, H, O);
    if (s) return s;
    CRISP_REQUIRE(params && X && T && grads && loss && B >= 1 && B < (1LL << 31), "crisp_mlp_loss_grad: bad arguments");
    cudaStream_t st = as_stream(stream);
    float *wb = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&wb, sizeof(float) * mlp_work_floats(H, O, B), st));
    s = mlp_loss_grad(params, F, H, O, X, T, B, grads, loss, carve_work(wb, H, O, B), st);
    crisp_scratch_free(wb, st);
    return s;
}

extern "C" crisp_status crisp_mlp_adam(float *params, const float *grads, float *m, float *v, int64_t n, float lr,
                                       float beta1, float beta2, float eps, int32_t t, void *stream) {
    CRISP_REQUIRE(params && grads && m && v && n >= 0 && t >= 1, "crisp_mlp_adam: bad arguments");
    if (n == 0) return CRISP_OK;
    float bc1 = 1.0f - powf(beta1, (float)t), bc2 = 1.0f - powf(beta2, (float)t);
    k_adam<<<g1(n, 256), 256, 0, as_stream(stream)>>>(params, grads, m, v, n, lr, beta1, beta2, eps, bc1, bc2);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

extern "C" crisp_status crisp_mlp_train(float *params, int32_t F, int32_t H, int32_t O, const float *X, const float *T,
                                        int64_t n, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                        float *epoch_loss, void *stream) {
    crisp_status s = check_mlp(F, H, O);
    if (s) return s;
    CRISP_REQUIRE(params && X && T && n >= 1 && epochs >= 0 && batch >= 1, "crisp_mlp_train: bad arguments");
    cudaStream_t st = as_stream(stream);
    const long long B = std::min<long long>(batch, n);
    const long long np = crisp_mlp_param_count(F, H, O);
    size_t fl = mlp_work_floats(H, O, B) + (size_t)B * (F + O) + 3 * (size_t)np + 1;
    float *wb = nullptr;
    long long *perm = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&wb, sizeof(float) * fl, st));
    CRISP_CK(crisp_scratch_alloc((void **)&perm, sizeof(long long) * (size_t)n, st));
    MlpWork w = carve_work(wb, H, O, B);
    float *Xb = wb + mlp_work_floats(H, O, B), *Tb = Xb + B * F, *G = Tb + B * O, *mm = G + np, *vv = mm + np,
          *loss = vv + np;
    CRISP_CK(cudaMemsetAsync(mm, 0, sizeof(float) * 2 * np, st));
    std::vector<long long> hp((size_t)n);
    for (long long i = 0; i < n; ++i) hp[i] = i;
    std::mt19937_64 rng(seed);
    int t = 0;
    for (int ep = 0; ep < epochs && s == CRISP_OK; ++ep) {
        std::shuffle(hp.begin(), hp.end(), rng);
        CRISP_CK(cudaMemcpyAsync(perm, hp.data(), sizeof(long long) * (size_t)n, cudaMemcpyHostToDevice, st));
        double ep_loss = 0.0;
        long long nb = 0;
        for (long long b0 = 0; b0 + B <= n && s == CRISP_OK; b0 += B) {
            k_gather_f<<<g1(B * F, 256), 256, 0, st>>>(X, F, perm + b0, B, Xb);
            k_gather_f<<<g1(B * O, 256), 256, 0, st>>>(T, O, perm + b0, B, Tb);
            s = mlp_loss_grad(params, F, H, O, Xb, Tb, B, G, loss, w, st);
            if (s) break;
            ++t;
            s = crisp_mlp_adam(params, G, mm, vv, np, lr, 0.9f, 0.999f, 1e-8f, t, st);
            if (epoch_loss && s == CRISP_OK) {
                float l = 0.0f;
                CRISP_CK(cudaMemcpyAsync(&l, loss, sizeof(float), cudaMemcpyDeviceToHost, st));
                CRISP_CK(cudaStreamSynchronize(st));
                ep_loss += l;
            }
            ++nb;
        }
        if (epoch_loss) epoch_loss[ep] = nb ? (float)(ep_loss / nb) : 0.0f;
        CRISP_CK(cudaStreamSynchronize(st));   // the host permutation is reused next epoch
    }
    crisp_scratch_free(wb, st);
    crisp_scratch_free(perm, st);
    CRISP_CK(cudaStreamSynchronize(st));
    return s;
}

extern "C" crisp_status crisp_index_set_model(crisp_index *ix, const float *params, int32_t H, void *stream) {
    CRISP_REQUIRE(ix && params, "crisp_index_set_model: null pointer");
    int F = 2 * ix->M + 68;
    crisp_status s = check_mlp(F, H, 2);
    if (s) return s;
    CRISP_REQUIRE(infer_smem(F, H) <= 220 * 1024, "crisp_index_set_model: model too wide");
    long long n = crisp_mlp_param_count(F, H, 2);
    cudaStream_t st = as_stream(stream);
    if (ix->mlp && ix->mlp_H != H) {
        CRISP_CK(cudaStreamSynchronize(st));
        cudaFree(ix->mlp);
        ix->bytes -= sizeof(float) * crisp_mlp_param_count(F, ix->mlp_H, 2);
        ix->mlp = nullptr;
    }
    if (!ix->mlp) {
        CRISP_CK(cudaMalloc((void **)&ix->mlp, sizeof(float) * (size_t)n));
        ix->bytes += sizeof(float) * n;
    }
    CRISP_CK(cudaMemcpyAsync(ix->mlp, params, sizeof(float) * (size_t)n, cudaMemcpyDefault, st));
    CRISP_CK(cudaStreamSynchronize(st));
    ix->mlp_H = H;
    return CRISP_OK;
}
