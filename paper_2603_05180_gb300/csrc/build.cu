// Index-build kernels of the CRISP engine (§4.1, §4.2) for sm_103a.
//
//   B1  k_col_mean / k_syrk_f64      sample covariance in FP64 (mean-centred, 1/(S-1))
//       k_house_* / k_sturm          Householder tridiagonalisation + Sturm bisection (eigenvalues)
//   B2  k_qr_*                       Householder QR of G, explicit Q, sign fix -> R
//       (the product X R runs in the rotation kernel of query.cu)
//       k_eye / k_put_block          block-diagonal R of the block-wise rotation (§7)
//   §7  k_col_var                    per-dimension variance for the adaptive boundaries
//   B3  k_km_assign / k_km_update    batched Lloyd k-means over every subspace half
//       k_assign_cells               u_m(x) = cL*K + cR for all rows
//   B4  k_csr_*                      stable counting sort of ids by cell: Offsets + ids
//   B5  k_sign_codes                 b(x) by warp ballots
#include <float.h>
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.cuh"

namespace {

// ================================================================ B1
__global__ void k_col_mean(const float *__restrict__ X, int D, int ldx, const long long *__restrict__ rows, long long S,
                           double *__restrict__ mu) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    double acc = 0.0;
    for (long long s = 0; s < S; ++s) acc += (double)X[rows[s] * ldx + d];
    mu[d] = acc / (double)S;
}

// var[d] = sum over the sample of (x_d - mu_d)^2 / (S - 1), FP64 (the statistic
// the variance-aware boundaries of §7 balance).
__global__ void k_col_var(const float *__restrict__ X, int D, int ldx, const long long *__restrict__ rows, long long S,
                          const double *__restrict__ mu, double *__restrict__ var) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    const double m = mu[d];
    double acc = 0.0;
    for (long long s = 0; s < S; ++s) {
        const double c = (double)X[rows[s] * ldx + d] - m;
        acc += c * c;
    }
    var[d] = acc / (double)(S - 1);
}

// R = I (D x D, FP32)
__global__ void k_eye(float *__restrict__ R, int D) {
    const long long n = (long long)D * D;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        R[e] = (e / D == e % D) ? 1.0f : 0.0f;
}

// R[lo + i][lo + j] = B[i][j] (FP64 -> FP32) for a w x w block; Bf gets the FP32 block too.
__global__ void k_put_block(const double *__restrict__ B, int w, float *__restrict__ R, int D, int lo,
                            float *__restrict__ Bf) {
    const long long n = (long long)w * w;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float v = (float)B[e];
        Bf[e] = v;
        R[(long long)(lo + e / w) * D + lo + e % w] = v;
    }
}

// cov[i][j] for 64x64 output tiles above the diagonal; 256 threads, 4x4 each.
constexpr int SY_T = 64, SY_K = 16;
__global__ void __launch_bounds__(256) k_syrk_f64(const float *__restrict__ X, int D, int ldx,
                                                  const long long *__restrict__ rows, long long S,
                                                  const double *__restrict__ mu, double *__restrict__ cov) {
    int bi = blockIdx.y, bj = blockIdx.x;
    if (bj < bi) return;
    __shared__ double Ai[SY_K][SY_T], Aj[SY_K][SY_T];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = bi * SY_T, j0 = bj * SY_T;
    double acc[4][4] = {};
    for (long long s0 = 0; s0 < S; s0 += SY_K) {
        for (int e = tid; e < SY_K * SY_T; e += 256) {
            int ss = e / SY_T, c = e % SY_T;
            long long s = s0 + ss;
            double a = 0.0, b = 0.0;
            if (s < S) {
                const float *xr = X + rows[s] * ldx;
                if (i0 + c < D) a = (double)xr[i0 + c] - mu[i0 + c];
                if (j0 + c < D) b = (double)xr[j0 + c] - mu[j0 + c];
            }
            Ai[ss][c] = a;
            Aj[ss][c] = b;
        }
        __syncthreads();
#pragma unroll
        for (int ss = 0; ss < SY_K; ++ss) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = Ai[ss][ty + 16 * u]; b[u] = Aj[ss][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            if (i < D && j < D && j >= i) {
                double c = acc[u][v] / (double)(S - 1);
                cov[(long long)i * D + j] = c;
                cov[(long long)j * D + i] = c;
            }
        }
}

// ---------------------------------------------- Householder tridiagonalisation
// Step k: x = A[k+1:, k]; v = (x - alpha e1)/|x - alpha e1|, alpha = -sign(x0)|x|.
// Writes v (length n' = D-k-1) and the subdiagonal e[k] = alpha; d[k] = A[k][k].
__global__ void k_house_vec(double *__restrict__ A, int D, int k, double *__restrict__ v, double *__restrict__ dd,
                            double *__restrict__ ee) {
    __shared__ double red[32];
    const int n = D - k - 1;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double x = A[(long long)(k + 1 + i) * D + k];
        s += x * x;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    double nrm2 = red[0];
    double x0 = A[(long long)(k + 1) * D + k];
    double nrm = sqrt(nrm2);
    double alpha = x0 > 0 ? -nrm : nrm;
    // |v|^2 = |x|^2 - 2 alpha x0 + alpha^2 = 2 (nrm2 - alpha x0)
    double vn2 = 2.0 * (nrm2 - alpha * x0);
    double inv = vn2 > 0 ? 1.0 / sqrt(vn2) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double x = A[(long long)(k + 1 + i) * D + k];
        v[i] = (i == 0 ? x - alpha : x) * inv;
    }
    if (threadIdx.x == 0) {
        dd[k] = A[(long long)k * D + k];
        ee[k] = vn2 > 0 ? alpha : x0;
    }
}

// p = A22 v (rows of the trailing block), one warp per row.
__global__ void k_house_symv(const double *__restrict__ A, int D, int k, const double *__restrict__ v,
                             double *__restrict__ p) {
    const int n = D - k - 1;
    int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double *a = A + (long long)(k + 1 + row) * D + (k + 1);
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += a[j] * v[j];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) p[row] = s;
}

// w = 2p - 2 (v.p) v
__global__ void k_house_w(int n, const double *__restrict__ v, const double *__restrict__ p, double *__restrict__ w) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * p[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    double c = red[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = 2.0 * p[i] - 2.0 * c * v[i];
}

// A22 -= v w^T + w v^T
__global__ void k_house_rank2(double *__restrict__ A, int D, int k, const double *__restrict__ v,
                              const double *__restrict__ w) {
    const int n = D - k - 1;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    int i = (int)(e / n), j = (int)(e % n);
    A[(long long)(k + 1 + i) * D + (k + 1 + j)] -= v[i] * w[j] + w[i] * v[j];
}

__global__ void k_tail_tridiag(const double *__restrict__ A, int D, double *__restrict__ dd, double *__restrict__ ee) {
    if (threadIdx.x == 0) {
        if (D >= 2) {
            dd[D - 2] = A[(long long)(D - 2) * D + (D - 2)];
            ee[D - 2] = A[(long long)(D - 1) * D + (D - 2)];
        }
        dd[D - 1] = A[(long long)(D - 1) * D + (D - 1)];
    }
}

// Number of eigenvalues of the tridiagonal (d, e) below x (Sturm count).
__device__ int sturm_count(const double *d, const double *e, int n, double x, double pivmin) {
    int c = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0) ++c;
    }
    return c;
}

// eigenvalue number j (ascending) by bisection; written descending to eig[n-1-j]
__global__ void k_sturm(const double *__restrict__ d, const double *__restrict__ e, int n, double lo0, double hi0,
                        double pivmin, double *__restrict__ eig) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double lo = lo0, hi = hi0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(d, e, n, mid, pivmin) > j) hi = mid;
        else lo = mid;
    }
    eig[n - 1 - j] = 0.5 * (lo + hi);
}

// ================================================================ B2
// Householder QR, step k on column k of A (D x D): v over rows k..D-1.
__global__ void k_qr_vec(double *__restrict__ A, int D, int k, double *__restrict__ V, double *__restrict__ alpha_out) {
    __shared__ double red[32];
    const int n = D - k;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double x = A[(long long)(k + i) * D + k];
        s += x * x;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    double nrm2 = red[0], x0 = A[(long long)k * D + k], nrm = sqrt(nrm2);
    double alpha = x0 > 0 ? -nrm : nrm;
    double vn2 = 2.0 * (nrm2 - alpha * x0);
    double inv = vn2 > 0 ? 1.0 / sqrt(vn2) : 0.0;
    double *v = V + (long long)k * D;             // v_k stored in row k of V (entries k..D-1)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double x = A[(long long)(k + i) * D + k];
        v[k + i] = (i == 0 ? x - alpha : x) * inv;
    }
    if (threadIdx.x == 0) alpha_out[k] = vn2 > 0 ? alpha : x0;
}

// wcol[j] = sum_i v[i] * B[i][j] over rows k..D-1, columns c0..D-1
__global__ void k_qr_vtB(const double *__restrict__ B, int D, int k, int c0, const double *__restrict__ v,
                         double *__restrict__ wcol) {
    int j = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    double s = 0.0;
    for (int i = k; i < D; ++i) s += v[i] * B[(long long)i * D + j];
    wcol[j] = s;
}

// B[i][j] -= 2 v[i] wcol[j] for rows k.., columns c0..
__global__ void k_qr_apply(double *__restrict__ B, int D, int k, int c0, const double *__restrict__ v,
                           const double *__restrict__ wcol) {
    int nc = D - c0, nr = D - k;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nr * nc) return;
    int i = k + (int)(e / nc), j = c0 + (int)(e % nc);
    B[(long long)i * D + j] -= 2.0 * v[i] * wcol[j];
}

__global__ void k_eye(double *__restrict__ B, int D) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)D * D) return;
    B[e] = (e / D == e % D) ? 1.0 : 0.0;
}

__global__ void k_sign_cols(double *__restrict__ R, int D, const double *__restrict__ alpha) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)D * D) return;
    int j = (int)(e % D);
    if (alpha[j] < 0) R[e] = -R[e];
}

__global__ void k_d2f(const double *__restrict__ a, float *__restrict__ b, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ================================================================ B3
struct KmJob {
    int off, h;
};

// asg[j][r] = argmin_c SEQ(T[r][off..off+h), C_j[c]) (ties to the lowest index)
__global__ void __launch_bounds__(128) k_km_assign(const float *__restrict__ T, long long S, int ldt,
                                                   const KmJob *__restrict__ jobs, int K, int H,
                                                   const float *__restrict__ C, int *__restrict__ asg) {
    extern __shared__ float Cs[];   // [K][H]
    const int j = blockIdx.y;
    const KmJob jb = jobs[j];
    const float *Cj = C + (long long)j * K * H;
    for (int e = threadIdx.x; e < K * H; e += blockDim.x) Cs[e] = Cj[e];
    __syncthreads();
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S) return;
    const float *x = T + r * ldt + jb.off;
    float acc[CRISP_KMAX];
#pragma unroll
    for (int c = 0; c < CRISP_KMAX; ++c) acc[c] = 0.0f;
    for (int d = 0; d < jb.h; ++d) {
        float xd = x[d];
#pragma unroll
        for (int c = 0; c < CRISP_KMAX; ++c) {
            if (c < K) {
                float diff = xd - Cs[c * H + d];
                acc[c] = fmaf(diff, diff, acc[c]);
            }
        }
    }
    int best = 0;
    float bd = acc[0];
#pragma unroll
    for (int c = 1; c < CRISP_KMAX; ++c)
        if (c < K && acc[c] < bd) { bd = acc[c]; best = c; }
    asg[(long long)j * S + r] = best;
}

// New centroid c of job j: FP64 mean of its members (fixed order), else unchanged.
__global__ void __launch_bounds__(256) k_km_update(const float *__restrict__ T, long long S, int ldt,
                                                   const KmJob *__restrict__ jobs, int K, int H,
                                                   const int *__restrict__ asg, float *__restrict__ C) {
    __shared__ double part[8][128];
    __shared__ long long cnt[8];
    const int c = blockIdx.x, j = blockIdx.y;
    const KmJob jb = jobs[j];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc[4] = {0, 0, 0, 0};
    long long n = 0;
    const int *a = asg + (long long)j * S;
    for (long long r0 = (long long)warp * 32; r0 < S; r0 += 8 * 32) {
        long long r = r0 + lane;
        bool hit = r < S && a[r] == c;
        unsigned bal = __ballot_sync(0xffffffffu, hit);
        while (bal) {
            int b = __ffs(bal) - 1;
            bal &= bal - 1;
            const float *x = T + (r0 + b) * ldt + jb.off;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int d = lane + 32 * u;
                if (d < jb.h) acc[u] += (double)x[d];
            }
            ++n;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) part[warp][lane + 32 * u] = acc[u];
    if (lane == 0) cnt[warp] = n;
    __syncthreads();
    if (warp == 0) {
        long long tot = 0;
        for (int w = 0; w < 8; ++w) tot += cnt[w];
        if (tot > 0) {
            for (int u = 0; u < 4; ++u) {
                int d = lane + 32 * u;
                if (d < jb.h) {
                    double s = 0.0;
                    for (int w = 0; w < 8; ++w) s += part[w][d];
                    C[((long long)j * K + c) * H + d] = (float)(s / (double)tot);
                }
            }
        }
    }
}

__global__ void k_km_init(const float *__restrict__ T, int ldt, const KmJob *__restrict__ jobs, int K, int H,
                          const int *__restrict__ init, float *__restrict__ C) {
    const int j = blockIdx.y, c = blockIdx.x;
    const KmJob jb = jobs[j];
    const float *x = T + (long long)init[(long long)j * K + c] * ldt + jb.off;
    for (int d = threadIdx.x; d < H; d += blockDim.x) C[((long long)j * K + c) * H + d] = d < jb.h ? x[d] : 0.0f;
}

__global__ void k_gather_rows(const float *__restrict__ X, int ld, const long long *__restrict__ rows, long long S,
                              float *__restrict__ T) {
    long long tot = S * (long long)ld;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        long long r = e / ld;
        int d = (int)(e % ld);
        T[e] = X[rows[r] * ld + d];
    }
}

// cells[m][n] for every row n (blockIdx.x) and subspace m (blockIdx.y)
__global__ void __launch_bounds__(128) k_assign_cells(const float *__restrict__ Xr, long long N, int Dp, int K, int H,
                                                      const int32_t *__restrict__ sub,
                                                      const float *__restrict__ cent,
                                                      uint16_t *__restrict__ cells) {
    extern __shared__ float Cs[];   // [2][K][H]
    const int m = blockIdx.y;
    const float *cm = cent + (long long)m * 2 * K * H;
    for (int e = threadIdx.x; e < 2 * K * H; e += blockDim.x) Cs[e] = cm[e];
    __syncthreads();
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int a = sub[m], b = sub[m + 1];
    int hl = (b - a) / 2, hr = (b - a) - hl;
    int arg[2];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const float *x = Xr + n * Dp + a + (half ? hl : 0);
        const float *C = Cs + half * K * H;
        int h = half ? hr : hl;
        float acc[CRISP_KMAX];
#pragma unroll
        for (int c = 0; c < CRISP_KMAX; ++c) acc[c] = 0.0f;
        for (int d = 0; d < h; ++d) {
            float xd = x[d];
#pragma unroll
            for (int c = 0; c < CRISP_KMAX; ++c) {
                if (c < K) {
                    float diff = xd - C[c * H + d];
                    acc[c] = fmaf(diff, diff, acc[c]);
                }
            }
        }
        int best = 0;
        float bd = acc[0];
#pragma unroll
        for (int c = 1; c < CRISP_KMAX; ++c)
            if (c < K && acc[c] < bd) { bd = acc[c]; best = c; }
        arg[half] = best;
    }
    cells[(long long)m * N + n] = (uint16_t)(arg[0] * K + arg[1]);
}

// ================================================================ B4
constexpr int CSR_CH = 4096;   // ids per chunk (12-bit local index)
constexpr int CSR_NT = 1024;

__global__ void k_csr_count(const uint16_t *__restrict__ cells, long long N, int K2, int *__restrict__ counts) {
    extern __shared__ int hist[];
    const long long c0 = (long long)blockIdx.x * CSR_CH;
    for (int i = threadIdx.x; i < K2; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < CSR_CH; i += blockDim.x) {
        long long n = c0 + i;
        if (n < N) atomicAdd(&hist[cells[n]], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K2; i += blockDim.x) counts[(long long)blockIdx.x * K2 + i] = hist[i];
}

// per cell: total over chunks, then base[chunk][cell] = exclusive prefix over chunks
__global__ void k_csr_colscan(int *__restrict__ counts, int nch, int K2, int *__restrict__ totals) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K2) return;
    int acc = 0;
    for (int b = 0; b < nch; ++b) {
        int v = counts[(long long)b * K2 + c];
        counts[(long long)b * K2 + c] = acc;
        acc += v;
    }
    totals[c] = acc;
}

__global__ void k_csr_offsets(const int *__restrict__ totals, int K2, int *__restrict__ offsets) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < K2; ++c) { offsets[c] = acc; acc += totals[c]; }
        offsets[K2] = acc;
    }
}

// sort the chunk's (cell, local) keys, then each id goes to
// offsets[cell] + base[chunk][cell] + (its rank inside the cell within the chunk)
__global__ void __launch_bounds__(CSR_NT) k_csr_scatter(const uint16_t *__restrict__ cells, long long N, int K2,
                                                        const int *__restrict__ base, const int *__restrict__ offsets,
                                                        int *__restrict__ ids) {
    __shared__ unsigned keys[CSR_CH];
    const long long c0 = (long long)blockIdx.x * CSR_CH;
    for (int i = threadIdx.x; i < CSR_CH; i += CSR_NT) {
        long long n = c0 + i;
        keys[i] = n < N ? ((unsigned)cells[n] << 12) | (unsigned)i : 0xFFFFFFFFu;
    }
    __syncthreads();
    for (int size = 2; size <= CSR_CH; size <<= 1) {
        for (int sd = size >> 1; sd > 0; sd >>= 1) {
            for (int i = threadIdx.x; i < CSR_CH; i += CSR_NT) {
                int j = i ^ sd;
                if (j > i) {
                    unsigned a = keys[i], b = keys[j];
                    bool up = (i & size) == 0;
                    if ((a > b) == up) { keys[i] = b; keys[j] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int p = threadIdx.x; p < CSR_CH; p += CSR_NT) {
        unsigned key = keys[p];
        if (key == 0xFFFFFFFFu) continue;
        int cell = (int)(key >> 12), local = (int)(key & 0xFFFu);
        // first position of this cell in the sorted chunk
        int lo = 0, hi = p;
        unsigned tgt = (unsigned)cell << 12;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (keys[mid] < tgt) lo = mid + 1;
            else hi = mid;
        }
        ids[(long long)offsets[cell] + base[(long long)blockIdx.x * K2 + cell] + (p - lo)] = (int)(c0 + local);
    }
}

// ================================================================ B5
__global__ void k_sign_codes(const float *__restrict__ Xr, long long N, int Dp, uint32_t *__restrict__ codes) {
    const int W = Dp / 32;
    long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    long long tot = N * W;
    for (; wid < tot; wid += ((long long)gridDim.x * blockDim.x) >> 5) {
        long long n = wid / W;
        int w = (int)(wid % W);
        unsigned b = __ballot_sync(0xffffffffu, Xr[n * Dp + 32 * w + lane] > 0.0f);
        if (lane == 0) codes[n * W + w] = b;
    }
}

// ================================================================ F2
__global__ void k_quant_bf16(const float *__restrict__ X, long long n, uint16_t *__restrict__ Xb) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Xb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(X[i]));
}

// one warp per row: scale = max|x| / 448 (1 for a zero row), codes of x / scale
__global__ void k_quant_e4m3(const float *__restrict__ Xr, long long N, int Dp, uint8_t *__restrict__ X8,
                             float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    for (long long n = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; n < N;
         n += ((long long)gridDim.x * blockDim.x) >> 5) {
        const float *x = Xr + n * Dp;
        float mx = 0.0f;
        for (int d = lane; d < Dp; d += 32) mx = fmaxf(mx, fabsf(x[d]));
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float s = mx > 0.0f ? mx / 448.0f : 1.0f;
        for (int d = lane; d < Dp; d += 32)
            X8[n * Dp + d] = (uint8_t)__nv_cvt_float_to_fp8(x[d] / s, __NV_SATFINITE, __NV_E4M3);
        if (lane == 0) scale[n] = s;
    }
}

unsigned grid1(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

}  // namespace

// ==================================================================== C ABI
extern "C" crisp_status crisp_covariance(const float *X, int64_t N, int32_t D, int32_t ldx, const int64_t *rows,
                                         int64_t S, double *cov, void *stream) {
    CRISP_REQUIRE(X && rows && cov, "crisp_covariance: null pointer");
    CRISP_REQUIRE(S >= 2 && D >= 1 && ldx >= D && N >= 1, "crisp_covariance: need S >= 2, D >= 1, ldx >= D");
    cudaStream_t st = as_stream(stream);
    double *mu = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&mu, sizeof(double) * D, st));
    k_col_mean<<<grid1(D, 128), 128, 0, st>>>(X, D, ldx, (const long long *)rows, S, mu);
    dim3 g((D + SY_T - 1) / SY_T, (D + SY_T - 1) / SY_T);
    k_syrk_f64<<<g, 256, 0, st>>>(X, D, ldx, (const long long *)rows, S, mu, cov);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(mu, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "covariance kernels", __FILE__, __LINE__);
    return CRISP_OK;
}

extern "C" crisp_status crisp_column_variance(const float *X, int64_t N, int32_t D, int32_t ldx, const int64_t *rows,
                                              int64_t S, double *var, void *stream) {
    CRISP_REQUIRE(X && rows && var, "crisp_column_variance: null pointer");
    CRISP_REQUIRE(S >= 2 && D >= 1 && ldx >= D && N >= 1, "crisp_column_variance: need S >= 2, D >= 1, ldx >= D");
    cudaStream_t st = as_stream(stream);
    double *mu = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&mu, sizeof(double) * D, st));
    k_col_mean<<<grid1(D, 128), 128, 0, st>>>(X, D, ldx, (const long long *)rows, S, mu);
    CRISP_COUNT_LAUNCH();
    k_col_var<<<grid1(D, 128), 128, 0, st>>>(X, D, ldx, (const long long *)rows, S, mu, var);
    CRISP_COUNT_LAUNCH();
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(mu, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "variance kernels", __FILE__, __LINE__);
    return CRISP_OK;
}

extern "C" crisp_status crisp_eigvalsh(double *A, int32_t D, double *eig, void *stream) {
    CRISP_REQUIRE(A && eig && D >= 1, "crisp_eigvalsh: bad arguments");
    cudaStream_t st = as_stream(stream);
    double *ws = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&ws, sizeof(double) * 5 * (size_t)(D + 1), st));
    double *v = ws, *p = ws + D + 1, *w = ws + 2 * (D + 1), *dd = ws + 3 * (D + 1), *ee = ws + 4 * (D + 1);
    for (int k = 0; k + 2 < D; ++k) {
        int n = D - k - 1;
        k_house_vec<<<1, 1024, 0, st>>>(A, D, k, v, dd, ee);
        k_house_symv<<<grid1(n, 8), 256, 0, st>>>(A, D, k, v, p);
        k_house_w<<<1, 1024, 0, st>>>(n, v, p, w);
        k_house_rank2<<<grid1((long long)n * n, 256), 256, 0, st>>>(A, D, k, v, w);
    }
    k_tail_tridiag<<<1, 32, 0, st>>>(A, D, dd, ee);
    CRISP_CK_LAUNCH();
    // Gershgorin bounds on the host
    std::vector<double> hd(D), he(D > 1 ? D - 1 : 1);
    CRISP_CK(cudaMemcpyAsync(hd.data(), dd, sizeof(double) * D, cudaMemcpyDeviceToHost, st));
    if (D > 1) CRISP_CK(cudaMemcpyAsync(he.data(), ee, sizeof(double) * (D - 1), cudaMemcpyDeviceToHost, st));
    CRISP_CK(cudaStreamSynchronize(st));
    double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
    for (int i = 0; i < D; ++i) {
        double r = (i > 0 ? fabs(he[i - 1]) : 0.0) + (i + 1 < D ? fabs(he[i]) : 0.0);
        lo = std::min(lo, hd[i] - r);
        hi = std::max(hi, hd[i] + r);
        emax = std::max(emax, fabs(hd[i]) + r);
    }
    double span = std::max(emax, 1e-300);
    lo -= 1e-12 * span;
    hi += 1e-12 * span;
    double pivmin = DBL_MIN * std::max(1.0, span * span);
    k_sturm<<<grid1(D, 128), 128, 0, st>>>(dd, ee, D, lo, hi, pivmin, eig);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "eigenvalue kernels", __FILE__, __LINE__);
    return CRISP_OK;
}

extern "C" crisp_status crisp_cev(const float *X, int64_t N, int32_t D, int32_t ldx, const int64_t *rows, int64_t S,
                                  double *cev, void *stream) {
    CRISP_REQUIRE(cev, "crisp_cev: null output");
    cudaStream_t st = as_stream(stream);
    double *buf = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&buf, sizeof(double) * ((size_t)D * D + D), st));
    crisp_status s = crisp_covariance(X, N, D, ldx, rows, S, buf, stream);
    if (!s) s = crisp_eigvalsh(buf, D, buf + (size_t)D * D, stream);
    std::vector<double> ev(D);
    if (!s) {
        cudaError_t e = cudaMemcpyAsync(ev.data(), buf + (size_t)D * D, sizeof(double) * D, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = crisp_cuda_fail(e, "crisp_cev readback", __FILE__, __LINE__);
    }
    cudaFreeAsync(buf, st);
    if (s) return s;
    // CEV = top floor(0.2 D) eigenvalues over all (§4.1); eigenvalues descending
    int kt = (int)floor(0.2 * D);
    double top = 0.0, tot = 0.0;
    for (int i = 0; i < D; ++i) {
        tot += ev[i];
        if (i < kt) top += ev[i];
    }
    *cev = tot > 0 ? top / tot : 0.0;
    return CRISP_OK;
}

extern "C" crisp_status crisp_rotation_from_gaussian(const double *G, int32_t D, double *R, void *stream) {
    CRISP_REQUIRE(G && R && D >= 1, "crisp_rotation_from_gaussian: bad arguments");
    cudaStream_t st = as_stream(stream);
    double *A = nullptr;
    size_t nD = (size_t)D * D;
    CRISP_CK(cudaMallocAsync((void **)&A, sizeof(double) * (2 * nD + 2 * (size_t)D), st));
    double *V = A + nD, *alpha = V + nD, *wcol = alpha + D;
    CRISP_CK(cudaMemcpyAsync(A, G, sizeof(double) * nD, cudaMemcpyDeviceToDevice, st));
    CRISP_CK(cudaMemsetAsync(V, 0, sizeof(double) * nD, st));
    for (int k = 0; k < D; ++k) {
        k_qr_vec<<<1, 1024, 0, st>>>(A, D, k, V, alpha);
        if (k + 1 < D) {
            const double *v = V + (size_t)k * D;
            k_qr_vtB<<<grid1(D - k - 1, 128), 128, 0, st>>>(A, D, k, k + 1, v, wcol);
            k_qr_apply<<<grid1((long long)(D - k) * (D - k - 1), 256), 256, 0, st>>>(A, D, k, k + 1, v, wcol);
        }
    }
    // Q = H_0 H_1 ... H_{D-1}: accumulate backwards on the identity
    k_eye<<<grid1((long long)nD, 256), 256, 0, st>>>(R, D);
    for (int k = D - 1; k >= 0; --k) {
        const double *v = V + (size_t)k * D;
        k_qr_vtB<<<grid1(D - k, 128), 128, 0, st>>>(R, D, k, k, v, wcol);
        k_qr_apply<<<grid1((long long)(D - k) * (D - k), 256), 256, 0, st>>>(R, D, k, k, v, wcol);
    }
    k_sign_cols<<<grid1((long long)nD, 256), 256, 0, st>>>(R, D, alpha);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(A, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "QR kernels", __FILE__, __LINE__);
    return CRISP_OK;
}

// tc_D > 0: the jobs are the 2M subspace halves (boundaries tc_sub, host) of a
// D-dim index in order and T has the index's row pitch, so the assignment step
// runs on the tensor cores (same assignments as k_km_assign, see
// crisp_assign_cells_tc).
static crisp_status kmeans_batched(const float *T, int64_t S, int32_t ldt, const std::vector<KmJob> &jobs, int32_t K,
                                   int32_t H, const int32_t *init_dev, int32_t iters, float *C, cudaStream_t st,
                                   int32_t tc_D = 0, const int32_t *tc_sub = nullptr) {
    int nj = (int)jobs.size();
    KmJob *djobs = nullptr;
    int *asg = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&djobs, sizeof(KmJob) * nj, st));
    CRISP_CK(cudaMallocAsync((void **)&asg, sizeof(int) * (size_t)nj * S, st));
    CRISP_CK(cudaMemcpyAsync(djobs, jobs.data(), sizeof(KmJob) * nj, cudaMemcpyHostToDevice, st));
    k_km_init<<<dim3(K, nj), 128, 0, st>>>(T, ldt, djobs, K, H, init_dev, C);
    size_t smem = sizeof(float) * (size_t)K * H;
    CRISP_CK(cudaFuncSetAttribute(k_km_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int it = 0; it < iters; ++it) {
        if (tc_D > 0) {
            crisp_status s = crisp_tc_assign(T, S, tc_D, ldt, nj / 2, K, H, tc_sub, C, nullptr, asg, st);
            if (s) {
                cudaFreeAsync(asg, st);
                cudaFreeAsync(djobs, st);
                return s;
            }
        } else {
            k_km_assign<<<dim3(grid1(S, 128), nj), 128, smem, st>>>(T, S, ldt, djobs, K, H, C, asg);
        }
        k_km_update<<<dim3(K, nj), 256, 0, st>>>(T, S, ldt, djobs, K, H, asg, C);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(asg, st);
    cudaFreeAsync(djobs, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "k-means kernels", __FILE__, __LINE__);
    // the host vector `jobs` was copied asynchronously: keep it alive until done
    CRISP_CK(cudaStreamSynchronize(st));
    return CRISP_OK;
}

extern "C" crisp_status crisp_kmeans(const float *T, int64_t S, int32_t ldt, int32_t off, int32_t h, int32_t K,
                                     int32_t H, const int32_t *init, int32_t iters, float *C, void *stream) {
    CRISP_REQUIRE(T && init && C, "crisp_kmeans: null pointer");
    CRISP_REQUIRE(K >= 2 && K <= CRISP_KMAX && h >= 1 && h <= H && H <= 128 && off >= 0 && off + h <= ldt && S >= K &&
                      iters >= 0,
                  "crisp_kmeans: bad sizes (K in [2, 64], 1 <= h <= H <= 128, S >= K)");
    std::vector<KmJob> jobs{{off, h}};
    return kmeans_batched(T, S, ldt, jobs, K, H, init, iters, C, as_stream(stream));
}

// Host boundaries [M+1] (NULL: the equal split), checked and copied.
static crisp_status host_bounds(const int32_t *sub, int32_t D, int32_t M, int32_t H, const char *who,
                                std::vector<int32_t> &out) {
    if (sub) out.assign(sub, sub + M + 1);
    else out = crisp_equal_bounds(D, M);
    if (sub && !crisp_bounds_valid(out.data(), D, M, who)) return CRISP_EINVAL;
    if (crisp_bounds_half_max(out.data(), M) > H) {
        crisp_set_error("%s: a subspace half is wider than H = %d", who, H);
        return CRISP_EINVAL;
    }
    return CRISP_OK;
}

extern "C" crisp_status crisp_assign_cells(const float *Xr, int64_t N, int32_t D, int32_t Dp, int32_t M, int32_t K,
                                           int32_t H, const int32_t *sub, const float *cent, uint16_t *cells,
                                           void *stream) {
    CRISP_REQUIRE(Xr && cent && cells, "crisp_assign_cells: null pointer");
    CRISP_REQUIRE(K >= 2 && K <= CRISP_KMAX && M >= 1 && 2 * M <= D && Dp >= D && N >= 1 && H <= 128,
                  "crisp_assign_cells: bad sizes");
    std::vector<int32_t> hb;
    crisp_status s = host_bounds(sub, D, M, H, "crisp_assign_cells", hb);
    if (s) return s;
    cudaStream_t st = as_stream(stream);
    int32_t *db = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&db, sizeof(int32_t) * hb.size(), st));
    cudaError_t e = cudaMemcpyAsync(db, hb.data(), sizeof(int32_t) * hb.size(), cudaMemcpyHostToDevice, st);
    size_t smem = sizeof(float) * 2 * (size_t)K * H;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_assign_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_assign_cells<<<dim3(grid1(N, 128), M), 128, smem, st>>>(Xr, N, Dp, K, H, db, cent, cells);
        CRISP_COUNT_LAUNCH();
        e = cudaGetLastError();
    }
    cudaFreeAsync(db, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "k_assign_cells", __FILE__, __LINE__);
    return CRISP_OK;
}

extern "C" crisp_status crisp_csr_build(const uint16_t *cells, int64_t N, int32_t K2, int32_t *offsets, int32_t *ids,
                                        void *stream) {
    CRISP_REQUIRE(cells && offsets && ids, "crisp_csr_build: null pointer");
    CRISP_REQUIRE(K2 >= 1 && K2 <= 4096 && N >= 1 && N < (1LL << 31), "crisp_csr_build: K2 > 4096 or bad N");
    cudaStream_t st = as_stream(stream);
    int nch = (int)((N + CSR_CH - 1) / CSR_CH);
    int *counts = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&counts, sizeof(int) * ((size_t)nch * K2 + K2), st));
    int *totals = counts + (size_t)nch * K2;
    k_csr_count<<<nch, 256, sizeof(int) * K2, st>>>(cells, N, K2, counts);
    k_csr_colscan<<<grid1(K2, 256), 256, 0, st>>>(counts, nch, K2, totals);
    k_csr_offsets<<<1, 32, 0, st>>>(totals, K2, offsets);
    k_csr_scatter<<<nch, CSR_NT, 0, st>>>(cells, N, K2, counts, offsets, ids);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(counts, st);
    if (e != cudaSuccess) return crisp_cuda_fail(e, "CSR kernels", __FILE__, __LINE__);
    return CRISP_OK;
}

extern "C" crisp_status crisp_sign_codes(const float *Xr, int64_t N, int32_t Dp, uint32_t *codes, void *stream) {
    CRISP_REQUIRE(Xr && codes && N >= 1 && Dp >= 32 && Dp % 32 == 0, "crisp_sign_codes: bad arguments");
    long long warps = (long long)N * (Dp / 32);
    long long blocks = std::min<long long>((warps * 32 + 255) / 256, 152LL * 64);
    k_sign_codes<<<(unsigned)blocks, 256, 0, as_stream(stream)>>>(Xr, N, Dp, codes);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

// ============================================================== crisp_build
crisp_status crisp_alloc_index(crisp_index *ix);
crisp_status crisp_finish_index(crisp_index *ix, cudaStream_t st);
crisp_status crisp_make_copies(crisp_index *ix, uint32_t copies, cudaStream_t st);

static std::vector<int64_t> sample_rows(int64_t N, int64_t S, std::mt19937_64 &rng) {
    // Floyd's algorithm: S distinct rows of 0..N-1, returned sorted
    std::vector<int64_t> out;
    out.reserve(S);
    std::vector<char> seen;
    bool dense = N <= (int64_t)64 << 20;
    if (dense) seen.assign((size_t)N, 0);
    std::vector<int64_t> set;
    for (int64_t j = N - S; j < N; ++j) {
        int64_t t = std::uniform_int_distribution<int64_t>(0, j)(rng);
        bool has;
        if (dense) has = seen[t];
        else has = std::find(set.begin(), set.end(), t) != set.end();
        int64_t pick = has ? j : t;
        if (dense) seen[pick] = 1;
        else set.push_back(pick);
        out.push_back(pick);
    }
    std::sort(out.begin(), out.end());
    return out;
}

extern "C" crisp_status crisp_build(const float *X, int64_t N, int32_t D, const crisp_build_params *p, void *stream,
                                    crisp_index **out) {
    CRISP_REQUIRE(X && p && out, "crisp_build: null pointer");
    CRISP_REQUIRE(N >= 2 && N < (1LL << 31) && D >= 2, "crisp_build: need 2 <= N < 2^31, D >= 2");
    CRISP_REQUIRE(p->M >= 1 && 2 * p->M <= D, "crisp_build: M outside [1, D/2]");
    CRISP_REQUIRE(p->K >= 2 && p->K <= CRISP_KMAX && p->K <= N, "crisp_build: K outside [2, min(64, N)]");
    CRISP_REQUIRE(p->rotate >= -1 && p->rotate <= 1, "crisp_build: rotate must be -1, 0 or 1");
    CRISP_REQUIRE(p->kmeans_iters >= 0, "crisp_build: kmeans_iters < 0");
    CRISP_REQUIRE((p->copies & ~3u) == 0, "crisp_build: copies must be a mask of 1 (BF16) and 2 (FP8)");
    CRISP_REQUIRE(p->adaptive == 0 || p->adaptive == 1, "crisp_build: adaptive must be 0 or 1");
    CRISP_REQUIRE(p->block_dims >= 0 && p->block_dims % 4 == 0, "crisp_build: block_dims must be a multiple of 4");
    cudaStream_t st = as_stream(stream);
    const int32_t M = p->M, K = p->K;
    if (p->adaptive && D > 256 * (int64_t)M) {
        crisp_set_error("crisp_build: variance-aware boundaries need D <= 256 M");
        return CRISP_EUNSUPPORTED;
    }
    crisp_index *ix = new crisp_index();
    ix->N = N; ix->D = D; ix->Dp = (D + 31) / 32 * 32; ix->M = M; ix->K = K;
    ix->block_dims = p->block_dims;
    ix->sub_h = crisp_equal_bounds(D, M);
    if (!p->adaptive && crisp_bounds_half_max(ix->sub_h.data(), M) > 128) {
        delete ix;
        crisp_set_error("crisp_build: subspace halves wider than 128 dims (raise M)");
        return CRISP_EUNSUPPORTED;
    }
    cudaGetDevice(&ix->device);
    std::mt19937_64 rng(p->seed);
    std::vector<int64_t> cs;
    if (p->cev_sample) cs.assign(p->cev_sample, p->cev_sample + p->cev_sample_n);
    else cs = sample_rows(N, std::min<int64_t>(N, std::max<int64_t>(2, std::min<int64_t>(N / 10, 100000))), rng);
    for (int64_t r : cs)
        if (r < 0 || r >= N || cs.size() < 2) {
            delete ix;
            crisp_set_error("crisp_build: covariance sample needs >= 2 rows in [0, N)");
            return CRISP_EINVAL;
        }
    crisp_status s = CRISP_OK;
    void *tmp = nullptr;
#define BSTEP(x)                     \
    do {                             \
        if (s == CRISP_OK) s = (x);  \
    } while (0)
#define BCUDA(x)                                                                \
    do {                                                                        \
        if (s == CRISP_OK) {                                                    \
            cudaError_t e_ = (x);                                               \
            if (e_ != cudaSuccess) s = crisp_cuda_fail(e_, #x, __FILE__, __LINE__); \
        }                                                                       \
    } while (0)
    // ---- B1: CEV on the covariance sample (and, block-wise, per block)
    int64_t *drows = nullptr;
    BCUDA(cudaMallocAsync((void **)&drows, sizeof(int64_t) * cs.size(), st));
    BCUDA(cudaMemcpyAsync(drows, cs.data(), sizeof(int64_t) * cs.size(), cudaMemcpyHostToDevice, st));
    double cev = 0.0;
    BSTEP(crisp_cev(X, N, D, D, drows, (int64_t)cs.size(), &cev, st));
    ix->cev = cev;
    std::vector<std::pair<int32_t, int32_t>> rot_blocks;   // [lo, hi) of the blocks to rotate
    if (p->block_dims > 0) {
        // §7 block-wise redistribution: each block of block_dims dims takes the
        // §4.1 test on its own covariance (the block of the sample covariance)
        for (int32_t lo = 0; lo < D && s == CRISP_OK; lo += p->block_dims) {
            const int32_t hi = std::min(D, lo + p->block_dims);
            double cb = 0.0;
            BSTEP(crisp_cev(X + lo, N, hi - lo, D, drows, (int64_t)cs.size(), &cb, st));
            if (p->rotate == 1 || (p->rotate == -1 && cb > p->tau_cev)) rot_blocks.push_back({lo, hi});
        }
        ix->rotated = !rot_blocks.empty();
        ix->rotated_blocks = (int32_t)rot_blocks.size();
    } else {
        ix->rotated = (p->rotate == 1) || (p->rotate == -1 && cev > p->tau_cev);
    }
    const int32_t H_eq = crisp_bounds_half_max(ix->sub_h.data(), M);
    ix->H = p->adaptive ? 0 : H_eq;   // centroids are allocated once H is known
    BSTEP(crisp_alloc_index(ix));
    // ---- B2: rotation (R from the QR of G), X' = X R; else zero-padded copy
    std::vector<double> G;
    const double *Gh = p->gaussian;
    if (s == CRISP_OK && ix->rotated && !Gh) {
        G.resize((size_t)D * D);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (auto &g : G) g = nd(rng);
        Gh = G.data();
    }
    // TMA reads of X need 16-byte aligned rows: other shapes go through a zero-padded copy
    const bool x_aligned = ((uintptr_t)X % 16) == 0 && D % 4 == 0;
    if (s == CRISP_OK && ix->rotated && p->block_dims == 0) {
        double *dG = nullptr;
        BCUDA(cudaMallocAsync((void **)&dG, sizeof(double) * 2 * (size_t)D * D, st));
        BCUDA(cudaMemcpyAsync(dG, Gh, sizeof(double) * (size_t)D * D, cudaMemcpyHostToDevice, st));
        BSTEP(crisp_rotation_from_gaussian(dG, D, dG + (size_t)D * D, st));
        if (s == CRISP_OK) {
            k_d2f<<<grid1((long long)D * D, 256), 256, 0, st>>>(dG + (size_t)D * D, ix->R32, (long long)D * D);
            BCUDA(cudaGetLastError());
        }
        BCUDA(cudaStreamSynchronize(st));   // G (host) must outlive its copy
        if (dG) cudaFreeAsync(dG, st);
        // X' = X R on the tensor cores
        if (x_aligned) {
            BSTEP(crisp_rotate_rows_tc(X, N, D, D, ix->R32, ix->Xr, ix->Dp, st));
        } else if (s == CRISP_OK) {
            float *Xp = nullptr;
            BCUDA(cudaMallocAsync((void **)&Xp, sizeof(float) * (size_t)N * ix->Dp, st));
            BSTEP(launch_pad_rows(X, N, D, D, Xp, ix->Dp, st));
            BSTEP(crisp_rotate_rows_tc(Xp, N, D, ix->Dp, ix->R32, ix->Xr, ix->Dp, st));
            if (Xp) cudaFreeAsync(Xp, st);
        }
    } else if (s == CRISP_OK && ix->rotated) {
        // block-diagonal R: identity, then each rotated block's own rotation from
        // its diagonal block of G; the stored rows are the padded copy with each
        // rotated block's columns replaced by x_B R_B (O(N sum w^2) on the tensor cores)
        k_eye<<<(unsigned)std::min<long long>(grid1((long long)D * D, 256), 152LL * 32), 256, 0, st>>>(ix->R32, D);
        BCUDA(cudaGetLastError());
        BSTEP(launch_pad_rows(X, N, D, D, ix->Xr, ix->Dp, st));
        const float *src = X;
        int32_t lds = D;
        float *Xp = nullptr;
        if (!x_aligned && s == CRISP_OK) {
            BCUDA(cudaMallocAsync((void **)&Xp, sizeof(float) * (size_t)N * ix->Dp, st));
            BSTEP(launch_pad_rows(X, N, D, D, Xp, ix->Dp, st));
            src = Xp;
            lds = ix->Dp;
        }
        int32_t wmax = 0;
        for (auto &bk : rot_blocks) wmax = std::max(wmax, bk.second - bk.first);
        double *dG = nullptr;
        float *Bf = nullptr;
        BCUDA(cudaMallocAsync((void **)&dG, sizeof(double) * 2 * (size_t)wmax * wmax, st));
        BCUDA(cudaMallocAsync((void **)&Bf, sizeof(float) * (size_t)wmax * wmax, st));
        std::vector<double> Gb((size_t)wmax * wmax);
        for (auto &bk : rot_blocks) {
            if (s != CRISP_OK) break;
            const int32_t lo = bk.first, w = bk.second - bk.first;
            for (int32_t i = 0; i < w; ++i)
                for (int32_t j = 0; j < w; ++j) Gb[(size_t)i * w + j] = Gh[(size_t)(lo + i) * D + lo + j];
            BCUDA(cudaMemcpyAsync(dG, Gb.data(), sizeof(double) * (size_t)w * w, cudaMemcpyHostToDevice, st));
            BSTEP(crisp_rotation_from_gaussian(dG, w, dG + (size_t)w * w, st));
            if (s == CRISP_OK) {
                k_put_block<<<(unsigned)std::min<long long>(grid1((long long)w * w, 256), 152LL * 32), 256, 0, st>>>(
                    dG + (size_t)w * w, w, ix->R32, D, lo, Bf);
                BCUDA(cudaGetLastError());
            }
            BSTEP(crisp_rotate_rows_tc_cols(src + lo, N, w, lds, Bf, ix->Xr + lo, ix->Dp, w, st));
            BCUDA(cudaStreamSynchronize(st));   // Gb and Bf are reused by the next block
        }
        if (dG) cudaFreeAsync(dG, st);
        if (Bf) cudaFreeAsync(Bf, st);
        if (Xp) cudaFreeAsync(Xp, st);
    } else if (s == CRISP_OK) {
        BSTEP(launch_pad_rows(X, N, D, D, ix->Xr, ix->Dp, st));
    }
    // ---- §7 variance-aware subspace boundaries from the stored rows' variances
    if (s == CRISP_OK && p->adaptive) {
        double *dvar = nullptr;
        std::vector<double> var(D);
        BCUDA(cudaMallocAsync((void **)&dvar, sizeof(double) * D, st));
        BSTEP(crisp_column_variance(ix->Xr, N, D, ix->Dp, drows, (int64_t)cs.size(), dvar, st));
        BCUDA(cudaMemcpyAsync(var.data(), dvar, sizeof(double) * D, cudaMemcpyDeviceToHost, st));
        BCUDA(cudaStreamSynchronize(st));
        if (dvar) cudaFreeAsync(dvar, st);
        BSTEP(crisp_adaptive_bounds(var.data(), D, M, ix->sub_h.data()));
        if (s == CRISP_OK) {
            ix->H = crisp_bounds_half_max(ix->sub_h.data(), M);
            const size_t cb = sizeof(float) * (size_t)M * 2 * K * ix->H;
            BCUDA(cudaMalloc((void **)&ix->cent, cb));
            if (s == CRISP_OK) ix->bytes += (int64_t)cb;
        }
    }
    if (drows) cudaFreeAsync(drows, st);
    const int32_t H = ix->H;
    const int32_t *sub = ix->sub_h.data();
    // ---- B3: k-means per subspace half on the training sample, then cells
    std::vector<int64_t> ks;
    if (p->kmeans_sample) ks.assign(p->kmeans_sample, p->kmeans_sample + p->kmeans_sample_n);
    else ks = sample_rows(N, std::min<int64_t>(N, p->kmeans_train > 0 ? p->kmeans_train : 100000), rng);
    int64_t TS = (int64_t)ks.size();
    if (s == CRISP_OK && TS < K) { crisp_set_error("crisp_build: k-means sample smaller than K"); s = CRISP_EINVAL; }
    std::vector<int32_t> init((size_t)M * 2 * K);
    if (p->kmeans_init) std::copy(p->kmeans_init, p->kmeans_init + init.size(), init.begin());
    else if (s == CRISP_OK)
        for (int32_t j = 0; j < 2 * M; ++j) {
            std::vector<int64_t> pick = sample_rows(TS, K, rng);
            std::shuffle(pick.begin(), pick.end(), rng);
            for (int32_t c = 0; c < K; ++c) init[(size_t)j * K + c] = (int32_t)pick[c];
        }
    for (int32_t v : init)
        if (s == CRISP_OK && (v < 0 || v >= TS)) { crisp_set_error("crisp_build: k-means init out of range"); s = CRISP_EINVAL; }
    std::vector<KmJob> jobs;
    for (int32_t m = 0; m < M; ++m) {
        const int32_t lo = sub[m], w = sub[m + 1] - sub[m], hl = w / 2;
        jobs.push_back({lo, hl});
        jobs.push_back({lo + hl, w - hl});
    }
    if (s == CRISP_OK) {
        size_t tb = sizeof(float) * (size_t)TS * ix->Dp, rb = sizeof(int64_t) * (size_t)TS,
               ib = sizeof(int32_t) * init.size(), cb = sizeof(uint16_t) * (size_t)M * N;
        size_t tot = tb + rb + ib + cb + 4 * 256;
        BCUDA(cudaMallocAsync(&tmp, tot, st));
        uint8_t *cur = (uint8_t *)tmp;
        auto take = [&](size_t n) { uint8_t *r = cur; cur += (n + 255) / 256 * 256; return r; };
        float *T = (float *)take(tb);
        int64_t *drs = (int64_t *)take(rb);
        int32_t *dinit = (int32_t *)take(ib);
        uint16_t *cells = (uint16_t *)take(cb);
        BCUDA(cudaMemcpyAsync(drs, ks.data(), rb, cudaMemcpyHostToDevice, st));
        BCUDA(cudaMemcpyAsync(dinit, init.data(), ib, cudaMemcpyHostToDevice, st));
        if (s == CRISP_OK) {
            k_gather_rows<<<(unsigned)std::min<long long>(grid1((long long)TS * ix->Dp, 256), 152LL * 32), 256, 0, st>>>(
                ix->Xr, ix->Dp, (const long long *)drs, TS, T);
            BCUDA(cudaGetLastError());
        }
        // centroids are laid out [M][2][K][H] = jobs in order
        // Lloyd's assignment steps and the final cells on the tensor cores
        BSTEP(kmeans_batched(T, TS, ix->Dp, jobs, K, H, dinit, p->kmeans_iters, ix->cent, st, D, sub));
        BSTEP(crisp_tc_assign(ix->Xr, N, D, ix->Dp, M, K, H, sub, ix->cent, cells, nullptr, st));
        // ---- B4: CSR per subspace
        for (int32_t m = 0; m < M && s == CRISP_OK; ++m)
            BSTEP(crisp_csr_build(cells + (size_t)m * N, N, K * K, ix->offsets + (size_t)m * (K * K + 1),
                                  ix->ids + (size_t)m * N, st));
        // ---- B5: sign codes
        BSTEP(crisp_sign_codes(ix->Xr, N, ix->Dp, ix->codes, st));
        // ---- F2: low-precision row copies
        BSTEP(crisp_make_copies(ix, p->copies, st));
        BCUDA(cudaStreamSynchronize(st));
        cudaFreeAsync(tmp, st);
    }
    BSTEP(crisp_finish_index(ix, st));
    BCUDA(cudaStreamSynchronize(st));
#undef BSTEP
#undef BCUDA
    if (s != CRISP_OK) {
        cudaStreamSynchronize(st);
        crisp_free(ix);
        return s;
    }
    *out = ix;
    return CRISP_OK;
}

// ==================================================================== F2 C ABI
extern "C" crisp_status crisp_quantize_bf16(const float *Xr, int64_t N, int32_t Dp, uint16_t *Xb, void *stream) {
    CRISP_REQUIRE(Xr && Xb && N >= 0 && Dp >= 1, "crisp_quantize_bf16: bad arguments");
    long long n = (long long)N * Dp;
    if (n == 0) return CRISP_OK;
    k_quant_bf16<<<(unsigned)std::min<long long>(grid1(n, 256), 152LL * 32), 256, 0, as_stream(stream)>>>(Xr, n, Xb);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

extern "C" crisp_status crisp_quantize_e4m3(const float *Xr, int64_t N, int32_t Dp, uint8_t *X8, float *scale,
                                            void *stream) {
    CRISP_REQUIRE(Xr && X8 && scale && N >= 0 && Dp >= 1, "crisp_quantize_e4m3: bad arguments");
    if (N == 0) return CRISP_OK;
    k_quant_e4m3<<<(unsigned)std::min<long long>(grid1((long long)N * 32, 256), 152LL * 32), 256, 0,
                   as_stream(stream)>>>(Xr, N, Dp, X8, scale);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_make_copies(crisp_index *ix, uint32_t copies, cudaStream_t st) {
    if ((copies & 1u) && !ix->Xb) {
        size_t b = sizeof(uint16_t) * (size_t)ix->N * ix->Dp;
        CRISP_CK(cudaMalloc((void **)&ix->Xb, b));
        ix->bytes += (int64_t)b;
        crisp_status s = crisp_quantize_bf16(ix->Xr, ix->N, ix->Dp, ix->Xb, st);
        if (s) return s;
        CRISP_CK(cudaMalloc((void **)&ix->xbn2, sizeof(float) * (size_t)ix->N));
        ix->bytes += (int64_t)(sizeof(float) * (size_t)ix->N);
        s = launch_row_norms_bf16(ix, st);
        if (s) return s;
    }
    if ((copies & 2u) && !ix->X8) {
        size_t b = (size_t)ix->N * ix->Dp, sb = sizeof(float) * (size_t)ix->N;
        CRISP_CK(cudaMalloc((void **)&ix->X8, b));
        CRISP_CK(cudaMalloc((void **)&ix->S8, sb));
        ix->bytes += (int64_t)(b + sb);
        crisp_status s = crisp_quantize_e4m3(ix->Xr, ix->N, ix->Dp, ix->X8, ix->S8, st);
        if (s) return s;
    }
    return CRISP_OK;
}

extern "C" crisp_status crisp_index_add_copies(crisp_index *ix, uint32_t copies, void *stream) {
    CRISP_REQUIRE(ix, "crisp_index_add_copies: null index");
    CRISP_REQUIRE((copies & ~3u) == 0, "crisp_index_add_copies: copies must be a mask of 1 (BF16) and 2 (FP8)");
    cudaStream_t st = as_stream(stream);
    crisp_status s = crisp_make_copies(ix, copies, st);
    if (s) return s;
    CRISP_CK(cudaStreamSynchronize(st));
    return CRISP_OK;
}
