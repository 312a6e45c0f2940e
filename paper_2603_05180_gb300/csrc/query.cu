// Query-side kernels of the CRISP engine (Algorithm 1, §4.3) for sm_103a.
//
//   k_rotate        Q1       y = x R, FP32, each output an fmaf chain over d in order
//   k_activate      Q2 + Q3  half distances, sorted lists, multi-sequence cell walk
//   k_count_cut     Q4 + Q5  collision counting in shared-memory id tiles + threshold cut
//   k_dist_flat     Q6       exact CR32 distances of (query, candidate) pairs, persistent
//                            (small batches, and the candidates the tensor-core re-rank of
//                            rerank_tc.cu keeps for the exact measure)
//   k_sched_pos     Q6 / F2  large batches: list position of each id range (the k-d query
//                   order of the groups is in rerank_tc.cu)
//   k_bound_select  Q6       per query: the candidates whose distance bound can reach the top-k
//   k_select_rows   Q6       per query: radix select + bitonic top-k of the exact distances
//   k_gunion        F2       large batches: per (query group, id range) the rows some member needs
//   k_score_flat    F2       BF16 / FP8 E4M3 coarse CR32 scores, persistent (small batches)
//   k_gscore        F2       the same coarse scores for large batches: each row read once per
//                            group and scored against its members, queries in tensor memory
//   k_short_select  F2       per query: the shortlist of the best coarse scores
#include <float.h>
#include <limits.h>
#include <math.h>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.cuh"
#include "ptx.cuh"

size_t crisp_query_order_scratch(int nq, int Dp);
crisp_status crisp_run_query_order(const float *Qr, int nq, int Dp, int G, void *scratch, int *qord, cudaStream_t st);

namespace {

// Subspace m covers dims [sub[m], sub[m+1]) (the index's boundaries: the equal
// split or the variance-aware ones); halves floor(w/2) and w - floor(w/2).
__device__ __forceinline__ void subspace_dev(const int32_t *__restrict__ sub, int m, int *lo, int *hl, int *hr) {
    int a = sub[m], b = sub[m + 1];
    int d = b - a;
    *lo = a;
    *hl = d / 2;
    *hr = d - d / 2;
}

// ------------------------------------------------------------------ block scans
// Exclusive scan of one int per thread over a block of NT threads; returns the
// prefix and writes the block total to *total.  `ws` holds NT/32 + 1 ints.
template <int NT>
__device__ __forceinline__ long long block_excl_scan(long long v, long long *ws, long long *total) {
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
        if (lane < NT / 32) ws[lane] = t;       // inclusive warp prefix
        if (lane == NT / 32 - 1) ws[NT / 32] = t;
    }
    __syncthreads();
    long long excl = x - v + (warp > 0 ? ws[warp - 1] : 0);
    *total = ws[NT / 32];
    __syncthreads();
    return excl;
}

// ======================================================= Q1 / B2 rotation
constexpr int RB_M = 128, RB_N = 128, RB_K = 16, RT = 8;

__global__ void __launch_bounds__(256) k_rotate(const float *__restrict__ X, long long N, int D, int ldx,
                                                const float *__restrict__ R, float *__restrict__ Y, int ldy) {
    __shared__ float As[RB_K][RB_M];
    __shared__ __align__(16) float Bs[RB_K][RB_N];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.y * RB_M;
    const int col0 = blockIdx.x * RB_N;
    float acc[RT][RT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < D; k0 += RB_K) {
        for (int e = tid; e < RB_M * RB_K; e += 256) {
            int r = e / RB_K, kk = e % RB_K;
            long long n = row0 + r;
            int d = k0 + kk;
            As[kk][r] = (n < N && d < D) ? X[n * ldx + d] : 0.0f;
        }
        for (int e = tid; e < RB_K * RB_N; e += 256) {
            int kk = e / RB_N, c = e % RB_N;
            int d = k0 + kk, j = col0 + c;
            Bs[kk][c] = (d < D && j < D) ? R[(long long)d * D + j] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RB_K; ++kk) {
            float a[RT], b[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) a[i] = As[kk][ty * RT + i];
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * RT]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * RT + 4]);
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int j = 0; j < RT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        long long n = row0 + ty * RT + i;
        if (n >= N) continue;
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            int c = col0 + tx * RT + j;
            if (c < ldy) Y[n * ldy + c] = c < D ? acc[i][j] : 0.0f;
        }
    }
}

__global__ void k_pad_rows(const float *__restrict__ X, long long N, int D, int ldx, float *__restrict__ Y, int ldy) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = N * (long long)ldy;
    for (; i < tot; i += (long long)gridDim.x * blockDim.x) {
        long long n = i / ldy;
        int j = (int)(i % ldy);
        Y[i] = j < D ? X[n * ldx + j] : 0.0f;
    }
}

// ================================================ Q2 + Q3 activation
constexpr int ACT_WARPS = 8;
constexpr int ACT_WARP_WORDS_FIXED = 7 * 64;

__global__ void __launch_bounds__(ACT_WARPS * 32) k_activate(IxView ix, const float *__restrict__ Qr, int nq, int phi,
                                                             int kk, long long budget, const QParam *__restrict__ qp,
                                                             int *__restrict__ act,
                                                             int *__restrict__ nact, long long *__restrict__ retrieved,
                                                             float *__restrict__ sorted_out, int *__restrict__ perm_out,
                                                             float *__restrict__ cost_first, float *__restrict__ cost_last) {
    extern __shared__ float sm[];
    const int K = ix.K, H = ix.H, K2 = K * K, m = blockIdx.y, M = ix.M;
    float *CtL = sm;
    float *CtR = CtL + H * K;
    int *offs = reinterpret_cast<int *>(CtR + H * K);
    float *wbase = reinterpret_cast<float *>(offs + K2 + 1);
    int lo, hl, hr;
    subspace_dev(ix.sub, m, &lo, &hl, &hr);
    const float *cL = ix.cent + ((long long)m * 2 + 0) * K * H;
    const float *cR = ix.cent + ((long long)m * 2 + 1) * K * H;
    for (int e = threadIdx.x; e < K * H; e += blockDim.x) {
        int c = e / H, d = e % H;
        CtL[d * K + c] = cL[e];
        CtR[d * K + c] = cR[e];
    }
    for (int e = threadIdx.x; e <= K2; e += blockDim.x) offs[e] = ix.offsets[(long long)m * (K2 + 1) + e];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * ACT_WARPS + warp;
    if (q >= nq) return;
    if (qp) {                           // per-query parameters
        phi = qp[q].phi;
        kk = qp[q].k;
        budget = qp[q].budget;
    }
    float *qs = wbase + warp * (2 * H + ACT_WARP_WORDS_FIXED);
    float *dl = qs + 2 * H, *dr = dl + 64, *s1 = dr + 64, *s2 = s1 + 64;
    int *p1 = reinterpret_cast<int *>(s2 + 64), *p2 = p1 + 64, *rowlen = p2 + 64;

    const float *qrow = Qr + (long long)q * ix.Dp + lo;
    for (int d = lane; d < hl + hr; d += 32) qs[d] = qrow[d];
    __syncwarp();
    // Dist1 / Dist2 (SEQ order) for centroids lane and lane + 32
    for (int c = lane; c < 64; c += 32) {
        float a = FLT_MAX, b = FLT_MAX;
        if (c < K) {
            a = 0.0f;
            for (int d = 0; d < hl; ++d) {
                float diff = qs[d] - CtL[d * K + c];
                a = fmaf(diff, diff, a);
            }
            b = 0.0f;
            for (int d = 0; d < hr; ++d) {
                float diff = qs[hl + d] - CtR[d * K + c];
                b = fmaf(diff, diff, b);
            }
        }
        dl[c] = a;
        dr[c] = b;
    }
    __syncwarp();
    // sort by (distance, index): rank = number of smaller keys
    for (int c = lane; c < K; c += 32) {
        float a = dl[c], b = dr[c];
        int ra = 0, rb = 0;
        for (int c2 = 0; c2 < K; ++c2) {
            float x = dl[c2], y = dr[c2];
            ra += (x < a) || (x == a && c2 < c);
            rb += (y < b) || (y == b && c2 < c);
        }
        s1[ra] = a; p1[ra] = c;
        s2[rb] = b; p2[rb] = c;
    }
    __syncwarp();
    if (sorted_out) {
        long long base = ((long long)q * M + m) * 2 * K;
        for (int c = lane; c < K; c += 32) {
            sorted_out[base + c] = s1[c]; perm_out[base + c] = p1[c];
            sorted_out[base + K + c] = s2[c]; perm_out[base + K + c] = p2[c];
        }
    }
    if (!act) return;

    // multi-sequence walk: row i's next cell is (i, rowlen[i]); it is on the
    // frontier once (i-1, rowlen[i]) has been visited.  Pop the frontier's
    // smallest (cost, i) until the ids retrieved reach the budget.
    for (int i = lane; i < 64; i += 32) rowlen[i] = 0;
    __syncwarp();
    long long got = 0;
    int count = 0;
    float c_first = 0.0f, c_last = 0.0f;
    int *out = act + ((long long)q * M + m) * K2;
    while (got < budget) {
        // the frontier's smallest (cost, row): costs are sums of squares (>= +0),
        // so their bit patterns order like the values and two warp minima find
        // it (no frontier row: key 0xFFFFFFFF, above every finite cost)
        unsigned key = 0xFFFFFFFFu;
        int row = INT_MAX;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int i = lane + 32 * r;
            if (i < K) {
                int j = rowlen[i];
                if (j < K && (i == 0 || rowlen[i - 1] > j)) {
                    const unsigned kb = __float_as_uint(s1[i] + s2[j]);
                    if (kb < key) { key = kb; row = i; }       // rows rise with r: ties keep the lower
                }
            }
        }
        const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
        if (kmin == 0xFFFFFFFFu) break;
        const int bi = __reduce_min_sync(0xffffffffu, key == kmin ? row : INT_MAX);
        const float bc = __uint_as_float(kmin);
        int j = rowlen[bi];
        int cell = p1[bi] * K + p2[j];
        if (count == 0) c_first = bc;
        c_last = bc;
        ++count;
        int w = (phi == 1 && count <= kk) ? 2 : 1;
        got += offs[cell + 1] - offs[cell];
        __syncwarp();
        if (lane == 0) {
            out[count - 1] = (w << 16) | cell;
            rowlen[bi] = j + 1;
        }
        __syncwarp();
    }
    if (lane == 0) {
        nact[(long long)q * M + m] = count;
        if (retrieved) retrieved[(long long)q * M + m] = got;
        if (cost_first) cost_first[(long long)q * M + m] = c_first;
        if (cost_last) cost_last[(long long)q * M + m] = c_last;
    }
}

// ==================================================== tile offsets
__global__ void k_tile_off(IxView ix, int *__restrict__ tile_off) {
    const int K2 = ix.K * ix.K, T = ix.T;
    long long total = (long long)ix.M * K2 * (T + 1);
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    int t = (int)(gid % (T + 1));
    long long mc = gid / (T + 1);
    int cell = (int)(mc % K2);
    int m = (int)(mc / K2);
    const int *off = ix.offsets + (long long)m * (K2 + 1);
    const int *ids = ix.ids + (long long)m * ix.N;
    int lo = off[cell], hi = off[cell + 1];
    long long target = (long long)t << CRISP_TILE_LOG2;
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if ((long long)ids[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    tile_off[gid] = lo;
}

// |x|^2 of every stored row: FP64 sum of squares rounded once to FP32 (the
// row norms of the tensor-core re-rank's distance expansion).
__global__ void k_row_norms(const float *__restrict__ Xr, long long N, int Dp, float *__restrict__ xn2) {
    const long long n = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= N) return;
    const float *x = Xr + n * Dp;
    double s = 0.0;
    for (int d = lane; d < Dp; d += 32) s += (double)x[d] * (double)x[d];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) xn2[n] = (float)s;
}

// |xb|^2 of the BF16 copy's rows, each value widened exactly to FP32.
__global__ void k_row_norms_bf16(const uint16_t *__restrict__ Xb, long long N, int Dp, float *__restrict__ xn2) {
    const long long n = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= N) return;
    const uint16_t *x = Xb + n * Dp;
    double s = 0.0;
    for (int d = lane; d < Dp; d += 32) {
        const double v = (double)__uint_as_float((unsigned)x[d] << 16);
        s += v * v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) xn2[n] = (float)s;
}

// ================================================== Q4 + Q5 count and cut
constexpr int CNT_NT = 512;
// Tuning (compile time): CNT_U flat ids per lane in flight, CNT_MINB resident
// CTAs per SM (the register budget), CNT_EC activated cells decoded once per
// query into shared memory (0: decoded again for every tile).
#ifndef CRISP_CNT_U
#define CRISP_CNT_U 4
#endif
#ifndef CRISP_CNT_MINB
#define CRISP_CNT_MINB 3
#endif
#ifndef CRISP_CNT_ECACHE
#define CRISP_CNT_ECACHE 0
#endif
// CRISP_CNT_QUAD: lanes take aligned 16-byte quads of the id array (four ids,
// those outside the cell's segment masked) instead of single ids; CNT_QU
// quads a lane in flight.
#ifndef CRISP_CNT_QUAD
#define CRISP_CNT_QUAD 1
#endif
#ifndef CRISP_CNT_QU
#define CRISP_CNT_QU 2
#endif
constexpr int CNT_U = CRISP_CNT_U;
constexpr int CNT_MINB = CRISP_CNT_MINB;
constexpr int CNT_EC = CRISP_CNT_ECACHE;
constexpr int CNT_QU = CRISP_CNT_QU;

// One flag bit per 32-bit counter word (four ids) of a tile.
constexpr int CNT_FLAG_WORDS = CRISP_TILE / 128;

struct CountShared {
    int base[129];
    union {
        unsigned hist[256];                // passes A and B (fallback / cap)
        unsigned flag[CNT_FLAG_WORDS];     // pass 1: counter words holding an id that reached tau
    };
    int w_gt[CNT_NT / 32], w_eq[CNT_NT / 32];
    long long w_eqbase[CNT_NT / 32], w_outbase[CNT_NT / 32];
    long long tile_sel, tile_eq;
    int sel_s, sel_need;
    // one batch of activated cells staged for one tile; only the cells with ids
    // in the tile are kept, so their flat starts strictly increase
    int c_pre[CNT_NT + 33];     // flat start of each kept cell; then the total, then INT_MAX
    int2 c_gw[CNT_NT + 1];      // per kept cell: id-array position of its flat id 0 (m N + first - c_pre)
                                // and its weight (entry CNT_NT: read by lanes past the end, unused)
    long long scan_ws[CNT_NT / 32 + 1];
    int ecache[CNT_EC > 0 ? CNT_EC : 1];   // (m << 20) | (w << 16) | cell per activated cell, when E <= CNT_EC
};

// Count tile t of query q into the byte counters `cnt` (zeroed here): every id
// of every activated cell that falls in the tile adds its cell's weight.  With
// FLAG, the counter's old value (returned by the shared atomic) tells whether
// this addition took the id from below tau to tau or above; such an id sets
// the flag bit of its counter word, so that the cut reads only flagged words
// (counters only grow, so every id with V >= tau crosses exactly once).  The
// cells are staged 512 at a time, keeping those with ids in the tile; the flat
// id range is then cut into one contiguous piece per warp, lanes on consecutive
// ids (coalesced loads).  A lane finds its cell from the cell starts inside its
// warp's 32 ids: lane j marks bit (start of cell ecur+1+j) - first id, the OR of
// the marks over the warp has one bit per start (starts are distinct), and a
// lane's cell is ecur plus the marks at or below its own position.
template <bool FLAG>
__device__ void count_tile(const IxView &ix, const int *__restrict__ actq, CountShared &S, int E, int t,
                           uint32_t *cnt, int tau = 0) {
    const int K2 = ix.K * ix.K, T = ix.T, M = ix.M;
    uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
    for (int i = threadIdx.x; i < CRISP_TILE / 16; i += CNT_NT) c4[i] = make_uint4(0, 0, 0, 0);
    if (FLAG)
        for (int i = threadIdx.x; i < CNT_FLAG_WORDS; i += CNT_NT) S.flag[i] = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tbase = t << CRISP_TILE_LOG2;
    const unsigned upto = 0xFFFFFFFFu >> (31 - lane);    // bits 0..lane
    for (int e0 = 0; e0 < E; e0 += CNT_NT) {
        const int ne = E - e0 < CNT_NT ? E - e0 : CNT_NT;
        int beg = 0, len = 0, w = 0, m = 0;
        const int i = threadIdx.x;
        if (i < ne) {
            const int e = e0 + i;
            int ent;
            if (CNT_EC > 0 && E <= CNT_EC) {
                const int pk = S.ecache[e];
                m = pk >> 20;
                ent = pk & 0xFFFFF;
            } else {
                int lo = 0, hi = M - 1;            // subspace m with base[m] <= e < base[m+1]
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (S.base[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                m = lo;
                ent = actq[(long long)m * K2 + (e - S.base[m])];
            }
            const int *to = ix.tile_off + ((long long)m * K2 + (ent & 0xFFFF)) * (T + 1) + t;
            beg = to[0];
            len = to[1] - beg;
            w = ent >> 16;
        }
#if CRISP_CNT_QUAD
        // flat units are the aligned quads of the id array that overlap a cell's
        // segment [gs, ge): one scan, quad counts in the high word, kept-cell
        // flags in the low word; per cell its first quad minus its flat start,
        // and the weight with the first quad's leading and the last quad's final
        // valid entry (gs & 3, (ge - 1) & 3)
        const int gs = m * (int)ix.N + beg, ge = gs + len;
        const int nqd = len > 0 ? ((ge + 3) >> 2) - (gs >> 2) : 0;
        long long tot;
        const long long ex = block_excl_scan<CNT_NT>(((long long)nqd << 32) | (len > 0 ? 1 : 0), S.scan_ws, &tot);
        const int total = (int)(tot >> 32), nne = (int)(tot & 0xFFFFFFFF);
        if (len > 0) {
            const int ci = (int)(ex & 0xFFFFFFFF), pre = (int)(ex >> 32);
            S.c_pre[ci] = pre;
            S.c_gw[ci] = make_int2((gs >> 2) - pre, (w & 0xFFFF) | ((gs & 3) << 16) | (((ge - 1) & 3) << 18));
        }
#else
        // one scan: id counts in the high word, kept-cell flags in the low word
        long long tot;
        const long long ex = block_excl_scan<CNT_NT>(((long long)len << 32) | (len > 0 ? 1 : 0), S.scan_ws, &tot);
        const int total = (int)(tot >> 32), nne = (int)(tot & 0xFFFFFFFF);
        if (len > 0) {
            const int ci = (int)(ex & 0xFFFFFFFF), pre = (int)(ex >> 32);
            S.c_pre[ci] = pre;
            S.c_gw[ci] = make_int2(m * (int)ix.N + beg - pre, w);
        }
#endif
        if (i <= 32) S.c_pre[nne + i] = i == 0 ? total : INT_MAX;
        __syncthreads();
        const int per = (total + CNT_NT / 32 - 1) / (CNT_NT / 32);
        const int f_lo = warp * per, f_hi = f_lo + per < total ? f_lo + per : total;
        if (f_lo < f_hi) {
            // the kept cell holding flat id f_lo
            int lo = 0, hi = nne - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (S.c_pre[mid] <= f_lo) lo = mid;
                else hi = mid - 1;
            }
            int ecur = lo;
            // counters and flags indexed by the global id (tbase is a multiple of 128)
            uint32_t *cnt_t = cnt - (tbase >> 2);
            unsigned *flag_t = S.flag - (tbase >> 7);
#if CRISP_CNT_QUAD
            const int4 *ids4 = reinterpret_cast<const int4 *>(ix.ids);
            for (int fb = f_lo; fb < f_hi; fb += 32 * CNT_QU) {
                int4 q4[CNT_QU];
                int wv[CNT_QU];
                unsigned vm[CNT_QU];
#pragma unroll
                for (int u = 0; u < CNT_QU; ++u) {
                    const int f0 = fb + 32 * u, f = f0 + lane;
                    int e = ecur;
                    // most 32-quad windows lie inside one cell: one broadcast read decides
                    if (S.c_pre[ecur + 1] < f0 + 32) {
                        const int B = S.c_pre[ecur + 1 + lane] - f0;     // > 0: cell ecur holds f0
                        unsigned bit;                                     // 1 << B, 0 for B outside [0, 31]
                        asm("shl.b32 %0, 1, %1;" : "=r"(bit) : "r"((unsigned)B));
                        const unsigned marks = __reduce_or_sync(0xffffffffu, bit);
                        e = ecur + __popc(marks & upto);
                        ecur = __shfl_sync(0xffffffffu, e, 31);
                    }
                    const int2 gw = S.c_gw[e];
                    // entries of the quad inside the cell's segment: from the first
                    // valid one of its first quad to the last valid one of its last
                    const int lo_j = f == S.c_pre[e] ? (gw.y >> 16) & 3 : 0;
                    const int hi_j = f == S.c_pre[e + 1] - 1 ? (gw.y >> 18) & 3 : 3;
                    vm[u] = f < f_hi ? (0xFu << lo_j) & (0xFu >> (3 - hi_j)) : 0u;
                    wv[u] = gw.y & 0xFFFF;
                    q4[u] = vm[u] ? __ldg(ids4 + (gw.x + f)) : make_int4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < CNT_QU; ++u) {
                    const int idv[4] = {q4[u].x, q4[u].y, q4[u].z, q4[u].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if ((vm[u] >> j) & 1u) {
                            const int id = idv[j], sh = (id & 3) * 8;
                            if (FLAG) {
                                const int ob =
                                    (int)((atomicAdd(&cnt_t[id >> 2], (uint32_t)wv[u] << sh) >> sh) & 0xFFu);
                                if ((unsigned)(ob + wv[u] - tau) < (unsigned)wv[u])
                                    atomicOr(&flag_t[id >> 7], 1u << ((id >> 2) & 31));
                            } else {
                                atomicAdd(&cnt_t[id >> 2], (uint32_t)wv[u] << sh);
                            }
                        }
                    }
                }
            }
#else
            for (int fb = f_lo; fb < f_hi; fb += 32 * CNT_U) {
                int ids_v[CNT_U], wv[CNT_U];
#pragma unroll
                for (int u = 0; u < CNT_U; ++u) {
                    const int f0 = fb + 32 * u, f = f0 + lane;
                    int e = ecur;
                    // most 32-id windows lie inside one cell: one broadcast read decides
                    if (S.c_pre[ecur + 1] < f0 + 32) {
                        const int B = S.c_pre[ecur + 1 + lane] - f0;     // > 0: cell ecur holds f0
                        unsigned bit;                                     // 1 << B, 0 for B outside [0, 31]
                        asm("shl.b32 %0, 1, %1;" : "=r"(bit) : "r"((unsigned)B));
                        const unsigned marks = __reduce_or_sync(0xffffffffu, bit);
                        e = ecur + __popc(marks & upto);
                        ecur = __shfl_sync(0xffffffffu, e, 31);
                    }
                    const int2 gw = S.c_gw[e];
                    wv[u] = gw.y;
                    ids_v[u] = f < f_hi ? __ldg(ix.ids + (gw.x + f)) : -1;
                }
#pragma unroll
                for (int u = 0; u < CNT_U; ++u) {
                    const int id = ids_v[u];
                    if (id >= 0) {
                        const int sh = (id & 3) * 8;
                        if (FLAG) {
                            // old byte ob crosses: tau - w <= ob < tau
                            const int ob = (int)((atomicAdd(&cnt_t[id >> 2], (uint32_t)wv[u] << sh) >> sh) & 0xFFu);
                            if ((unsigned)(ob + wv[u] - tau) < (unsigned)wv[u])
                                atomicOr(&flag_t[id >> 7], 1u << ((id >> 2) & 31));
                        } else {
                            atomicAdd(&cnt_t[id >> 2], (uint32_t)wv[u] << sh);
                        }
                    }
                }
            }
#endif
        }
        __syncthreads();
    }
    __syncthreads();   // zeroing and counting complete before anyone reads the tile (also when E == 0)
}

// Byte masks (0xFF per byte) of v > s and v == s for the four bytes of w.
// Counters are scores <= 2M <= 254.  For s in [0, 127] and v <= 127 the sum
// v + (127 - s) stays below 256 in every byte (no carry into the next byte) and
// has bit 7 set exactly when v > s; bytes above 127 are caught by their own
// bit 7.  The general SIMD compare serves the other thresholds.
__device__ __forceinline__ unsigned gt_mask(unsigned w, int s) {
    if (s < 0) return 0xFFFFFFFFu;
    if (s > 254) return 0u;
    if (s <= 127) {
        unsigned hi = w & 0x80808080u;                              // bytes >= 128 (> s)
        unsigned lo = ((w & 0x7F7F7F7Fu) + (unsigned)(127 - s) * 0x01010101u) & 0x80808080u;
        unsigned m = hi | lo;                                       // bit 7 of each byte
        return (m >> 7) * 0xFFu;
    }
    return __vcmpgtu4(w, (unsigned)s * 0x01010101u);
}
// Bit 7 of each byte of w set where that byte is > s (the other bits clear).
__device__ __forceinline__ unsigned gt_bits(unsigned w, int s) {
    if (s < 0) return 0x80808080u;
    if (s > 254) return 0u;
    if (s <= 127) return (((w & 0x7F7F7F7Fu) + (unsigned)(127 - s) * 0x01010101u) | w) & 0x80808080u;
    return __vcmpgtu4(w, (unsigned)s * 0x01010101u) & 0x80808080u;
}
__device__ __forceinline__ unsigned eq_mask(unsigned w, int s) {
    if (s < 0 || s > 255) return 0u;
    return __vcmpeq4(w, (unsigned)s * 0x01010101u);
}
// 0xFF for bytes b < nvalid of a word whose first byte is number `first`.
__device__ __forceinline__ unsigned valid_mask(int first, int nvalid) {
    int k = nvalid - first;
    if (k >= 4) return 0xFFFFFFFFu;
    if (k <= 0) return 0u;
    return (1u << (8 * k)) - 1u;
}

constexpr int CNT_WARP_BYTES = CRISP_TILE / (CNT_NT / 32);  // 4096 bytes of counters per warp
constexpr int CNT_ROUNDS = CNT_WARP_BYTES / 512;             // 16 bytes per lane per round

// Bit 7 of each byte of w that is > s, for s in [0, 127] (addc = (127 - s)
// 0x01010101): the branch-free core of gt_bits.
__device__ __forceinline__ unsigned gt_bits_lo(unsigned w, unsigned addc) {
    return (((w & 0x7F7F7F7Fu) + addc) | w) & 0x80808080u;
}

// One warp's emit over its counters: FAST (every byte valid and s_hi in
// [0, 127]) uses gt_bits_lo without the valid-byte masks.
template <bool FAST>
__device__ __forceinline__ int emit_count(const uint4 *wc, int s_hi, unsigned addc, int vlim) {
    const int lane = threadIdx.x & 31;
    int c_gt = 0;
#pragma unroll 4
    for (int r = 0; r < CNT_ROUNDS; ++r) {
        const int b0 = r * 512 + lane * 16;
        const uint4 v = wc[r * 32 + lane];
        const unsigned ws[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            c_gt += __popc(FAST ? gt_bits_lo(ws[u], addc) : gt_bits(ws[u], s_hi) & valid_mask(b0 + 4 * u, vlim));
    }
    return c_gt;
}

template <bool FAST>
__device__ __forceinline__ void emit_write(const uint4 *wc, int s_hi, unsigned addc, int vlim, long long pos_run,
                                           long long id0, int *candq, uint8_t *scoreq, long long stride) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < CNT_ROUNDS; ++r) {
        const int b0 = r * 512 + lane * 16;
        const uint4 v = wc[r * 32 + lane];
        const unsigned ws[4] = {v.x, v.y, v.z, v.w};
        unsigned gm[4];
        int g_l = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            gm[u] = FAST ? gt_bits_lo(ws[u], addc) : gt_bits(ws[u], s_hi) & valid_mask(b0 + 4 * u, vlim);
            g_l += __popc(gm[u]);
        }
        if (!__any_sync(0xffffffffu, g_l > 0)) continue;
        int s_in = g_l;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s_in, o);
            if (lane >= o) s_in += y;
        }
        long long pos = pos_run + (s_in - g_l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            unsigned m = gm[u];
            while (m) {
                const int bb = (__ffs(m) - 1) >> 3;     // byte of the lowest set bit 7 + 8 bb
                m &= m - 1;
                if (pos < stride) {
                    candq[pos] = (int)(id0 + b0 + 4 * u + bb);
                    if (scoreq) scoreq[pos] = (uint8_t)((ws[u] >> (8 * bb)) & 0xFFu);
                }
                ++pos;
            }
        }
        pos_run += __shfl_sync(0xffffffffu, s_in, 31);
    }
}

// Emit, in ascending id, the ids of tile t whose counter v satisfies v > s_hi
// (the need_eq == 0 form of emit_tile): count per warp, then each warp re-reads
// its counters and writes each lane's selected ids by walking the set bits of
// its masks.
__device__ long long emit_tile_gt(const IxView &ix, CountShared &S, const uint32_t *cnt, int t, int s_hi,
                                  long long out_base, int *candq, uint8_t *scoreq, long long stride) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long id0 = ((long long)t << CRISP_TILE_LOG2) + (long long)warp * CNT_WARP_BYTES;
    long long lim = ix.N - id0;
    const int vlim = lim <= 0 ? 0 : (lim >= CNT_WARP_BYTES ? CNT_WARP_BYTES : (int)lim);
    const uint4 *wc = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(cnt) + warp * CNT_WARP_BYTES);
    const bool fast = vlim == CNT_WARP_BYTES && s_hi >= 0 && s_hi <= 127;    // warp-uniform
    const unsigned addc = fast ? (unsigned)(127 - s_hi) * 0x01010101u : 0u;
    int c_gt = fast ? emit_count<true>(wc, s_hi, addc, vlim) : emit_count<false>(wc, s_hi, addc, vlim);
#pragma unroll
    for (int o = 16; o; o >>= 1) c_gt += __shfl_xor_sync(0xffffffffu, c_gt, o);
    if (lane == 0) S.w_gt[warp] = c_gt;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long outb = out_base;
        for (int w = 0; w < CNT_NT / 32; ++w) {
            S.w_outbase[w] = outb;
            outb += S.w_gt[w];
        }
        S.tile_sel = outb - out_base;
    }
    __syncthreads();
    const long long tot_sel = S.tile_sel;
    if (S.w_gt[warp] > 0) {
        if (fast) emit_write<true>(wc, s_hi, addc, vlim, S.w_outbase[warp], id0, candq, scoreq, stride);
        else emit_write<false>(wc, s_hi, addc, vlim, S.w_outbase[warp], id0, candq, scoreq, stride);
    }
    __syncthreads();
    return tot_sel;
}

// Emit, in ascending id, the ids of tile t whose counter v satisfies v >= tau
// (tau >= 1), from the flags count_tile<true> set: lane l of warp w owns flag
// word 32 w + l, i.e. counter words 32 (32 w + l) .. + 31 (128 ids), and reads
// only the flagged ones.  Ids past N are never counted, so their counters stay
// 0 and need no mask.  Same output as emit_tile_gt(s_hi = tau - 1).
__device__ long long emit_tile_flag(CountShared &S, const uint32_t *cnt, int t, int tau, long long out_base,
                                    int *candq, uint8_t *scoreq, long long stride) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fw = warp * 32 + lane;
    const unsigned fl = S.flag[fw];
    const uint32_t *cw = cnt + fw * 32;
    const long long id0 = ((long long)t << CRISP_TILE_LOG2) + (long long)fw * 128;
    int c = 0;
    for (unsigned m = fl; m; m &= m - 1) c += __popc(gt_bits(cw[__ffs(m) - 1], tau - 1));
    int c_in = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, c_in, o);
        if (lane >= o) c_in += y;
    }
    if (lane == 31) S.w_gt[warp] = c_in;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long outb = out_base;
        for (int w = 0; w < CNT_NT / 32; ++w) {
            S.w_outbase[w] = outb;
            outb += S.w_gt[w];
        }
        S.tile_sel = outb - out_base;
    }
    __syncthreads();
    const long long tot_sel = S.tile_sel;
    long long pos = S.w_outbase[warp] + (c_in - c);
    for (unsigned m = fl; m; m &= m - 1) {
        const int b = __ffs(m) - 1;
        const unsigned v = cw[b];
        for (unsigned g = gt_bits(v, tau - 1); g; g &= g - 1) {
            const int bb = (__ffs(g) - 1) >> 3;
            if (pos < stride) {
                candq[pos] = (int)(id0 + 4 * b + bb);
                if (scoreq) scoreq[pos] = (uint8_t)((v >> (8 * bb)) & 0xFFu);
            }
            ++pos;
        }
    }
    __syncthreads();
    return tot_sel;
}

// Emit, in ascending id, the ids of tile t whose counter v satisfies v > s_hi,
// or v == s_hi and the id is among the first need_eq such ids counted from the
// start of the query (*eq_seen holds how many came before this tile).  Each
// warp owns a contiguous 4 KB of counters, read 512 B per round without bank
// conflicts.  Returns the number emitted (block-uniform).
__device__ long long emit_tile(const IxView &ix, CountShared &S, const uint32_t *cnt, int t, int s_hi, long long need_eq,
                               long long *eq_seen, long long out_base, int *candq, uint8_t *scoreq, long long stride) {
    if (need_eq <= 0) return emit_tile_gt(ix, S, cnt, t, s_hi, out_base, candq, scoreq, stride);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long id0 = ((long long)t << CRISP_TILE_LOG2) + (long long)warp * CNT_WARP_BYTES;
    long long lim = ix.N - id0;
    const int vlim = lim <= 0 ? 0 : (lim >= CNT_WARP_BYTES ? CNT_WARP_BYTES : (int)lim);
    const uint4 *wc = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(cnt) + warp * CNT_WARP_BYTES);
    int c_gt = 0, c_eq = 0;
    const bool want_eq = need_eq > 0;
#pragma unroll 4
    for (int r = 0; r < CNT_ROUNDS; ++r) {
        int b0 = r * 512 + lane * 16;
        uint4 v = wc[r * 32 + lane];
        unsigned ws[4] = {v.x, v.y, v.z, v.w};
        if (b0 + 16 <= vlim) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c_gt += __popc(gt_mask(ws[u], s_hi)) >> 3;
                if (want_eq) c_eq += __popc(eq_mask(ws[u], s_hi)) >> 3;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                unsigned vm = valid_mask(b0 + 4 * u, vlim);
                c_gt += __popc(gt_mask(ws[u], s_hi) & vm) >> 3;
                if (want_eq) c_eq += __popc(eq_mask(ws[u], s_hi) & vm) >> 3;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        c_gt += __shfl_xor_sync(0xffffffffu, c_gt, o);
        c_eq += __shfl_xor_sync(0xffffffffu, c_eq, o);
    }
    if (lane == 0) { S.w_gt[warp] = c_gt; S.w_eq[warp] = c_eq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long eqb = *eq_seen, outb = out_base;
        for (int w = 0; w < CNT_NT / 32; ++w) {
            S.w_eqbase[w] = eqb;
            S.w_outbase[w] = outb;
            long long take = need_eq - eqb;
            take = take < 0 ? 0 : (take > S.w_eq[w] ? S.w_eq[w] : take);
            outb += S.w_gt[w] + take;
            eqb += S.w_eq[w];
        }
        S.tile_sel = outb - out_base;
        S.tile_eq = eqb - *eq_seen;
    }
    __syncthreads();
    long long eq_run = S.w_eqbase[warp], pos_run = S.w_outbase[warp];
    const long long tot_sel = S.tile_sel, tot_eq = S.tile_eq;
    if (S.w_gt[warp] + S.w_eq[warp] > 0) {
        for (int r = 0; r < CNT_ROUNDS; ++r) {
            int b0 = r * 512 + lane * 16;
            uint4 v = wc[r * 32 + lane];
            unsigned ws[4] = {v.x, v.y, v.z, v.w};
            unsigned gm[4], em[4];
            int e_l = 0, g_l = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                unsigned vm = valid_mask(b0 + 4 * u, vlim);
                gm[u] = gt_mask(ws[u], s_hi) & vm;
                em[u] = want_eq ? eq_mask(ws[u], s_hi) & vm : 0u;
                g_l += __popc(gm[u]) >> 3;
                e_l += __popc(em[u]) >> 3;
            }
            int e_in = e_l, e_tot = e_l;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, e_in, o);
                if (lane >= o) e_in += y;
            }
            e_tot = __shfl_sync(0xffffffffu, e_in, 31);
            long long eq_start = eq_run + (e_in - e_l);
            long long tk = need_eq - eq_start;
            int take = tk <= 0 ? 0 : (tk >= e_l ? e_l : (int)tk);
            int s_l = g_l + take, s_in = s_l;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s_in, o);
                if (lane >= o) s_in += y;
            }
            int s_tot = __shfl_sync(0xffffffffu, s_in, 31);
            if (s_l > 0) {
                long long pos = pos_run + (s_in - s_l);
                int taken = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        bool g = (gm[u] >> (8 * bb)) & 1u;
                        bool e = (em[u] >> (8 * bb)) & 1u;
                        bool sel = g || (e && taken < take);
                        taken += (e && !g && taken < take) ? 1 : 0;
                        if (sel) {
                            if (pos < stride) {
                                candq[pos] = (int)(id0 + b0 + 4 * u + bb);
                                if (scoreq) scoreq[pos] = (uint8_t)((ws[u] >> (8 * bb)) & 0xFFu);
                            }
                            ++pos;
                        }
                    }
                }
            }
            eq_run += e_tot;
            pos_run += s_tot;
        }
    }
    *eq_seen += tot_eq;
    __syncthreads();
    return tot_sel;
}

__global__ void __launch_bounds__(CNT_NT, CNT_MINB) k_count_cut(IxView ix, const int *__restrict__ act,
                                                      const int *__restrict__ nact, int nq, int tau, int kk,
                                                      long long cap, const QParam *__restrict__ qp,
                                                      int *__restrict__ cand, long long stride,
                                                      long long *__restrict__ ncand, uint8_t *__restrict__ score,
                                                      int *__restrict__ how) {
    extern __shared__ __align__(16) uint32_t cnt[];
    __shared__ CountShared S;
    const int q = blockIdx.x, M = ix.M, K2 = ix.K * ix.K;
    if (qp) {                           // per-query parameters
        tau = qp[q].tau;
        kk = qp[q].k;
        cap = qp[q].cap;
    }
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int m = 0; m < M; ++m) {
            S.base[m] = acc;
            acc += nact[(long long)q * M + m];
        }
        S.base[M] = acc;
    }
    __syncthreads();
    const int E = S.base[M];
    const int *actq = act + (long long)q * M * K2;
    if (CNT_EC > 0 && E <= CNT_EC) {
        for (int e = threadIdx.x; e < E; e += CNT_NT) {
            int lo = 0, hi = M - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (S.base[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            S.ecache[e] = (lo << 20) | actq[(long long)lo * K2 + (e - S.base[lo])];
        }
        __syncthreads();
    }
    int *candq = cand + (long long)q * stride;
    uint8_t *scoreq = score ? score + (long long)q * stride : nullptr;
    const int T = ix.T;

    // pass 1: C = {x : V[x] >= tau}
    long long total = 0, eq_seen = 0;
    for (int t = 0; t < T; ++t) {
        if (tau >= 1) {
            count_tile<true>(ix, actq, S, E, t, cnt, tau);
            total += emit_tile_flag(S, cnt, t, tau, total, candq, scoreq, stride);
        } else {
            count_tile<false>(ix, actq, S, E, t, cnt);
            total += emit_tile(ix, S, cnt, t, tau - 1, 0, &eq_seen, total, candq, scoreq, stride);
        }
    }
    int mode = 0;
    long long want = 0;
    int lo = 0;
    if (tau >= 1 && total < kk) { mode = 1; want = kk; lo = 1; }
    else if (cap > 0 && total > cap) { mode = 2; want = cap; lo = tau < 0 ? 0 : tau; }
    if (mode == 0) {
        if (threadIdx.x == 0) {
            ncand[q] = total;
            if (how) how[q] = total > stride ? -1 : 0;
        }
        return;
    }
    // pass A: histogram of V over v >= lo (rare path: fallback or cap)
    for (int i = threadIdx.x; i < 256; i += CNT_NT) S.hist[i] = 0;
    __syncthreads();
    for (int t = 0; t < T; ++t) {
        count_tile<false>(ix, actq, S, E, t, cnt);
        const long long id0 = ((long long)t << CRISP_TILE_LOG2);
        const uint8_t *cb = reinterpret_cast<const uint8_t *>(cnt);
        for (int i = threadIdx.x; i < CRISP_TILE; i += CNT_NT) {
            if (id0 + i >= ix.N) break;
            int v = cb[i];
            if (v >= lo) atomicAdd(&S.hist[v], 1u);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // largest s >= lo with #{V >= s} >= want, taking only the first `need`
        // ids at V == s; if no such s, every v >= lo
        long long above = 0;
        int s_star = -1;
        long long need = 0;
        for (int s = 255; s >= lo; --s) {
            long long h = S.hist[s];
            if (above + h >= want) { s_star = s; need = want - above; break; }
            above += h;
        }
        if (s_star < 0) { s_star = lo; need = INT_MAX; }
        S.sel_s = s_star;
        S.sel_need = (int)need;
    }
    __syncthreads();
    const int s_star = S.sel_s;
    const long long need = S.sel_need;
    long long out = 0;
    eq_seen = 0;
    for (int t = 0; t < T; ++t) {
        count_tile<false>(ix, actq, S, E, t, cnt);
        out += emit_tile(ix, S, cnt, t, s_star, need, &eq_seen, out, candq, scoreq, stride);
    }
    if (threadIdx.x == 0) {
        ncand[q] = out;
        if (how) how[q] = out > stride ? -1 : mode;
    }
}

// ==================================================== Q6 re-rank + top-k
constexpr int RR_NT = 256;
constexpr int RR_U = 8;   // 32-dim blocks in flight per lane

// CR32 block sum of one 32-dim block for the 8-lane group holding x4/q4 in lane
// (lane & 7): four fmaf into a lane partial, then the xor 4, 2, 1 tree.
__device__ __forceinline__ float cr32_block(float4 x, float4 qv, unsigned gmask) {
    float d0 = x.x - qv.x, d1 = x.y - qv.y, d2 = x.z - qv.z, d3 = x.w - qv.w;
    float a = 0.0f;
    a = fmaf(d0, d0, a);
    a = fmaf(d1, d1, a);
    a = fmaf(d2, d2, a);
    a = fmaf(d3, d3, a);
    a = a + __shfl_xor_sync(gmask, a, 4);
    a = a + __shfl_xor_sync(gmask, a, 2);
    a = a + __shfl_xor_sync(gmask, a, 1);
    return a;
}

constexpr int SEL_U = 8;    // keys a thread loads before using them (top-k passes)

struct TopkShared {
    unsigned hist[256];
    long long scan_ws[RR_NT / 32 + 1];
    unsigned skey[CRISP_KOUT_MAX];
    int sid[CRISP_KOUT_MAX];
    unsigned prefix;
    int need;
    unsigned count, fill;   // radix_kth_gather: keys in the selected bin; keys gathered
};

// Block-wide radix select over the FP32 keys dist[i * ks], i in [0, n)
// (non-negative, so their bit patterns order like the values): the key of the
// kk-th smallest (*prefix) and how many entries equal to it are among the kk
// smallest (*need).
__device__ void radix_kth(const float *distq, long long n, int kk, TopkShared &S, unsigned *out_prefix, int *out_need,
                          int ks = 1) {
    const int tid = threadIdx.x;
    unsigned prefix = 0, mask = 0;
    int need = kk;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += RR_NT) S.hist[i] = 0;
        __syncthreads();
        // keys share their leading bytes, so whole warps hit one bin: combine the
        // lanes of a bin first (one shared atomic per distinct bin per warp).
        // SEL_U keys a thread are loaded before any is binned (independent loads).
        for (long long i0 = 0; i0 < n; i0 += (long long)RR_NT * SEL_U) {
            unsigned key[SEL_U];
#pragma unroll
            for (int u = 0; u < SEL_U; ++u) {
                const long long i = i0 + (long long)u * RR_NT + tid;
                key[u] = i < n ? __float_as_uint(distq[i * ks]) : 0u;
            }
#pragma unroll
            for (int u = 0; u < SEL_U; ++u) {
                const long long i = i0 + (long long)u * RR_NT + tid;
                const bool hit = i < n && (key[u] & mask) == prefix;
                const unsigned bin = hit ? (key[u] >> shift) & 255u : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (hit && (__ffs(peers) - 1) == (int)(tid & 31)) atomicAdd(&S.hist[bin], (unsigned)__popc(peers));
            }
        }
        __syncthreads();
        if (tid == 0) {
            unsigned cum = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (cum + S.hist[b] >= (unsigned)need) break;
                cum += S.hist[b];
            }
            S.prefix = prefix | ((unsigned)b << shift);
            S.need = need - (int)cum;
        }
        __syncthreads();
        prefix = S.prefix;
        need = S.need;
        mask |= 255u << shift;
        __syncthreads();
    }
    *out_prefix = prefix;
    *out_need = need;
}

// One radix pass: the histogram of digit (key >> shift) & 255 over the keys
// whose bits under `mask` equal `prefix` (key(i) for i in [0, n)), then the
// digit holding the need-th of them; updates prefix / need (block-uniform).
template <class KeyAt>
__device__ void radix_pass(KeyAt key_at, long long n, int shift, unsigned &mask, unsigned &prefix, int &need,
                           TopkShared &S) {
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += RR_NT) S.hist[i] = 0;
    __syncthreads();
    for (long long i0 = 0; i0 < n; i0 += (long long)RR_NT * SEL_U) {
        unsigned key[SEL_U];
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {
            const long long i = i0 + (long long)u * RR_NT + tid;
            key[u] = i < n ? key_at(i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {
            const long long i = i0 + (long long)u * RR_NT + tid;
            const bool hit = i < n && (key[u] & mask) == prefix;
            const unsigned bin = hit ? (key[u] >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (hit && (__ffs(peers) - 1) == (int)(tid & 31)) atomicAdd(&S.hist[bin], (unsigned)__popc(peers));
        }
    }
    __syncthreads();
    if (tid == 0) {
        unsigned cum = 0;
        int b = 0;
        for (; b < 255; ++b) {
            if (cum + S.hist[b] >= (unsigned)need) break;
            cum += S.hist[b];
        }
        S.prefix = prefix | ((unsigned)b << shift);
        S.need = need - (int)cum;
        S.count = S.hist[b];
    }
    __syncthreads();
    prefix = S.prefix;
    need = S.need;
    mask |= 255u << shift;
    __syncthreads();
}

constexpr int BS_CAP = 2048;   // keys of the selected 16-bit prefix finished in shared memory

// The key of the kk-th smallest of n non-negative FP32 keys (contiguous): the
// two high digits are selected over the keys in global memory; the keys that
// share the resulting 16-bit prefix are then gathered into shared memory (when
// at most BS_CAP of them) and the two low digits are selected there.
__device__ unsigned radix_kth_gather(const float *keys, long long n, int kk, TopkShared &S, unsigned *buf) {
    unsigned prefix = 0, mask = 0;
    int need = kk;
    auto gk = [&](long long i) { return __float_as_uint(keys[i]); };
    radix_pass(gk, n, 24, mask, prefix, need, S);
    radix_pass(gk, n, 16, mask, prefix, need, S);
    if (S.count > (unsigned)BS_CAP) {
        radix_pass(gk, n, 8, mask, prefix, need, S);
        radix_pass(gk, n, 0, mask, prefix, need, S);
        return prefix;
    }
    if (threadIdx.x == 0) S.fill = 0;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += RR_NT) {
        const unsigned k = gk(i);
        if ((k & mask) == prefix) buf[atomicAdd(&S.fill, 1u)] = k;
    }
    __syncthreads();
    const long long m = S.fill;
    auto sk = [&](long long i) { return buf[i]; };
    radix_pass(sk, m, 8, mask, prefix, need, S);
    radix_pass(sk, m, 0, mask, prefix, need, S);
    return prefix;
}

// Visit, in list order, the entries with key < prefix and the first `need`
// with key == prefix (the list is in ascending id, so ties go to lower ids);
// f(slot, i) is called for each selected entry i with its output slot.
template <class F>
__device__ long long collect_ordered(const float *distq, long long n, unsigned prefix, int need, TopkShared &S, F f) {
    const int tid = threadIdx.x;
    long long eq_seen = 0, sel_seen = 0;
    for (long long c00 = 0; c00 < n; c00 += (long long)RR_NT * SEL_U) {
        unsigned keys[SEL_U];
        bool any = false;
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {
            const long long i = c00 + (long long)u * RR_NT + tid;
            keys[u] = i < n ? __float_as_uint(distq[i]) : 0xFFFFFFFFu;
            any = any || (i < n && keys[u] <= prefix);
        }
        // most chunks hold nothing at or below the k-th key: one vote skips them
        if (!__syncthreads_or(any)) continue;
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {                  // chunks in list order
            const long long i = c00 + (long long)u * RR_NT + tid;
            const unsigned key = keys[u];
            if (!__syncthreads_or(i < n && key <= prefix)) continue;
            int is_eq = (i < n && key == prefix);
            long long eq_tot;
            long long eq_off = block_excl_scan<RR_NT>(is_eq, S.scan_ws, &eq_tot);
            int sel = (i < n) && (key < prefix || (is_eq && eq_seen + eq_off < need));
            long long sel_tot;
            long long sel_off = block_excl_scan<RR_NT>(sel, S.scan_ws, &sel_tot);
            if (sel) f(sel_seen + sel_off, i);
            eq_seen += eq_tot;
            sel_seen += sel_tot;
        }
    }
    return sel_seen;
}

// Block-wide: the kk smallest (key, id) of n entries (keys from dist[], ids
// from candq[], ids ascending in list order), sorted, into S.skey / S.sid.
// Returns the number selected (min(n, kk)).
__device__ int select_topk(const float *distq, const int *candq, long long n, int kk, TopkShared &S) {
    const int tid = threadIdx.x;
    int nsel;
    if (n <= kk) {
        for (int i = tid; i < n; i += RR_NT) { S.skey[i] = __float_as_uint(distq[i]); S.sid[i] = candq[i]; }
        nsel = (int)n;
    } else {
        unsigned prefix;
        int need;
        radix_kth(distq, n, kk, S, &prefix, &need);
        collect_ordered(distq, n, prefix, need, S, [&](long long slot, long long i) {
            S.skey[slot] = __float_as_uint(distq[i]);
            S.sid[slot] = candq[i];
        });
        nsel = kk;
    }
    __syncthreads();
    // bitonic sort of CRISP_KOUT_MAX entries by (key, id); padding sorts last
    for (int i = nsel + tid; i < CRISP_KOUT_MAX; i += RR_NT) { S.skey[i] = 0xFFFFFFFFu; S.sid[i] = INT_MAX; }
    __syncthreads();
    for (int size = 2; size <= CRISP_KOUT_MAX; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < CRISP_KOUT_MAX; i += RR_NT) {
                int j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    unsigned ki = S.skey[i], kj = S.skey[j];
                    int ii = S.sid[i], ij = S.sid[j];
                    bool gt = ki > kj || (ki == kj && ii > ij);
                    if (gt == up) { S.skey[i] = kj; S.skey[j] = ki; S.sid[i] = ij; S.sid[j] = ii; }
                }
            }
            __syncthreads();
        }
    }
    return nsel;
}

// ------------------------------------------------ re-rank, streaming form
// Work items are (query, chunk of RF_CH candidates); item offsets per query
// come from a scan, and a persistent grid walks the items.  The distances go
// to dbuf; k_select_rows then picks the top-k of each query.
constexpr int RF_CH = 512;

__global__ void k_chunk_offsets(const long long *__restrict__ ncand, long long stride, int nq, int ch,
                                long long *__restrict__ off) {
    // single block: off[q] = sum over q' < q of ceil(n_q' / ch); off[nq] = total
    __shared__ long long ws[RR_NT / 32 + 1];
    long long carry = 0;
    for (int q0 = 0; q0 < nq; q0 += RR_NT) {
        int q = q0 + threadIdx.x;
        long long n = q < nq ? (ncand[q] < stride ? ncand[q] : stride) : 0;
        long long c = (n + ch - 1) / ch, tot;
        long long ex = block_excl_scan<RR_NT>(c, ws, &tot);
        if (q < nq) off[q] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) off[nq] = carry;
}

__global__ void __launch_bounds__(RR_NT, 5) k_dist_flat(IxView ix, const float *__restrict__ Qr, int nq,
                                                        const int *__restrict__ cand, long long stride,
                                                        const long long *__restrict__ ncand,
                                                        const long long *__restrict__ off, float *__restrict__ dbuf) {
    extern __shared__ __align__(16) float qs[];
    __shared__ int s_q;
    const int Dp = ix.Dp, nb = Dp / 32;
    // off == nullptr: every query has ceil(stride / RF_CH) items (empty ones end at once)
    const long long cpq = (stride + RF_CH - 1) / RF_CH;
    const long long total = off ? off[nq] : (long long)nq * cpq;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 3, l = threadIdx.x & 7;
    const unsigned gmask = 0xFFu << (lane & 24);
    int cur_q = -1;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        if (threadIdx.x == 0) {
            if (off) {
                int lo = 0, hi = nq - 1;             // query q with off[q] <= w < off[q+1]
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= w) lo = mid;
                    else hi = mid - 1;
                }
                s_q = lo;
            } else {
                s_q = (int)(w / cpq);
            }
        }
        __syncthreads();
        const int q = s_q;
        if (q != cur_q) {
            for (int d = threadIdx.x; d < Dp; d += RR_NT) qs[d] = Qr[(long long)q * Dp + d];
            cur_q = q;
        }
        __syncthreads();
        long long n = ncand[q] < stride ? ncand[q] : stride;
        const long long c0 = (off ? w - off[q] : w % cpq) * RF_CH;
        const long long c1 = c0 + RF_CH < n ? c0 + RF_CH : n;
        const int *candq = cand + (long long)q * stride;
        float *distq = dbuf + (long long)q * stride;
        for (long long i = c0 + g; i < c1; i += RR_NT / 8) {
            const float4 *row = reinterpret_cast<const float4 *>(ix.Xr + (long long)candq[i] * Dp) + l;
            float acc = 0.0f;
            for (int b0 = 0; b0 < nb; b0 += RR_U) {
                float4 v[RR_U];
#pragma unroll
                for (int u = 0; u < RR_U; ++u)
                    if (b0 + u < nb) v[u] = __ldcs(row + 8 * (b0 + u));
#pragma unroll
                for (int u = 0; u < RR_U; ++u) {
                    if (b0 + u < nb) {
                        float4 qv = *reinterpret_cast<const float4 *>(qs + 32 * (b0 + u) + 4 * l);
                        acc = acc + cr32_block(v[u], qv, gmask);
                    }
                }
            }
            if (l == 0) distq[i] = acc;
        }
        __syncthreads();
    }
}

// Coarse scores of every (query, candidate) pair, streaming form of the F2
// scorers: the same persistent walk over (query, chunk) items as k_dist_flat,
// rows read with several 16-byte loads in flight per lane.  The arithmetic is
// the CR32 order of cr32_row_bf16 / cr32_row_e4m3 (lane partials, xor tree,
// blocks in order), so the scores are the same bits.
constexpr int SB_U = 8;    // BF16: 16-byte loads in flight per lane (2 blocks per group each)
constexpr int SE_U = 4;    // E4M3: 16-byte loads in flight per lane (4 blocks per group each)

// CR32 distance of q to a BF16 row: an 8-lane group covers two 32-dim blocks
// per 16-byte slice j (lanes 0-3 block 2j, lanes 4-7 block 2j+1; lane li holds
// the CR32 lane partials 2li and 2li+1); SB_U slices are loaded before any is
// summed.
__device__ __forceinline__ float cr32_row_bf16_stream(const uint4 *row, const float *qs, int nb, int gl, int base,
                                                      unsigned gmask) {
    const int half = gl >> 2, li = gl & 3;
    const int nj = (nb + 1) >> 1;
    float acc = 0.0f;
    for (int j0 = 0; j0 < nj; j0 += SB_U) {
        uint4 v[SB_U];
#pragma unroll
        for (int u = 0; u < SB_U; ++u) {
            const int j = j0 + u;
            if (j < nj && 2 * j + half < nb) v[u] = __ldcs(row + 8 * j + gl);
            else v[u] = make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < SB_U; ++u) {
            const int j = j0 + u;
            if (j >= nj) break;                 // uniform over the group
            const int b = 2 * j + half;
            float e = 0.0f, o = 0.0f;
            if (b < nb) {
                const float *qv = qs + 32 * b + 8 * li;
                const unsigned w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    float d = __uint_as_float(w[t] << 16) - qv[2 * t];
                    e = fmaf(d, d, e);
                    d = __uint_as_float(w[t] & 0xFFFF0000u) - qv[2 * t + 1];
                    e = fmaf(d, d, e);
                }
#pragma unroll
                for (int t = 2; t < 4; ++t) {
                    float d = __uint_as_float(w[t] << 16) - qv[2 * t];
                    o = fmaf(d, d, o);
                    d = __uint_as_float(w[t] & 0xFFFF0000u) - qv[2 * t + 1];
                    o = fmaf(d, d, o);
                }
            }
            e = e + __shfl_xor_sync(gmask, e, 2);
            o = o + __shfl_xor_sync(gmask, o, 2);
            e = e + __shfl_xor_sync(gmask, e, 1);
            o = o + __shfl_xor_sync(gmask, o, 1);
            const float sm = e + o;
            const float slo = __shfl_sync(gmask, sm, base);
            const float shi = __shfl_sync(gmask, sm, base + 4);
            acc = acc + slo;
            if (2 * j + 1 < nb) acc = acc + shi;
        }
    }
    return acc;
}

// two E4M3 codes (low half of c) -> two FP32 values, exactly (E4M3 values are FP16 values)
__device__ __forceinline__ float2 e4m3x2_to_f32(unsigned c) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(c & 0xFFFFu), __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}

__device__ __forceinline__ float cr32_row_e4m3_stream(const uint4 *row, float sc, const float *qs, int nb, int gl,
                                                      int base, unsigned gmask) {
    const int h = gl & 1;
    const int nj = (nb + 3) >> 2;
    float acc = 0.0f;
    for (int j0 = 0; j0 < nj; j0 += SE_U) {
        uint4 v[SE_U];
#pragma unroll
        for (int u = 0; u < SE_U; ++u) {
            const int j = j0 + u;
            if (j < nj && 4 * j + (gl >> 1) < nb) v[u] = __ldcs(row + 8 * j + gl);
            else v[u] = make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < SE_U; ++u) {
            const int j = j0 + u;
            if (j >= nj) break;                 // uniform over the group
            const int b = 4 * j + (gl >> 1);
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (b < nb) {
                const float *qv = qs + 32 * b + 16 * h;
                const unsigned w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float2 x01 = e4m3x2_to_f32(w[t]), x23 = e4m3x2_to_f32(w[t] >> 16);
                    float d = x01.x * sc - qv[4 * t];
                    a[t] = fmaf(d, d, a[t]);
                    d = x01.y * sc - qv[4 * t + 1];
                    a[t] = fmaf(d, d, a[t]);
                    d = x23.x * sc - qv[4 * t + 2];
                    a[t] = fmaf(d, d, a[t]);
                    d = x23.y * sc - qv[4 * t + 3];
                    a[t] = fmaf(d, d, a[t]);
                }
            }
            const float t0 = a[0] + __shfl_xor_sync(gmask, a[0], 1);
            const float t1 = a[1] + __shfl_xor_sync(gmask, a[1], 1);
            const float t2 = a[2] + __shfl_xor_sync(gmask, a[2], 1);
            const float t3 = a[3] + __shfl_xor_sync(gmask, a[3], 1);
            const float sm = (t0 + t2) + (t1 + t3);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float sr = __shfl_sync(gmask, sm, base + 2 * r);
                if (4 * j + r < nb) acc = acc + sr;
            }
        }
    }
    return acc;
}

template <int PREC>
__global__ void __launch_bounds__(RR_NT, 4) k_score_flat(IxView ix, const float *__restrict__ Qr, int nq,
                                                         const int *__restrict__ cand, long long stride,
                                                         const long long *__restrict__ ncand,
                                                         const long long *__restrict__ off, float *__restrict__ dbuf) {
    extern __shared__ __align__(16) float qs[];
    __shared__ int s_q;
    const int Dp = ix.Dp, nb = Dp / 32;
    const long long total = off[nq];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 3, gl = threadIdx.x & 7, base = lane & 24;
    const unsigned gmask = 0xFFu << base;
    int cur_q = -1;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = nq - 1;             // query q with off[q] <= w < off[q+1]
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= w) lo = mid;
                else hi = mid - 1;
            }
            s_q = lo;
        }
        __syncthreads();
        const int q = s_q;
        if (q != cur_q) {
            for (int d = threadIdx.x; d < Dp; d += RR_NT) qs[d] = Qr[(long long)q * Dp + d];
            cur_q = q;
        }
        __syncthreads();
        const long long n = ncand[q] < stride ? ncand[q] : stride;
        const long long c0 = (w - off[q]) * RF_CH;
        const long long c1 = c0 + RF_CH < n ? c0 + RF_CH : n;
        const int *candq = cand + (long long)q * stride;
        float *distq = dbuf + (long long)q * stride;
        for (long long i = c0 + g; i < c1; i += RR_NT / 8) {
            const long long id = candq[i];
            // the row this group scores next comes into L2 while this one is summed
            const long long inext = i + RR_NT / 8;
            if (gl == 0 && inext < c1) {
                const long long idn = candq[inext];
                if (PREC == 1) bulk_prefetch_l2(ix.Xb + idn * Dp, (uint32_t)Dp * 2);
                else bulk_prefetch_l2(ix.X8 + idn * Dp, (uint32_t)Dp);
            }
            float acc;
            if (PREC == 1)
                acc = cr32_row_bf16_stream(reinterpret_cast<const uint4 *>(ix.Xb + id * Dp), qs, nb, gl, base, gmask);
            else
                acc = cr32_row_e4m3_stream(reinterpret_cast<const uint4 *>(ix.X8 + id * Dp), ix.S8[id], qs, nb, gl,
                                           base, gmask);
            if (gl == 0) distq[i] = acc;
        }
        __syncthreads();
    }
}

// ------------------------------------------- grouped scoring (row reuse)
// The candidate sets of a large batch overlap: on the 1M-row workload a row is a
// candidate of about 200 of 10,000 queries.  Queries are ordered by a k-d
// partition of their coordinates along the batch's top principal directions
// (crisp_run_query_order: queries close in space share most candidates) and
// cut into groups (of GT_G, at most GS_G); the id
// space into ranges of GS_SPAN ids.  k_gunion lists, for each (group, range),
// the rows some member needs, with the member mask and where each (row, member)
// distance goes in that member's list.  The coarse scorers (k_gscore)
// then read each listed row once and score it against every member that needs
// it.  The per-(row, query) arithmetic is the streaming kernels' CR32 order, and
// every distance lands in its own slot, so results do not depend on grouping.
constexpr int GS_G = 32;            // most members a group can have (bit mask)
constexpr int GS_SPAN = 4096;       // ids per range
constexpr int SCH_MAXQ = CRISP_GROUP_MAXQ;  // the ordering sorts 64-bit keys of 14-bit query numbers in one CTA
constexpr int GS_MINQ = 1024;       // batches smaller than this stream per query
constexpr int GS_MINSTRIDE = 2048;  // so do short candidate lists (shortlists)
constexpr int GU_NT = 256;
// scorer CTA: 24 warps, 80 registers a thread at most, no spills
constexpr int GK_NT = 768;

// pos[q][r] = first list position with id >= r GS_SPAN (r = 0..R).
__global__ void k_sched_pos(const int *__restrict__ cand, long long stride, const long long *__restrict__ ncand,
                            int nq, int R, int *__restrict__ pos) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nq * (R + 1)) return;
    const int q = (int)(e / (R + 1)), r = (int)(e % (R + 1));
    const long long n = ncand[q] < stride ? ncand[q] : stride;
    const int *c = cand + (long long)q * stride;
    const long long bound = (long long)r * GS_SPAN;
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)c[mid] < bound) lo = mid + 1;
        else hi = mid;
    }
    pos[e] = (int)lo;
}


struct GUnion {
    const int *qord;            // [nq]
    const int *pos;             // [nq][R + 1]
    int *ent_row;               // [cap] row id
    unsigned *ent_mask;         // [cap] members that need the row
    int *ent_pb;                // [cap] first pair slot of the row
    int *pair_pos;              // [cap] list position of each (row, member) pair, members in bit order
    int2 *items;                // [ngroups][R] (first entry, entries)
    unsigned long long *counts; // [0] entries, [1] pairs, [2] scoring item counter
    long long cap;
    int R, nq;
    int G;                      // queries per group (<= GS_G)
};

// Entry bucket of a member mask: 33 * lowest member + next member (32 if none).
constexpr int GU_NBK = 32 * 33;
__device__ __forceinline__ int gu_bucket(unsigned m) {
    const int lo = __ffs(m) - 1;
    const unsigned rest = m & (m - 1);
    return 33 * lo + (rest ? __ffs(rest) - 1 : 32);
}

// One block per (range r, group g): the group's candidates in the range, their
// rows' member masks, and the pair slots.
__global__ void __launch_bounds__(GU_NT) k_gunion(const int *__restrict__ cand, long long stride, GUnion u) {
    __shared__ unsigned mask[GS_SPAN];
    __shared__ int pbl[GS_SPAN];
    __shared__ int bk[GU_NBK];
    __shared__ int s_q[GS_G], s_base[GS_G], s_off[GS_G + 1];
    __shared__ long long scan_ws[GU_NT / 32 + 1];
    __shared__ long long s_eb, s_pb;
    __shared__ int s_np;
    const int r = blockIdx.x, g = blockIdx.y, lane = threadIdx.x & 31;
    const int gsize = (g + 1) * u.G <= u.nq ? u.G : u.nq - g * u.G;
    if (threadIdx.x < 32) {
        int a = 0, b = 0, q = 0;
        if (lane < gsize) {
            q = u.qord[g * u.G + lane];
            const long long row = (long long)q * (u.R + 1) + r;
            a = u.pos[row];
            b = u.pos[row + 1];
        }
        const int cnt = b - a;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        s_q[lane] = q;
        s_base[lane] = a;
        s_off[lane] = incl - cnt;
        if (lane == 31) {
            s_off[32] = incl;
            s_np = incl;
        }
    }
    for (int o = threadIdx.x; o < GS_SPAN; o += GU_NT) mask[o] = 0u;
    __syncthreads();
    const int np = s_np;
    const long long lo_id = (long long)r * GS_SPAN;
    for (int e = threadIdx.x; e < np; e += GU_NT) {
        int lo = 0, hi = GS_G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const int id = cand[(long long)s_q[lo] * stride + s_base[lo] + (e - s_off[lo])];
        atomicOr(&mask[id - lo_id], 1u << lo);
    }
    __syncthreads();
    // first pair slot of each row and the number of rows some member needs.  Any
    // assignment that gives each row popc(mask) consecutive slots will do, so
    // thread t takes the slots t, t + GU_NT, ... (conflict-free reads) and one
    // packed block scan (pairs high, rows low) places the threads.
    long long carry;
    {
        int pairs = 0, rows = 0;
#pragma unroll
        for (int k = 0; k < GS_SPAN / GU_NT; ++k) {
            const int c = __popc(mask[threadIdx.x + k * GU_NT]);
            pairs += c;
            rows += c > 0 ? 1 : 0;
        }
        int run = (int)(block_excl_scan<GU_NT>(((long long)pairs << 32) | rows, scan_ws, &carry) >> 32);
#pragma unroll
        for (int k = 0; k < GS_SPAN / GU_NT; ++k) {
            const int o = threadIdx.x + k * GU_NT;
            pbl[o] = run;
            run += __popc(mask[o]);
        }
    }
    if (threadIdx.x == 0) {
        const long long ne = carry & 0xFFFFFFFF;
        s_eb = (long long)atomicAdd(&u.counts[0], (unsigned long long)ne);
        s_pb = (long long)atomicAdd(&u.counts[1], (unsigned long long)np);
        const bool fits = s_eb + ne <= u.cap && s_pb + np <= u.cap;
        u.items[(long long)g * u.R + r] = make_int2(fits ? (int)s_eb : 0, fits ? (int)ne : 0);
        if (!fits) { s_eb = -1; }
    }
    __syncthreads();
    if (s_eb < 0) return;
    // entries, bucketed by (lowest member, next member): rows that share their
    // first members sit next to each other, so the warps of a scoring CTA work on
    // the same few members at a time (measured faster than id order).  The order
    // inside a bucket is arbitrary (every pair has its own slot, so results do
    // not depend on it).
    for (int i = threadIdx.x; i < GU_NBK; i += GU_NT) bk[i] = 0;
    __syncthreads();
    for (int o = threadIdx.x; o < GS_SPAN; o += GU_NT) {
        const unsigned m = mask[o];
        if (m) atomicAdd(&bk[gu_bucket(m)], 1);
    }
    __syncthreads();
    {
        constexpr int PER = (GU_NBK + GU_NT - 1) / GU_NT;
        int loc[PER], sum = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x * PER + k;
            loc[k] = i < GU_NBK ? bk[i] : 0;
            sum += loc[k];
        }
        long long tot;
        int run = (int)block_excl_scan<GU_NT>(sum, scan_ws, &tot);
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x * PER + k;
            if (i < GU_NBK) {
                bk[i] = run;
                run += loc[k];
            }
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < GS_SPAN; o += GU_NT) {
        const unsigned m = mask[o];
        if (m) {
            const long long ei = s_eb + atomicAdd(&bk[gu_bucket(m)], 1);
            u.ent_row[ei] = (int)(lo_id + o);
            u.ent_mask[ei] = m;
            u.ent_pb[ei] = (int)(s_pb + pbl[o]);
        }
    }
    // pair slots: member j of row o goes to slot first(o) + (members of o below j)
    for (int e = threadIdx.x; e < np; e += GU_NT) {
        int lo = 0, hi = GS_G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const int t = e - s_off[lo];
        const int id = cand[(long long)s_q[lo] * stride + s_base[lo] + t];
        const int o = id - (int)lo_id;
        const int slot = (int)s_pb + pbl[o] + __popc(mask[o] & ((1u << lo) - 1u));
        u.pair_pos[slot] = s_base[lo] + t;
    }
}

// The grouped scorers.  A CTA (one per SM) takes (block of id ranges, group)
// items; a warp takes one listed row at a time, keeps it in registers and scores
// it against every member of the group that needs it.  The group's 16 queries
// sit in tensor memory (TMEM), so a pair's query read stays out of the L1 /
// shared-memory pipe.
//  - BF16 / E4M3 rows (k_gscore): lane l holds the row's 32-dim block l, widened
//    (dequantised) to FP32 once per row, so the CR32 lane partials and their xor
//    tree ((a0+a4)+(a2+a6))+((a1+a5)+(a3+a7)) stay in registers.
// Each pair ends with the sum of block `lane` in every lane, and the block sums
// are added in block order by the batched gather.
// Packed FP32 pairs (sm_100 family): each half is one IEEE round-to-nearest
// subtraction or addition, exactly the scalar instruction's result.
__device__ __forceinline__ float2 sub2(float a0, float a1, float b0, float b1) {
    float2 d;
    asm("{.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tsub.rn.f32x2 d, a, b;\n\t"
        "mov.b64 {%0, %1}, d;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
    return d;
}

__device__ __forceinline__ float2 add2(float a0, float a1, float b0, float b1) {
    float2 d;
    asm("{.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tadd.rn.f32x2 d, a, b;\n\t"
        "mov.b64 {%0, %1}, d;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
    return d;
}

// ((a0 + a4) + (a2 + a6)) + ((a1 + a5) + (a3 + a7)), the first two levels as pairs
__device__ __forceinline__ float block_tree(const float (&a)[8]) {
    const float2 s01 = add2(a[0], a[1], a[4], a[5]), s23 = add2(a[2], a[3], a[6], a[7]);
    const float2 u = add2(s01.x, s01.y, s23.x, s23.y);
    return u.x + u.y;
}

template <int PREC>
__device__ __forceinline__ void row_load_lb(uint4 (&v)[8], const IxView &ix, long long id, int nb) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (lane < nb && ((PREC == 1 && u < 4) || (PREC == 2 && u < 2))) {
            if (PREC == 1) v[u] = __ldg(reinterpret_cast<const uint4 *>(ix.Xb + id * ix.Dp + 32 * lane + 8 * u));
            else v[u] = __ldg(reinterpret_cast<const uint4 *>(ix.X8 + id * ix.Dp + 32 * lane + 16 * u));
        } else {
            v[u] = make_uint4(0, 0, 0, 0);
        }
    }
}

// BF16 row slice widened to FP32 once per row (exact): xr[8 h + 2 i] and
// xr[8 h + 2 i + 1] are the low and high halves of word i of v[h].
__device__ __forceinline__ void widen_bf16(const uint4 (&v)[8], float (&xr)[32]) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const unsigned w[4] = {v[h].x, v[h].y, v[h].z, v[h].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xr[8 * h + 2 * i] = __uint_as_float(w[i] << 16);
            xr[8 * h + 2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
    }
}

// E4M3 row slice dequantised once per row: xr[4 i + k] = e4m3(byte k of word i)
// times the row scale, one FP32 product each (the F2 definition).
__device__ __forceinline__ void widen_e4m3(const uint4 (&v)[8], float sc, float (&xr)[32]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const unsigned w[4] = {v[h].x, v[h].y, v[h].z, v[h].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 x01 = e4m3x2_to_f32(w[i]), x23 = e4m3x2_to_f32(w[i] >> 16);
            xr[16 * h + 4 * i] = x01.x * sc;
            xr[16 * h + 4 * i + 1] = x01.y * sc;
            xr[16 * h + 4 * i + 2] = x23.x * sc;
            xr[16 * h + 4 * i + 3] = x23.y * sc;
        }
    }
}

// Batched gather of the block sums: each scored (row, member) pair leaves its
// 32 block sums as one row of the warp's gather buffer (row stride GB_LD, so a
// column read by 32 lanes hits 32 banks); once GB_K pairs are pending, lane p
// adds row p in block order and stores pair p's distance.
constexpr int GB_K = 16;
constexpr int GB_LD = 33;
// id ranges per scoring item (one query load per item): the CTAs in flight share
// one block of ranges, which must stay in L2
constexpr int GS_RB = 8;
// per-warp shared scratch: the gather rows
template <int PREC> __host__ __device__ constexpr int gw_floats() { return GB_K * GB_LD; }

// Group layout in tensor memory: member j of a group of GT_G = 16 occupies
// columns [32 j, 32 j + 32) of every lane quarter; 16 members x 32 columns fill
// the 512 columns of one CTA.

constexpr int GT_G = 16;
constexpr int GT_COLS = 512;

__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// BF16 / E4M3 rows, lane per block, the group's 16 queries in TMEM laid out the
// same way (member j at columns [32 j, 32 j + 32), lane l holding dims
// 32 l .. 32 l + 31 of block l): sum of block `lane` of the widened row xr.
__device__ __forceinline__ float block_sum_tm(const float (&xr)[32], uint32_t tq) {
    float a[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t q[16];
        tm_ld16(tq + 16 * h, q);
#pragma unroll
        for (int uu = 0; uu < 4; ++uu) {
            const int u = 4 * h + uu;
            const float2 t01 = sub2(xr[4 * u], xr[4 * u + 1], __uint_as_float(q[4 * uu]), __uint_as_float(q[4 * uu + 1]));
            const float2 t23 = sub2(xr[4 * u + 2], xr[4 * u + 3], __uint_as_float(q[4 * uu + 2]), __uint_as_float(q[4 * uu + 3]));
            float x = 0.0f;
            x = fmaf(t01.x, t01.x, x);
            x = fmaf(t01.y, t01.y, x);
            x = fmaf(t23.x, t23.x, x);
            x = fmaf(t23.y, t23.y, x);
            a[u] = x;
        }
    }
    return block_tree(a);
}

template <int PREC>
__global__ void __launch_bounds__(GK_NT, 1) k_gscore(IxView ix, const float *__restrict__ Qr, long long stride,
                                                    GUnion u, float *__restrict__ dbuf) {
    constexpr int NW = GK_NT / 32;
    extern __shared__ __align__(16) float gsm[];
    __shared__ long long s_it;
    __shared__ int s_mem[GT_G];
    __shared__ uint32_t s_tmem;
    const int Dp = ix.Dp, nb = Dp >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *gb = gsm + (size_t)warp * gw_floats<PREC>();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(GT_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tq0 = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const int ngroups = (u.nq + GT_G - 1) / GT_G;
    const int nrb = (u.R + GS_RB - 1) / GS_RB;
    const long long items = (long long)ngroups * nrb;
    int cur_g = -1;
    int npend = 0, pj = 0, ppos = 0;
    auto push = [&](float bs, int j, int slot) {
        gb[npend * GB_LD + lane] = bs;
        if (lane == npend) {
            pj = j;
            ppos = u.pair_pos[slot];
        }
        __syncwarp();
        if (++npend == GB_K) {
            if (lane < npend) {
                const float *row = gb + lane * GB_LD;
                float acc = 0.0f;
                for (int b = 0; b < nb; ++b) acc = acc + row[b];
                dbuf[(long long)s_mem[pj] * stride + ppos] = acc;
            }
            __syncwarp();
            npend = 0;
        }
    };
    for (;;) {
        if (threadIdx.x == 0) s_it = (long long)atomicAdd(&u.counts[2], 1ull);
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        const long long it = s_it;
        if (it >= items) break;
        const int g = (int)(it % ngroups), rb = (int)(it / ngroups);
        const int gsize = (g + 1) * GT_G <= u.nq ? GT_G : u.nq - g * GT_G;
        if (g != cur_g) {
            if (threadIdx.x < gsize) s_mem[threadIdx.x] = u.qord[g * GT_G + threadIdx.x];
            __syncthreads();
            for (int j = warp >> 2; j < GT_G; j += NW / 4) {
                const float *qrow = Qr + (long long)(j < gsize ? s_mem[j] : 0) * Dp;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t q[16];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const int d = 32 * lane + 16 * h + 4 * cc;
                        const uint4 x = j < gsize && d < Dp ? __ldg(reinterpret_cast<const uint4 *>(qrow + d))
                                                            : make_uint4(0, 0, 0, 0);
                        q[4 * cc] = x.x;
                        q[4 * cc + 1] = x.y;
                        q[4 * cc + 2] = x.z;
                        q[4 * cc + 3] = x.w;
                    }
                    __syncwarp();
                    tm_st16(tq0 + 32 * j + 16 * h, q);
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            cur_g = g;
            tm_fence_before();
            __syncthreads();
            tm_fence_after();
        }
        const int r_end = (rb + 1) * GS_RB < u.R ? (rb + 1) * GS_RB : u.R;
        for (int r = rb * GS_RB; r < r_end; ++r) {
            const int2 itm = u.items[(long long)g * u.R + r];
            const int e0 = itm.x, ne = itm.y;
            uint4 v[8];
            int id_next = warp < ne ? u.ent_row[e0 + warp] : 0;
            for (int e = warp; e < ne; e += NW) {
                const long long id = id_next;
                if (e + NW < ne) id_next = u.ent_row[e0 + e + NW];
                row_load_lb<PREC>(v, ix, id, nb);
                float xr[32];
                if (PREC == 1) widen_bf16(v, xr);
                else widen_e4m3(v, ix.S8[id], xr);
                const unsigned m0 = u.ent_mask[e0 + e];
                const int pb = u.ent_pb[e0 + e];
                unsigned m = m0;
                for (int i = 0; m; ++i) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    __syncwarp();
                    push(block_sum_tm(xr, tq0 + 32 * j), j, pb + i);
                }
            }
        }
        if (lane < npend) {
            const float *row = gb + lane * GB_LD;
            float acc = 0.0f;
            for (int b = 0; b < nb; ++b) acc = acc + row[b];
            dbuf[(long long)s_mem[pj] * stride + ppos] = acc;
        }
        __syncwarp();
        npend = 0;
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(GT_COLS) : "memory");
    }
}

// Grouped scoring of a batch into dbuf, or *done = false when the batch does not
// qualify (then the caller streams per query).
template <int PREC>
static crisp_status run_grouped(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand, int64_t stride,
                                const int64_t *ncand, float *dbuf, cudaStream_t st, bool *done) {
    *done = false;
    if (nq < GS_MINQ || nq > SCH_MAXQ || ix->Dp > 1024 || stride < GS_MINSTRIDE) return CRISP_OK;
    const int R = (int)((ix->N + GS_SPAN - 1) / GS_SPAN);
    const int G = GT_G;
    const int ngroups = (nq + G - 1) / G;
    const long long cap = (long long)nq * std::min<int64_t>(stride, ix->N);
    if (cap > (1LL << 31) - 1) return CRISP_OK;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += (b + 255) / 256 * 256; return o; };
    const size_t o_cnt = take(3 * sizeof(unsigned long long)), o_ord = take(crisp_query_order_scratch(nq, ix->Dp)),
                 o_qord = take(sizeof(int) * nq), o_pos = take(sizeof(int) * (size_t)nq * (R + 1)),
                 o_items = take(sizeof(int2) * (size_t)ngroups * R), o_row = take(sizeof(int) * (size_t)cap),
                 o_mask = take(sizeof(unsigned) * (size_t)cap), o_pb = take(sizeof(int) * (size_t)cap),
                 o_pp = take(sizeof(int) * (size_t)cap);
    uint8_t *buf = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&buf, off, st));
    GUnion u;
    u.counts = (unsigned long long *)(buf + o_cnt);
    u.qord = (int *)(buf + o_qord);
    u.pos = (int *)(buf + o_pos);
    u.items = (int2 *)(buf + o_items);
    u.ent_row = (int *)(buf + o_row);
    u.ent_mask = (unsigned *)(buf + o_mask);
    u.ent_pb = (int *)(buf + o_pb);
    u.pair_pos = (int *)(buf + o_pp);
    u.cap = cap;
    u.R = R;
    u.nq = nq;
    u.G = G;
    crisp_status s = CRISP_OK;
    do {
        cudaError_t e = cudaMemsetAsync(u.counts, 0, 3 * sizeof(unsigned long long), st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__); break; }
        s = crisp_run_query_order(Qr, nq, ix->Dp, G, buf + o_ord, (int *)u.qord, st);
        if (s) break;
        const long long npos = (long long)nq * (R + 1);
        k_sched_pos<<<(unsigned)((npos + 255) / 256), 256, 0, st>>>(cand, (long long)stride,
                                                                    (const long long *)ncand, nq, R, (int *)u.pos);
        CRISP_COUNT_LAUNCH();
        k_gunion<<<dim3(R, ngroups), GU_NT, 0, st>>>(cand, (long long)stride, u);
        CRISP_COUNT_LAUNCH();
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // one CTA per SM (its registers fill the SM), so its 512 TMEM columns are always free
        const size_t smem = sizeof(float) * (size_t)(GK_NT / 32) * gw_floats<PREC>();
        e = cudaFuncSetAttribute(k_gscore<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__); break; }
        k_gscore<PREC><<<sms, GK_NT, smem, st>>>(ix_view(ix), Qr, (long long)stride, u, dbuf);
        CRISP_COUNT_LAUNCH();
        e = cudaGetLastError();
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "grouped scoring", __FILE__, __LINE__); break; }
        *done = true;
    } while (0);
    crisp_scratch_free(buf, st);
    return s;
}

}  // namespace

// pos[q][r] of a large batch for the tensor-core re-rank: the first list
// position of query q with id >= r GS_SPAN (r = 0..R).
crisp_status crisp_run_group_pos(const int32_t *cand, int64_t stride, const int64_t *ncand, int32_t nq, int32_t R,
                                 int32_t *pos, cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    const long long npos = (long long)nq * (R + 1);
    k_sched_pos<<<(unsigned)((npos + 255) / 256), 256, 0, st>>>(cand, (long long)stride, (const long long *)ncand,
                                                                nq, R, pos);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

namespace {

// The S_keep best (score, list position) of each query's scored candidates, in
// list (ascending id) order: the shortlist for the FP32 re-rank.
__global__ void __launch_bounds__(RR_NT) k_short_select(int nq, const int *__restrict__ cand, long long stride,
                                                        const long long *__restrict__ ncand, int S_keep,
                                                        const float *__restrict__ dbuf, int *__restrict__ out,
                                                        long long out_stride, long long *__restrict__ nout,
                                                        const long long *__restrict__ S_per_query,
                                                        const QParam *__restrict__ qp) {
    __shared__ TopkShared S;
    const int q = blockIdx.x;
    if (qp) S_keep = qp[q].S;
    const long long n = ncand[q] < stride ? ncand[q] : stride;
    const int *candq = cand + (long long)q * stride;
    const float *distq = dbuf + (long long)q * stride;
    int *outq = out + (long long)q * out_stride;
    if (S_per_query) S_keep = (int)(S_per_query[q] < out_stride ? S_per_query[q] : out_stride);
    long long kept;
    if (n <= S_keep) {
        for (long long i = threadIdx.x; i < n; i += RR_NT) outq[i] = candq[i];
        kept = n;
    } else {
        unsigned prefix;
        int need;
        radix_kth(distq, n, S_keep, S, &prefix, &need);
        kept = collect_ordered(distq, n, prefix, need, S, [&](long long slot, long long i) { outq[slot] = candq[i]; });
    }
    if (threadIdx.x == 0) nout[q] = kept;
}

// Top-kk of each query's list into rows of ko >= kk entries (the rest padded
// -1 / +inf); with per-query parameters kk is the query's own k.
__global__ void __launch_bounds__(RR_NT) k_select_rows(int nq, const int *__restrict__ cand, long long stride,
                                                       const long long *__restrict__ ncand, int kk,
                                                       const QParam *__restrict__ qp, int ko,
                                                       const float *__restrict__ dbuf, long long *__restrict__ out_ids,
                                                       float *__restrict__ out_d) {
    __shared__ TopkShared S;
    const int q = blockIdx.x;
    if (qp) kk = qp[q].k;
    long long n = ncand[q] < stride ? ncand[q] : stride;
    int nsel = select_topk(dbuf + (long long)q * stride, cand + (long long)q * stride, n, kk, S);
    for (int r = threadIdx.x; r < ko; r += RR_NT) {
        bool ok = r < nsel && r < kk;
        out_ids[(long long)q * ko + r] = ok ? (long long)S.sid[r] : -1LL;
        out_d[(long long)q * ko + r] = ok ? __uint_as_float(S.skey[r]) : INFINITY;
    }
}

// Re-measure set of the tensor-core re-rank.  ub / lb hold, for every listed
// candidate, an upper and a lower bound of its CR32 distance.  With U a value
// that has at least kk upper bounds at or below it (so U >= the kk-th smallest
// upper bound), every candidate whose lower bound is <= U is written (in list
// order, so ascending id) to rc, their number to nr.  A candidate left out
// has CR32 distance >= its lower bound > U >= the kk-th smallest CR32 distance,
// so it cannot be among the kk nearest by (distance, id); the exact re-rank of
// rc alone therefore gives the top-kk of the whole list.
// If the scorer reported a failure (*err != 0) its bounds cannot be trusted
// and every candidate is kept, so the result is still exact.
// Target per query: kq[q] if given, else the query's k (qfield 0) or
// shortlist size S (qfield 1) from qp, else kk.  ub / lb: each pair's upper and
// lower bound, at the candidate's list position.
__global__ void __launch_bounds__(RR_NT) k_bound_select(int nq, const int *__restrict__ cand, long long stride,
                                                        const long long *__restrict__ ncand, int kk,
                                                        const QParam *__restrict__ qp, int qfield,
                                                        const long long *__restrict__ kq,
                                                        const float *__restrict__ ub, const float *__restrict__ lb,
                                                        const unsigned *__restrict__ err, int *__restrict__ rc,
                                                        long long *__restrict__ nr) {
    __shared__ TopkShared S;
    __shared__ unsigned gbuf[BS_CAP];
    const int q = blockIdx.x, tid = threadIdx.x;
    if (kq) kk = (int)(kq[q] < (long long)INT_MAX ? kq[q] : (long long)INT_MAX);
    else if (qp) kk = qfield ? qp[q].S : qp[q].k;
    const long long n = ncand[q] < stride ? ncand[q] : stride;
    const int *candq = cand + (long long)q * stride;
    int *rcq = rc + (long long)q * stride;
    if (n <= kk || (err && *err != 0u)) {
        for (long long i = tid; i < n; i += RR_NT) rcq[i] = candq[i];
        if (tid == 0) nr[q] = n;
        return;
    }
    unsigned ukey;
    if (kk <= RR_NT) {
        // The cut from each thread's smallest upper bound over its strided share:
        // V, the kk-th smallest of these minima, has at least kk upper bounds at
        // or below it (each thread's minimum is one), so the kk-th smallest upper
        // bound is <= V and V cuts exactly as well (it may keep a few more).
        // One read of the bounds; V found bit by bit (keys are non-negative
        // FP32, ordered like their bit patterns) with block-wide counts.
        const float *uq = ub + (long long)q * stride;
        unsigned mn = 0x7F800000u;              // +inf: a thread with no entry
        for (long long c00 = 0; c00 < n; c00 += (long long)RR_NT * SEL_U) {
            unsigned key[SEL_U];
#pragma unroll
            for (int u = 0; u < SEL_U; ++u) {
                const long long i = c00 + (long long)u * RR_NT + tid;
                key[u] = i < n ? __float_as_uint(uq[i]) : 0x7F800000u;
            }
#pragma unroll
            for (int u = 0; u < SEL_U; ++u) mn = key[u] < mn ? key[u] : mn;
        }
        unsigned p = 0;                          // smallest p with #{mn <= p} >= kk
        for (int b = 30; b >= 0; --b) {
            const unsigned c = p | ((1u << b) - 1u);
            if (__syncthreads_count(mn <= c) < kk) p |= 1u << b;
        }
        ukey = p;
    } else {
        ukey = radix_kth_gather(ub + (long long)q * stride, n, kk, S, gbuf);
    }
    const float U = __uint_as_float(ukey);
    const float *lq = lb + (long long)q * stride;
    long long run = 0;
    for (long long c00 = 0; c00 < n; c00 += (long long)RR_NT * SEL_U) {
        float lv[SEL_U];
        bool any = false;
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {
            const long long i = c00 + (long long)u * RR_NT + tid;
            lv[u] = i < n ? lq[i] : INFINITY;
            any = any || lv[u] <= U;
        }
        if (!__syncthreads_or(any)) continue;       // most chunks hold nothing to re-measure
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {
            const long long i = c00 + (long long)u * RR_NT + tid;
            const int sel = lv[u] <= U;
            if (!__syncthreads_or(sel)) continue;
            long long tot;
            const long long off = block_excl_scan<RR_NT>(sel, S.scan_ws, &tot);
            if (sel) rcq[run + off] = candq[i];
            run += tot;
        }
    }
    if (tid == 0) nr[q] = run;
}

__global__ void k_stats(int nq, const long long *ncand, const int *how, const long long *retrieved, int M,
                        const long long *nver, const long long *nfull, int tau, const QParam *qp,
                        crisp_query_stats *st) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    if (qp) tau = qp[q].tau;
    crisp_query_stats s;
    s.n_candidates = ncand[q];
    long long r = 0;
    if (retrieved)
        for (int m = 0; m < M; ++m) r += retrieved[(long long)q * M + m];
    s.n_retrieved = r;
    s.n_verified = nver ? nver[q] : ncand[q];
    s.n_full = nfull ? nfull[q] : ncand[q];
    int h = how ? how[q] : 0;
    s.fallback = h == 1;
    s.capped = h == 2;
    s.tau = tau;
    s._pad = h < 0 ? 1 : 0;
    st[q] = s;
}

// Row i of Q[perm[i]] into Y (per-query batches ordered by parameter class).
__global__ void k_gather_rows(const float *__restrict__ Q, int D, const int *__restrict__ perm, int n,
                              float *__restrict__ Y) {
    const long long tot = (long long)n * D;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / D;
        Y[e] = Q[(long long)perm[i] * D + (e - i * D)];
    }
}

// Result row i (and its stats) to row perm[i] of the caller's arrays.
__global__ void k_scatter_results(const long long *__restrict__ ids_t, const float *__restrict__ d2_t,
                                  const crisp_query_stats *__restrict__ st_t, int ko, const int *__restrict__ perm,
                                  int n, long long *__restrict__ ids, float *__restrict__ d2,
                                  crisp_query_stats *__restrict__ stats) {
    const long long tot = (long long)n * ko;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / ko, c = e - i * ko, o = (long long)perm[i] * ko + c;
        ids[o] = ids_t[e];
        d2[o] = d2_t[e];
        if (stats && c == 0) stats[perm[i]] = st_t[i];
    }
}

}  // namespace

// ============================================================ launchers
crisp_status launch_gather_rows(const float *Q, int32_t D, const int32_t *perm, int32_t n, float *Y, cudaStream_t st) {
    if (n <= 0) return CRISP_OK;
    const long long tot = (long long)n * D;
    const int blocks = (int)((tot + 255) / 256 < 152 * 32 ? (tot + 255) / 256 : 152 * 32);
    k_gather_rows<<<blocks, 256, 0, st>>>(Q, D, perm, n, Y);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status launch_scatter_results(const int64_t *ids_t, const float *d2_t, const crisp_query_stats *st_t, int32_t ko,
                                    const int32_t *perm, int32_t n, int64_t *ids, float *d2, crisp_query_stats *stats,
                                    cudaStream_t st) {
    if (n <= 0) return CRISP_OK;
    const long long tot = (long long)n * ko;
    const int blocks = (int)((tot + 255) / 256 < 152 * 32 ? (tot + 255) / 256 : 152 * 32);
    k_scatter_results<<<blocks, 256, 0, st>>>((const long long *)ids_t, d2_t, st_t, ko, perm, n, (long long *)ids, d2,
                                              stats);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}
crisp_status launch_pad_rows(const float *X, int64_t N, int32_t D, int32_t ldx, float *Y, int32_t ldy,
                             cudaStream_t st) {
    if (N <= 0) return CRISP_OK;
    long long tot = (long long)N * ldy;
    int blocks = (int)((tot + 255) / 256 < 152 * 64 ? (tot + 255) / 256 : 152 * 64);
    k_pad_rows<<<blocks, 256, 0, st>>>(X, N, D, ldx, Y, ldy);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status launch_tile_offsets(crisp_index *ix, cudaStream_t st) {
    long long total = (long long)ix->M * ix->K * ix->K * (ix->T + 1);
    k_tile_off<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ix_view(ix), ix->tile_off);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status launch_row_norms(crisp_index *ix, cudaStream_t st) {
    if (ix->N <= 0) return CRISP_OK;
    k_row_norms<<<(unsigned)((ix->N + 7) / 8), 256, 0, st>>>(ix->Xr, (long long)ix->N, ix->Dp, ix->xn2);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status launch_row_norms_bf16(crisp_index *ix, cudaStream_t st) {
    if (ix->N <= 0 || !ix->Xb || !ix->xbn2) return CRISP_OK;
    k_row_norms_bf16<<<(unsigned)((ix->N + 7) / 8), 256, 0, st>>>(ix->Xb, (long long)ix->N, ix->Dp, ix->xbn2);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status launch_write_stats(int32_t nq, const int64_t *ncand, const int32_t *how, const int64_t *retrieved,
                                int32_t M, const int64_t *nver, const int64_t *nfull, int32_t tau,
                                crisp_query_stats *stats, cudaStream_t st, const QParam *qp) {
    if (nq <= 0 || !stats) return CRISP_OK;
    k_stats<<<(nq + 255) / 256, 256, 0, st>>>(nq, (const long long *)ncand, how, (const long long *)retrieved, M,
                                              (const long long *)nver, (const long long *)nfull, tau, qp, stats);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

static size_t activate_smem(const crisp_index *ix) {
    return sizeof(float) * (2 * (size_t)ix->H * ix->K) + sizeof(int) * ((size_t)ix->K * ix->K + 1) +
           sizeof(float) * ACT_WARPS * (2 * (size_t)ix->H + ACT_WARP_WORDS_FIXED);
}

static crisp_status run_activate(const crisp_index *ix, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                 int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, float *sorted,
                                 int32_t *perm, cudaStream_t st, float *cost_first = nullptr,
                                 float *cost_last = nullptr, const QParam *qp = nullptr) {
    if (nq <= 0) return CRISP_OK;
    size_t smem = activate_smem(ix);
    CRISP_CK(cudaFuncSetAttribute(k_activate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((nq + ACT_WARPS - 1) / ACT_WARPS, ix->M);
    k_activate<<<grid, ACT_WARPS * 32, smem, st>>>(ix_view(ix), Qr, nq, phi, k, (long long)budget, qp, act, nact,
                                                   (long long *)retrieved, sorted, perm, cost_first, cost_last);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_activate(const crisp_index *ix, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, cudaStream_t st,
                                float *cost_first, float *cost_last, const QParam *qp) {
    return run_activate(ix, Qr, nq, phi, k, budget, act, nact, retrieved, nullptr, nullptr, st, cost_first, cost_last,
                        qp);
}

crisp_status crisp_run_count_cut(const crisp_index *ix, const int32_t *act, const int32_t *nact, int32_t nq,
                                 int32_t tau, int32_t k, int64_t cap, int32_t *cand, int64_t stride, int64_t *ncand,
                                 uint8_t *score, int32_t *how, cudaStream_t st, const QParam *qp) {
    if (nq <= 0) return CRISP_OK;
    CRISP_REQUIRE((int64_t)ix->M * ix->N < ((int64_t)1 << 31), "count: M * N must stay below 2^31");
    size_t smem = CRISP_TILE;
    CRISP_CK(cudaFuncSetAttribute(k_count_cut, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_count_cut<<<nq, CNT_NT, smem, st>>>(ix_view(ix), act, nact, nq, tau, k, (long long)cap, qp, cand,
                                         (long long)stride, (long long *)ncand, score, how);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_rerank_tc(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                 int64_t stride, const int64_t *ncand, int32_t k, const QParam *qp, int32_t ko,
                                 float *dbuf, int64_t *ids, float *d2, cudaStream_t st, bool *done);
crisp_status crisp_run_shortlist_tc(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                    int64_t stride, const int64_t *ncand, int32_t S, const int64_t *S_per_query,
                                    const QParam *qp, float *dbuf, int32_t *out, int64_t out_stride, int64_t *nout,
                                    cudaStream_t st, bool *done);

// Large batches (1,024 queries or more with long lists) take the tensor-core
// path of rerank_tc.cu (bounded TF32 scores, exact CR32 re-measure of the
// candidates that can reach the top-k); the rest stream every (query,
// candidate) pair.  Both give the top-k of the exact CR32 distances.
crisp_status crisp_run_rerank(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                              int64_t stride, const int64_t *ncand, int32_t k, float *dbuf, int64_t *ids, float *d2,
                              cudaStream_t st, bool no_alloc = false, bool may_group = true,
                              const QParam *qp = nullptr, int32_t ko = 0) {
    if (nq <= 0) return CRISP_OK;
    if (ko <= 0) ko = k;
    size_t smem = sizeof(float) * (size_t)ix->Dp;
    if (!no_alloc && may_group) {
        bool done = false;
        crisp_status ts = crisp_run_rerank_tc(ix, Qr, nq, cand, stride, ncand, k, qp, ko, dbuf, ids, d2, st, &done);
        if (ts || done) return ts;
    }
    long long *off = nullptr;           // no_alloc: a fixed number of items per query, no offsets
    if (!no_alloc) {
        CRISP_CK(crisp_scratch_alloc((void **)&off, sizeof(long long) * ((size_t)nq + 1), st));
        k_chunk_offsets<<<1, RR_NT, 0, st>>>((const long long *)ncand, (long long)stride, nq, RF_CH, off);
        CRISP_COUNT_LAUNCH();
    }
    if (smem > 48 * 1024)
        CRISP_CK(cudaFuncSetAttribute(k_dist_flat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dist_flat, RR_NT, smem);
        int grid = sms * (per_sm > 0 ? per_sm : 4);
        k_dist_flat<<<grid, RR_NT, smem, st>>>(ix_view(ix), Qr, nq, cand, (long long)stride,
                                               (const long long *)ncand, off, dbuf);
        CRISP_COUNT_LAUNCH();
    }
    k_select_rows<<<nq, RR_NT, 0, st>>>(nq, cand, (long long)stride, (const long long *)ncand, k, qp, ko, dbuf,
                                        (long long *)ids, d2);
    CRISP_COUNT_LAUNCH();
    if (off) crisp_scratch_free(off, st);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_bound_select(int32_t nq, const int32_t *cand, int64_t stride, const int64_t *ncand, int32_t k,
                                    const QParam *qp, int32_t qfield, const int64_t *kq, const float *ub,
                                    const float *lb, const unsigned *err, int32_t *rc, int64_t *nr, cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    k_bound_select<<<nq, RR_NT, 0, st>>>(nq, cand, (long long)stride, (const long long *)ncand, k, qp, qfield,
                                         (const long long *)kq, ub, lb, err, rc, (long long *)nr);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

crisp_status crisp_run_shortlist(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                 int64_t stride, const int64_t *ncand, int32_t precision, int32_t S, float *dbuf,
                                 int32_t *out, int64_t out_stride, int64_t *nout, cudaStream_t st,
                                 const int64_t *S_per_query, const QParam *qp, bool may_group) {
    if (nq <= 0) return CRISP_OK;
    size_t smem = sizeof(float) * (size_t)ix->Dp;
    bool grouped = false;
    if (may_group && precision == 1) {
        // large batches: bounds from one BF16 tensor-core pass, exact scores of the
        // candidates that can reach the shortlist only
        bool done = false;
        crisp_status ts = crisp_run_shortlist_tc(ix, Qr, nq, cand, stride, ncand, S, S_per_query, qp, dbuf, out,
                                                 out_stride, nout, st, &done);
        if (ts || done) return ts;
    }
    if (may_group) {
        crisp_status gs = precision == 1 ? run_grouped<1>(ix, Qr, nq, cand, stride, ncand, dbuf, st, &grouped)
                                         : run_grouped<2>(ix, Qr, nq, cand, stride, ncand, dbuf, st, &grouped);
        if (gs) return gs;
    }
    if (grouped) {
        k_short_select<<<nq, RR_NT, 0, st>>>(nq, cand, (long long)stride, (const long long *)ncand, S, dbuf, out,
                                             (long long)out_stride, (long long *)nout,
                                             (const long long *)S_per_query, qp);
        CRISP_COUNT_LAUNCH();
        CRISP_CK_LAUNCH();
        return CRISP_OK;
    }
    long long *off = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&off, sizeof(long long) * ((size_t)nq + 1), st));
    k_chunk_offsets<<<1, RR_NT, 0, st>>>((const long long *)ncand, (long long)stride, nq, RF_CH, off);
    CRISP_COUNT_LAUNCH();
    int dev = 0, sms = 152, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (precision == 1) {
        if (smem > 48 * 1024)
            CRISP_CK(cudaFuncSetAttribute(k_score_flat<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score_flat<1>, RR_NT, smem);
        k_score_flat<1><<<sms * (per_sm > 0 ? per_sm : 4), RR_NT, smem, st>>>(
            ix_view(ix), Qr, nq, cand, (long long)stride, (const long long *)ncand, off, dbuf);
    } else {
        if (smem > 48 * 1024)
            CRISP_CK(cudaFuncSetAttribute(k_score_flat<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score_flat<2>, RR_NT, smem);
        k_score_flat<2><<<sms * (per_sm > 0 ? per_sm : 4), RR_NT, smem, st>>>(
            ix_view(ix), Qr, nq, cand, (long long)stride, (const long long *)ncand, off, dbuf);
    }
    CRISP_COUNT_LAUNCH();
    k_short_select<<<nq, RR_NT, 0, st>>>(nq, cand, (long long)stride, (const long long *)ncand, S, dbuf, out,
                                         (long long)out_stride, (long long *)nout, (const long long *)S_per_query, qp);
    CRISP_COUNT_LAUNCH();
    crisp_scratch_free(off, st);
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

// ============================================================ C ABI steps
extern "C" crisp_status crisp_rotate_rows(const float *X, int64_t N, int32_t D, int32_t ldx, const float *R, float *Y,
                                          int32_t ldy, void *stream) {
    CRISP_REQUIRE(N >= 0 && D >= 1 && ldx >= D && ldy >= D, "crisp_rotate_rows: bad sizes");
    CRISP_REQUIRE(N == 0 || (X && R && Y), "crisp_rotate_rows: null pointer");
    CRISP_REQUIRE((const void *)X != (const void *)Y, "crisp_rotate_rows: Y overlaps X");
    if (N == 0) return CRISP_OK;
    dim3 grid((ldy + RB_N - 1) / RB_N, (unsigned)((N + RB_M - 1) / RB_M));
    CRISP_REQUIRE(grid.y <= 65535u * 1024u, "crisp_rotate_rows: N too large");
    for (long long r0 = 0; r0 < N; r0 += 65535LL * RB_M) {
        long long nr = N - r0 < 65535LL * RB_M ? N - r0 : 65535LL * RB_M;
        dim3 g((ldy + RB_N - 1) / RB_N, (unsigned)((nr + RB_M - 1) / RB_M));
        k_rotate<<<g, 256, 0, as_stream(stream)>>>(X + r0 * ldx, nr, D, ldx, R, Y + r0 * ldy, ldy);
        CRISP_COUNT_LAUNCH();
        CRISP_CK_LAUNCH();
    }
    return CRISP_OK;
}

static crisp_status check_query_step(const crisp_index *ix, const void *Qr, int32_t nq) {
    CRISP_REQUIRE(ix != nullptr, "null index");
    CRISP_REQUIRE(nq >= 0, "nq < 0");
    CRISP_REQUIRE(nq == 0 || Qr != nullptr, "null query pointer");
    return CRISP_OK;
}

extern "C" crisp_status crisp_half_dists(const crisp_index *ix, const float *Qr, int32_t nq, float *sorted,
                                         int32_t *perm, void *stream) {
    crisp_status s = check_query_step(ix, Qr, nq);
    if (s) return s;
    CRISP_REQUIRE(nq == 0 || (sorted && perm), "crisp_half_dists: null output");
    return run_activate(ix, Qr, nq, 0, 0, 0, nullptr, nullptr, nullptr, sorted, perm, as_stream(stream));
}

extern "C" crisp_status crisp_activate(const crisp_index *ix, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                       int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, void *stream) {
    crisp_status s = check_query_step(ix, Qr, nq);
    if (s) return s;
    CRISP_REQUIRE(phi == 0 || phi == 1, "crisp_activate: phi must be 0 or 1");
    CRISP_REQUIRE(budget >= 1, "crisp_activate: budget < 1");
    CRISP_REQUIRE(nq == 0 || (act && nact), "crisp_activate: null output");
    return run_activate(ix, Qr, nq, phi, k, budget, act, nact, retrieved, nullptr, nullptr, as_stream(stream));
}

extern "C" crisp_status crisp_activate_costs(const crisp_index *ix, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                             int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved,
                                             float *cost_first, float *cost_last, void *stream) {
    crisp_status s = check_query_step(ix, Qr, nq);
    if (s) return s;
    CRISP_REQUIRE(phi == 0 || phi == 1, "crisp_activate_costs: phi must be 0 or 1");
    CRISP_REQUIRE(budget >= 1, "crisp_activate_costs: budget < 1");
    CRISP_REQUIRE(nq == 0 || (act && nact), "crisp_activate_costs: null output");
    return run_activate(ix, Qr, nq, phi, k, budget, act, nact, retrieved, nullptr, nullptr, as_stream(stream),
                        cost_first, cost_last);
}

extern "C" crisp_status crisp_count_cut(const crisp_index *ix, const int32_t *act, const int32_t *nact, int32_t nq,
                                        int32_t tau, int32_t k, int64_t cap, int32_t *cand, int64_t cand_stride,
                                        int64_t *ncand, uint8_t *score, int32_t *how, void *stream) {
    crisp_status s = check_query_step(ix, act, nq);
    if (s) return s;
    CRISP_REQUIRE(ix->M <= 127, "crisp_count_cut: M > 127 overflows the byte counters");
    CRISP_REQUIRE(k >= 1 && cap >= 0 && (cap == 0 || cap >= k), "crisp_count_cut: need k >= 1, cap 0 or >= k");
    CRISP_REQUIRE(cap <= cand_stride, "crisp_count_cut: cap > cand_stride");
    CRISP_REQUIRE(cand_stride >= 1, "crisp_count_cut: cand_stride < 1");
    CRISP_REQUIRE(nq == 0 || (nact && cand && ncand), "crisp_count_cut: null pointer");
    return crisp_run_count_cut(ix, act, nact, nq, tau, k, cap, cand, cand_stride, ncand, score, how,
                               as_stream(stream), nullptr);
}

extern "C" crisp_status crisp_rerank(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                     int64_t cand_stride, const int64_t *ncand, int32_t k, int64_t *ids, float *sqdist,
                                     void *stream) {
    crisp_status s = check_query_step(ix, Qr, nq);
    if (s) return s;
    CRISP_REQUIRE(k >= 1 && k <= CRISP_KOUT_MAX, "crisp_rerank: k outside [1, 256]");
    CRISP_REQUIRE(nq == 0 || (cand && ncand && ids && sqdist), "crisp_rerank: null pointer");
    if (nq == 0) return CRISP_OK;
    cudaStream_t st = as_stream(stream);
    float *dbuf = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&dbuf, sizeof(float) * (size_t)nq * cand_stride, st));
    crisp_status r = crisp_run_rerank(ix, Qr, nq, cand, cand_stride, ncand, k, dbuf, ids, sqdist, st);
    crisp_scratch_free(dbuf, st);
    return r;
}

// ==================================================== no-allocation re-rank
// Distance scratch of crisp_rerank_noalloc: a fixed device array instead of an
// allocation, for callers that cannot allocate device memory while searching.
// In host code the name below is only a host-side stand-in; its device address
// is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) float g_rerank_noalloc_dist[CRISP_RERANK_NOALLOC_MAX];

#include <mutex>
static std::mutex g_noalloc_mu;
static float *g_noalloc_ptr[64];

// Device address of the array on the current device (set up on first use).
static crisp_status noalloc_scratch(float **out) {
    int dev = 0;
    CRISP_CK(cudaGetDevice(&dev));
    CRISP_REQUIRE(dev >= 0 && dev < 64, "crisp_rerank_noalloc: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        CRISP_CK(cudaGetSymbolAddress(&p, g_rerank_noalloc_dist));
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return CRISP_OK;
}

extern "C" crisp_status crisp_rerank_noalloc(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                             int64_t cand_stride, const int64_t *ncand, int32_t k, int64_t *ids,
                                             float *sqdist, void *stream) {
    crisp_status s = check_query_step(ix, Qr, nq);
    if (s) return s;
    CRISP_REQUIRE(k >= 1 && k <= CRISP_KOUT_MAX, "crisp_rerank_noalloc: k outside [1, 256]");
    CRISP_REQUIRE(cand_stride >= 1, "crisp_rerank_noalloc: cand_stride < 1");
    CRISP_REQUIRE(nq == 0 || (cand && ncand && ids && sqdist), "crisp_rerank_noalloc: null pointer");
    // compared without forming nq * cand_stride, which could overflow
    CRISP_REQUIRE(cand_stride <= (int64_t)CRISP_RERANK_NOALLOC_MAX / (nq > 0 ? nq : 1),
                  "crisp_rerank_noalloc: nq * cand_stride (%d x %lld) exceeds the fixed scratch of %d floats", nq,
                  (long long)cand_stride, CRISP_RERANK_NOALLOC_MAX);
    if (nq == 0) return CRISP_OK;
    float *dbuf = nullptr;
    s = noalloc_scratch(&dbuf);
    if (s) return s;
    return crisp_run_rerank(ix, Qr, nq, cand, cand_stride, ncand, k, dbuf, ids, sqdist, as_stream(stream), true);
}

extern "C" crisp_status crisp_shortlist(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                        int64_t cand_stride, const int64_t *ncand, int32_t precision, int32_t S,
                                        int32_t *out, int64_t out_stride, int64_t *nout, void *stream) {
    crisp_status s = check_query_step(ix, Qr, nq);
    if (s) return s;
    CRISP_REQUIRE(precision == 1 || precision == 2, "crisp_shortlist: precision must be 1 (BF16) or 2 (FP8)");
    CRISP_REQUIRE(precision != 1 || ix->Xb, "crisp_shortlist: the index has no BF16 copy");
    CRISP_REQUIRE(precision != 2 || ix->X8, "crisp_shortlist: the index has no FP8 copy");
    CRISP_REQUIRE(S >= 1 && out_stride >= S && cand_stride >= 1, "crisp_shortlist: need S >= 1, out_stride >= S");
    CRISP_REQUIRE(nq == 0 || (cand && ncand && out && nout), "crisp_shortlist: null pointer");
    if (nq == 0) return CRISP_OK;
    cudaStream_t st = as_stream(stream);
    float *dbuf = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&dbuf, sizeof(float) * (size_t)nq * cand_stride, st));
    s = crisp_run_shortlist(ix, Qr, nq, cand, cand_stride, ncand, precision, S, dbuf, out, out_stride, nout, st,
                            nullptr, nullptr, true);
    crisp_scratch_free(dbuf, st);
    return s;
}
