// Exact re-rank of large batches on the tcgen05 tensor cores (§4.3.2 Stage 3,
// the O(|C| D) verification the paper names as the dominant query cost, §4.4).
//
// The candidate lists of a large batch overlap: on the 1M-row workload a row is
// a candidate of about 200 of 10,000 queries.  The queries are ordered by a k-d
// partition of their coordinates along the batch's top principal directions
// (queries close in space share most candidates) and cut into groups of TG (64)
// queries; the id space into ranges of TSPAN ids.  For every (group, range) k_union lists the rows
// some member needs, with a 64-bit member mask and each (row, member) pair's
// slot in that member's list.  Then:
//
//   k_rerank_tc   each listed row is fetched once per group (16-byte cp.async
//                 copies straight into the 128-byte swizzled operand layout) and
//                 multiplied against the group's queries (one TMA tile) on the
//                 tensor cores: dot = x . q in one TF32 pass over the FP32 rows,
//                 or, when the index keeps its BF16 copy, in one BF16 pass over
//                 that copy against the queries rounded to BF16 (half the bytes
//                 per row), FP32 accumulation in tensor memory.  The epilogue
//                 forms the expansion d~ = |x|^2 + |q|^2 - 2 dot (|x|^2 of the
//                 FP32 row) and, from a proven error bound E, an upper and a
//                 lower bound of the pair's CR32 distance.
//   k_bound_select (query.cu) per query: U = the k-th smallest upper bound;
//                 every candidate whose lower bound is <= U is kept.
//   k_dist_flat + k_select_rows (query.cu): the kept candidates are measured
//                 exactly in the CR32 order and the top-k is taken from them.
//
// The same machinery makes the BF16 coarse-score shortlists of large batches
// (precision 1 and the learned path): the pass reads the BF16 copy against the
// queries rounded to BF16, the bounds are of the coarse score (the CR32
// distance of the FP32 query to the widened BF16 row, whose |xb|^2 the index
// keeps), the selection keeps what can reach the S-th smallest upper bound, and
// the kept candidates' coarse scores are computed exactly (k_score_flat).
//
// No candidate outside the kept set can be among the k nearest (its CR32
// distance exceeds U, which is at least the k-th smallest CR32 distance), and
// every kept distance is the CR32 value itself, so the result is bit-for-bit
// the one of measuring every candidate exactly.
//
// Error bound of d~ against the exact real distance d of the FP32 rows:
//  - TF32 keeps 10 mantissa bits, so each operand is within 2^-10 of itself
//    (relative, truncation or rounding) and each product within
//    (2^-9 + 2^-20) |x_i q_i|; summed, |dot~ - x.q| <= (2^-9 + 2^-20) S with
//    S = sum |x_i q_i| <= |x| |q| (Cauchy-Schwarz).  BF16 keeps 8 bits and
//    both roundings are to nearest (2^-9 each), so each product is within
//    (2^-8 + 2^-18) |x_i q_i| (the product of two BF16 values is exact in FP32);
//    for a coarse score the row is the BF16 row itself and only the query is
//    rounded: 2^-9 + 2^-18 (with margin);
//  - the tensor core's FP32 accumulation: every MMA step adds its K products
//    (K = 8 TF32, 16 BF16) to the running sum, charged (K + 1) 2^-22 S per
//    step (K + 1 additions, each within 2^-23 of a magnitude <= 2 S), over
//    Dp / K + 1 steps;
//  - operands or products below the FP32 normal range may be flushed: at most
//    2^-126 sqrt(Dp) (|x| + |q|) + Dp 2^-126, covered by c3 (|x| + |q|) + c4
//    with c3 = 2^-110, c4 = 2^-100;
//  - |x|^2 and |q|^2 are FP64 sums rounded once, and d~ takes three FP32
//    operations: all within 2^-19 (|x|^2 + |q|^2);
// so |d~ - d| <= E = c1 |x| |q| + c2 (|x|^2 + |q|^2) + c3 (|x| + |q|) + c4,
// c1 = 2 (p + (Dp / K + 1)(K + 1) 2^-22) 1.01 with p = 2^-9 + 2^-20 (TF32),
// 2^-8 + 2^-18 (BF16) or 2^-9 + 2^-18 (coarse), c2 = 2^-19.  The CR32 value d32 of the same pair
// (zero-padded blocks of 32 dims, a subtraction, a 4-term fma chain, a 3-level
// tree and Dp / 32 block additions per term) is within g d of d, with
// g = (Dp / 32 + 12) 2^-23 + 2^-20 (twice the first-order summation bound).
// Hence d32 lies in [d~ - E', d~ + E'] with E' = E + g (|d~| + E).
//
// Every mbarrier wait is bounded in time; a wait that gives up records an
// error word and the kernel winds down (waiting, bounded, for its copies and
// MMAs in flight, then freeing its tensor memory).  The bound selection reads
// the word and then keeps every candidate, so the result stays exact.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "ptx.cuh"

bool crisp_make_map_bf16(CUtensorMap *m, const uint16_t *base, long long rows, int cols, int ld, int box_rows);
bool crisp_make_map_f32(CUtensorMap *m, const float *base, long long rows, int cols, int ld, int box_rows);
crisp_status crisp_run_group_pos(const int32_t *cand, int64_t stride, const int64_t *ncand, int32_t nq, int32_t R,
                                 int32_t *pos, cudaStream_t st);
size_t crisp_query_order_scratch(int nq, int Dp);
crisp_status crisp_run_query_order(const float *Qr, int nq, int Dp, int G, void *scratch, int *qord, cudaStream_t st);
crisp_status crisp_run_bound_select(int32_t nq, const int32_t *cand, int64_t stride, const int64_t *ncand, int32_t k,
                                    const QParam *qp, int32_t qfield, const int64_t *kq, const float *ub,
                                    const float *lb, const unsigned *err, int32_t *rc, int64_t *nr, cudaStream_t st);
crisp_status crisp_run_shortlist(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                 int64_t stride, const int64_t *ncand, int32_t precision, int32_t S, float *dbuf,
                                 int32_t *out, int64_t out_stride, int64_t *nout, cudaStream_t st,
                                 const int64_t *S_per_query, const QParam *qp, bool may_group);
crisp_status crisp_run_rerank(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                              int64_t stride, const int64_t *ncand, int32_t k, float *dbuf, int64_t *ids, float *d2,
                              cudaStream_t st, bool no_alloc, bool may_group, const QParam *qp, int32_t ko);

namespace {

// Queries per group (N of the MMA; 64 or 128): a group's member mask is TGW
// 64-bit words.
#ifndef CRISP_TR_TG
#define CRISP_TR_TG 64
#endif
constexpr int TG = CRISP_TR_TG;
constexpr int TGW = TG / 64;
static_assert(TG == 64 || TG == 128, "query groups of 64 or 128");
constexpr int TR_MINQ = 256;        // smaller batches re-rank query by query
constexpr int TSPAN = 4096;         // ids per range (the ordering's range size)
// k_union tuning (compile time): threads a CTA, ids a lane loaded before use,
// CTAs an SM the registers are budgeted for (512 x 4: a full SM of warps).
#ifndef CRISP_TU_NT
#define CRISP_TU_NT 512
#endif
#ifndef CRISP_TU_U
#define CRISP_TU_U 4
#endif
#ifndef CRISP_TU_MINB
#define CRISP_TU_MINB 4
#endif
constexpr int TU_NT = CRISP_TU_NT;  // k_union threads
constexpr int TR_ROWS = 256;        // rows per tile: two M = 128 accumulators
// Stage geometry (tunable at compile time): TR_NS stages of TR_KB 32-float
// k-blocks of a tile each, TR_NB accumulator buffers, TR_RB id ranges per item.
#ifndef CRISP_TR_NS
#define CRISP_TR_NS (CRISP_TR_TG == 64 ? 4 : 3)
#endif
#ifndef CRISP_TR_KB
#define CRISP_TR_KB 1
#endif
#ifndef CRISP_TR_RB
#define CRISP_TR_RB 4
#endif
#ifndef CRISP_TR_PMAX
#define CRISP_TR_PMAX 2048
#endif
constexpr int TR_NS = CRISP_TR_NS;  // shared-memory stages
constexpr int TR_KB = CRISP_TR_KB;  // 32-float k-blocks of the tile's rows and queries per stage
constexpr int TR_NB = 512 / (2 * TG);   // tensor-memory accumulator buffers of 2 TG columns (512 in all)
constexpr int TR_LT = 128;          // copy threads (warps 8-11)
constexpr int TR_NT = 448;          // warps 0-7 epilogue, 8-11 copies, 12 tile preparation, 13 MMA issue
constexpr int TR_WC = 8, TR_WP = 12, TR_WM = 13;   // first copy warp, preparation warp, MMA warp
constexpr int TR_RB = CRISP_TR_RB;  // id ranges per work item
constexpr int TR_PMAX = CRISP_TR_PMAX;   // (row, member) pairs of a tile whose list positions are staged in shared memory
constexpr uint32_t TR_A_BYTES = 128 * 128;                     // 128 rows x one k-block
constexpr uint32_t TR_B_BYTES = TG * 128;                      // the group's queries x one k-block
constexpr uint32_t TR_STAGE = TR_KB * (2 * TR_A_BYTES + TR_B_BYTES);   // rows of both halves, then the queries

__device__ unsigned int g_tr_error;   // first failing wait: 1 + its site code

__device__ __forceinline__ void tr_error(unsigned site) { atomicCAS(&g_tr_error, 0u, 1u + site); }

// Group-ordered copy of the queries: slot s = g TG + j holds query qord[s]
// (zero rows past nq), with |q|^2 (FP64 sum rounded to FP32) and |q|.  One warp
// per slot.
// Qgb (when not null): the same rows rounded to BF16 (to nearest even), Dp64 =
// Dp rounded up to 64 columns, zeros past Dp.
__global__ void k_group_queries(const float *__restrict__ Qr, int nq, int Dp, const int *__restrict__ qord,
                                int nslots, float *__restrict__ Qg, uint16_t *__restrict__ Qgb, int Dp64,
                                int *__restrict__ gq, float *__restrict__ gn2, float *__restrict__ gn1) {
    const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (slot >= nslots) return;
    const int q = slot < nq ? qord[slot] : -1;
    double s = 0.0;
    for (int d = lane; d < Dp; d += 32) {
        const float v = q >= 0 ? Qr[(long long)q * Dp + d] : 0.0f;
        Qg[(long long)slot * Dp + d] = v;
        s += (double)v * (double)v;
    }
    if (Qgb)
        for (int d = lane; d < Dp64; d += 32) {
            const float v = (q >= 0 && d < Dp) ? Qr[(long long)q * Dp + d] : 0.0f;
            Qgb[(long long)slot * Dp64 + d] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        gq[slot] = q;
        gn2[slot] = (float)s;
        gn1[slot] = (float)sqrt(s);
    }
}

struct TUnion {
    const int *gq;                  // [ngroups * TG] query of each group slot, -1 past nq
    const int *pos;                 // [nq][R + 1] first list position with id >= r TSPAN
    int *ent_row;                   // [ecap] row id
    unsigned long long *ent_mask;   // [ecap][TGW] members that need the row
    int *ent_pb;                    // [ecap] first pair slot of the row
    float *ent_nx;                  // [ecap] |x|^2 of the row
    const float *xn2;               // [N] row norms of the index
    int *pair_pos;                  // [pcap] list position of each (row, member) pair, members in bit order
    int2 *items;                    // [ngroups][R] (first entry, entries)
    unsigned long long *counts;     // [0] entries, [1] pairs, [2] scoring item counter
    long long ecap, pcap;
    int R;
};

// Exclusive scan of one value per thread over the block (NT threads); the
// block total goes to *total.  ws holds NT / 32 + 1 values.
template <int NT>
__device__ __forceinline__ long long tr_block_scan(long long v, long long *ws, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < NT / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NT / 32) ws[lane] = t;
        if (lane == NT / 32 - 1) ws[NT / 32] = t;
    }
    __syncthreads();
    const long long excl = x - v + (warp > 0 ? ws[warp - 1] : 0);
    *total = ws[NT / 32];
    __syncthreads();
    return excl;
}

// One block per (range r, group g): the rows of the range that some member of
// the group needs, their member masks, and the slot of every (row, member)
// pair.  Entry order inside a (group, range) is arbitrary: every pair has its
// own slot, so nothing downstream depends on it.
// The ids of a group's members j = warp, warp + 8, ... (one warp's share) in
// the current range, visited as one flat list: lanes on consecutive entries
// (coalesced), TU_U entries a lane loaded before any is used (independent
// loads in flight), f(j, t, id) for entry t of member j.  A lane finds its
// member from the members' cumulative counts, held in registers.
constexpr int TU_NW = TU_NT / 32, TU_MPW = TG / TU_NW, TU_U = CRISP_TU_U;
static_assert(TG % TU_NW == 0 && TU_MPW <= 32, "k_union: members per warp");
template <class F>
__device__ __forceinline__ void warp_member_ids(const int *__restrict__ cand, long long stride, const int *s_q,
                                                const int *s_base, const int *s_cnt, int warp, int lane, F f) {
    int c = lane < TU_MPW ? s_cnt[warp + TU_NW * lane] : 0;
#pragma unroll
    for (int o = 1; o < TU_MPW; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, c, o);
        if (lane >= o) c += y;
    }
    int ends[TU_MPW];                        // inclusive scan: end of member i's entries
#pragma unroll
    for (int i = 0; i < TU_MPW; ++i) ends[i] = __shfl_sync(0xffffffffu, c, i);
    const int total = ends[TU_MPW - 1];
    for (int f0 = 0; f0 < total; f0 += 32 * TU_U) {
        int id[TU_U], jj[TU_U], tt[TU_U];
#pragma unroll
        for (int u = 0; u < TU_U; ++u) {
            const int fi = f0 + 32 * u + lane;
            int i = 0, start = 0;
#pragma unroll
            for (int k = 0; k < TU_MPW - 1; ++k)
                if (fi >= ends[k]) { i = k + 1; start = ends[k]; }
            const int j = warp + TU_NW * i;
            jj[u] = j;
            tt[u] = fi - start;
            id[u] = fi < total ? __ldg(cand + (long long)s_q[j] * stride + s_base[j] + (fi - start)) : -1;
        }
#pragma unroll
        for (int u = 0; u < TU_U; ++u)
            if (id[u] >= 0) f(jj[u], tt[u], id[u]);
    }
}

__global__ void __launch_bounds__(TU_NT, CRISP_TU_MINB) k_union(const int *__restrict__ cand, long long stride, TUnion u) {
    extern __shared__ __align__(16) unsigned long long usm[];
    unsigned long long *mask = usm;                      // [TSPAN][TGW]
    int *pbl = reinterpret_cast<int *>(usm + TSPAN * TGW);   // [TSPAN] pair base of each row, within the block
    __shared__ int s_q[TG], s_base[TG], s_cnt[TG], s_np[TG / 32];
    __shared__ long long scan_ws[TU_NT / 32 + 1];
    __shared__ long long s_eb, s_pb;
    const int r = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
    if (tid < TG) {
        const int q = u.gq[g * TG + tid];
        int a = 0, b = 0;
        if (q >= 0) {
            const long long row = (long long)q * (u.R + 1) + r;
            a = u.pos[row];
            b = u.pos[row + 1];
        }
        s_q[tid] = q < 0 ? 0 : q;
        s_base[tid] = a;
        s_cnt[tid] = b - a;
        const int w_np = __reduce_add_sync(0xffffffffu, b - a);
        if ((tid & 31) == 0) s_np[tid >> 5] = w_np;
    }
    for (int o = tid; o < TSPAN * TGW; o += TU_NT) mask[o] = 0ull;
    __syncthreads();
    int np = 0;
#pragma unroll
    for (int w = 0; w < TG / 32; ++w) np += s_np[w];
    const long long lo_id = (long long)r * TSPAN;
    const int warp = tid >> 5, lane = tid & 31;
    // member masks: every member's ids in the range set the member's bit
    // (32-bit halves of the little-endian 64-bit words: bit j of row o is bit
    // j & 31 of half 2 TGW o + (j >> 5))
    unsigned *mask32 = reinterpret_cast<unsigned *>(mask);
    warp_member_ids(cand, stride, s_q, s_base, s_cnt, warp, lane, [&](int j, int, int id) {
        atomicOr(&mask32[(id - (int)lo_id) * 2 * TGW + (j >> 5)], 1u << (j & 31));
    });
    __syncthreads();
    // thread t owns the ids t, t + TU_NT, ... (conflict-free reads); one packed
    // scan (pairs high, rows low) places every thread's rows and pairs
    constexpr int PER = TSPAN / TU_NT;
    int rows = 0, pairs = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int c = 0;
#pragma unroll
        for (int w = 0; w < TGW; ++w) c += __popcll(mask[(tid + k * TU_NT) * TGW + w]);
        pairs += c;
        rows += c > 0 ? 1 : 0;
    }
    long long tot;
    const long long ex = tr_block_scan<TU_NT>(((long long)pairs << 32) | rows, scan_ws, &tot);
    if (tid == 0) {
        const long long ne = tot & 0xFFFFFFFFll;
        s_eb = (long long)atomicAdd(&u.counts[0], (unsigned long long)ne);
        s_pb = (long long)atomicAdd(&u.counts[1], (unsigned long long)np);
        const bool fits = s_eb + ne <= u.ecap && s_pb + np <= u.pcap;
        u.items[(long long)g * u.R + r] = make_int2(fits ? (int)s_eb : 0, fits ? (int)ne : 0);
        if (!fits) {
            tr_error(10);       // never expected (the capacities bound every list); the selection then keeps all
            s_eb = -1;
        }
    }
    __syncthreads();
    if (s_eb < 0) return;
    int er = (int)(ex & 0xFFFFFFFFll), pr = (int)(ex >> 32);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int o = tid + k * TU_NT;
        int c = 0;
#pragma unroll
        for (int w = 0; w < TGW; ++w) c += __popcll(mask[o * TGW + w]);
        if (c) {
            const long long ei = s_eb + er;
            u.ent_row[ei] = (int)(lo_id + o);
#pragma unroll
            for (int w = 0; w < TGW; ++w) u.ent_mask[ei * TGW + w] = mask[o * TGW + w];
            u.ent_pb[ei] = (int)(s_pb + pr);
            u.ent_nx[ei] = u.xn2[lo_id + o];
            pbl[o] = pr;
            ++er;
            pr += c;
        }
    }
    __syncthreads();
    // pair slots: member j of row o goes to slot base(o) + (members of o below j)
    warp_member_ids(cand, stride, s_q, s_base, s_cnt, warp, lane, [&](int j, int t, int id) {
        const int o = id - (int)lo_id;
        int below = __popcll(mask[o * TGW + (j >> 6)] & ((1ull << (j & 63)) - 1ull));
        if (TGW > 1 && j >= 64) below += __popcll(mask[o * TGW]);
        u.pair_pos[s_pb + pbl[o] + below] = s_base[j] + t;
    });
}

// ------------------------------------ query order: k-d partition of the batch
// Groups whose members have similar candidate sets list fewer rows (fewer row
// fetches and MMAs for the same pairs).  Queries close in space share most of
// their activated cells, hence most candidates, so the batch is ordered by a
// k-d partition of the queries' coordinates along the batch's top PD_P
// principal directions: every node larger than a group splits at a
// group-aligned median of the coordinate with the widest range, so the leaves
// are the groups.  The directions come from PD_IT subspace iterations on up to
// PD_NS evenly spaced queries.  The order only decides which queries share a
// group (speed); every result is the same for any order.
#ifndef CRISP_PD_NS
#define CRISP_PD_NS 1024
#endif
#ifndef CRISP_PD_IT
#define CRISP_PD_IT 4
#endif
constexpr int PD_P = 4, PD_NS = CRISP_PD_NS, PD_IT = CRISP_PD_IT, PD_CH = 32, PD_NT = 128;
constexpr int KD_NT = 1024, KD_MAXN = 256, KD_PER = CRISP_GROUP_MAXQ / KD_NT;

// Sampled row r of n (r nq / n; every row when n = nq).
__device__ __forceinline__ long long pd_row(int r, int nq, int n) { return (long long)r * nq / n; }

// part[c][d] = sum over the sampled rows r of chunk c (blockIdx.y) of
// (Qr[q_r][d] - mu[d]) Y[r]; with Y null, the plain column sums (in .x).
__global__ void __launch_bounds__(PD_NT, 1) k_pd_back(const float *__restrict__ Qr, int nq, int Dp, int ns,
                                                   const float *__restrict__ mu, const float4 *__restrict__ Y,
                                                   float4 *__restrict__ part) {
    const int d = blockIdx.x * PD_NT + threadIdx.x, c = blockIdx.y;
    if (d >= Dp) return;
    const int r0 = (int)((long long)ns * c / PD_CH), r1 = (int)((long long)ns * (c + 1) / PD_CH);
    const float m = mu ? mu[d] : 0.0f;
    float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 8
    for (int r = r0; r < r1; ++r) {
        const float x = Qr[pd_row(r, nq, ns) * Dp + d] - m;
        if (Y) {
            const float4 y = Y[r];
            a.x += x * y.x;
            a.y += x * y.y;
            a.z += x * y.z;
            a.w += x * y.w;
        } else {
            a.x += x;
        }
    }
    part[(long long)c * Dp + d] = a;
}

// Sum of v over the CTA (fixed order), returned to every thread.
__device__ float pd_block_sum(float v, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        float t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    const float t = red[32];
    __syncthreads();
    return t;
}

// A fixed value in [-1, 1) for (d, j): the subspace iteration's start.
__device__ __forceinline__ float pd_start(int d, int j) {
    unsigned h = (unsigned)d * 0x9E3779B1u + (unsigned)j * 0x7F4A7C15u + 0x165667B1u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

// One CTA.  W = the chunks' sum of part; mode 0: mu = W.x / ns and V starts
// from pd_start; mode 1: V = W.  V's PD_P columns are then orthonormalised
// (modified Gram-Schmidt; a column that vanishes becomes a unit vector).
__global__ void __launch_bounds__(1024) k_pd_finish(const float4 *__restrict__ part, int Dp, int ns, int mode,
                                                    float *__restrict__ mu, float4 *__restrict__ V) {
    __shared__ float red[33];
    float *Vf = reinterpret_cast<float *>(V);
    for (int d = threadIdx.x; d < Dp; d += blockDim.x) {
        float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int c = 0; c < PD_CH; ++c) {
            const float4 p = part[(long long)c * Dp + d];
            w.x += p.x;
            w.y += p.y;
            w.z += p.z;
            w.w += p.w;
        }
        if (mode == 0) {
            mu[d] = w.x / (float)ns;
            w = make_float4(pd_start(d, 0), pd_start(d, 1), pd_start(d, 2), pd_start(d, 3));
        }
        V[d] = w;
    }
    __syncthreads();
    for (int j = 0; j < PD_P; ++j) {
        for (int i = 0; i < j; ++i) {
            float t = 0.0f;
            for (int d = threadIdx.x; d < Dp; d += blockDim.x) t += Vf[4 * d + i] * Vf[4 * d + j];
            const float dot = pd_block_sum(t, red);
            for (int d = threadIdx.x; d < Dp; d += blockDim.x) Vf[4 * d + j] -= dot * Vf[4 * d + i];
            __syncthreads();
        }
        float t = 0.0f;
        for (int d = threadIdx.x; d < Dp; d += blockDim.x) t += Vf[4 * d + j] * Vf[4 * d + j];
        const float nrm = sqrtf(pd_block_sum(t, red));
        for (int d = threadIdx.x; d < Dp; d += blockDim.x)
            Vf[4 * d + j] = nrm > 1e-30f ? Vf[4 * d + j] / nrm : (d == j ? 1.0f : 0.0f);
        __syncthreads();
    }
}

// Y[r] = (Qr[q_r] - mu) V for the rows r < n: one warp a row.
__global__ void __launch_bounds__(256) k_pd_proj(const float *__restrict__ Qr, int nq, int Dp, int n,
                                                 const float *__restrict__ mu, const float4 *__restrict__ V,
                                                 float4 *__restrict__ Y) {
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *x = Qr + pd_row(r, nq, n) * Dp;
    float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int d = lane; d < Dp; d += 32) {
        const float v = x[d] - mu[d];
        const float4 w = V[d];
        a.x += v * w.x;
        a.y += v * w.y;
        a.z += v * w.z;
        a.w += v * w.w;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        a.z += __shfl_xor_sync(0xffffffffu, a.z, o);
        a.w += __shfl_xor_sync(0xffffffffu, a.w, o);
    }
    if (lane == 0) Y[r] = a;
}

// FP32 bits mapped so that unsigned order is the value order.
__device__ __forceinline__ unsigned pd_key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float pd_unkey(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ float pd_comp(const float4 &y, int j) {
    return j == 0 ? y.x : j == 1 ? y.y : j == 2 ? y.z : y.w;
}

// One CTA: the k-d order qord of nq <= CRISP_GROUP_MAXQ queries with
// coordinates Y, leaves of G (nodes hold positions [start, start + size) of
// perm; a node larger than G splits into its h = G ceil(size / 2G) smallest
// along the chosen coordinate, ties by position, and the rest).  Per level:
// the coordinate ranges of every splitting node (shared atomics on ordered
// keys), a 4-bit radix select of each node's h-th smallest key, and a stable
// partition from one packed scan (keys below the pivot in the low half, equal
// keys in the high half: both counts stay below 2^16).
__global__ void __launch_bounds__(KD_NT, 1) k_kd_order(const float4 *__restrict__ Y, int nq, int G,
                                                       int *__restrict__ qord) {
    extern __shared__ __align__(16) uint8_t kd_sm[];
    unsigned *keys = reinterpret_cast<unsigned *>(kd_sm);
    uint16_t *perm = reinterpret_cast<uint16_t *>(keys + CRISP_GROUP_MAXQ);
    uint16_t *perm2 = perm + CRISP_GROUP_MAXQ;
    uint8_t *nid = reinterpret_cast<uint8_t *>(perm2 + CRISP_GROUP_MAXQ);
    __shared__ int n_start[KD_MAXN], n_size[KD_MAXN], n_h[KD_MAXN], n_need[KD_MAXN], n_dim[KD_MAXN];
    __shared__ int t_start[KD_MAXN], t_size[KD_MAXN];
    __shared__ unsigned n_pref[KD_MAXN], n_base[KD_MAXN], n_mn[KD_MAXN][PD_P], n_mx[KD_MAXN][PD_P];
    __shared__ unsigned hist[KD_MAXN * 16];
    __shared__ long long scan_ws[KD_NT / 32 + 1];
    __shared__ int s_nn, s_split;
    const int tid = threadIdx.x;
    for (int i = tid; i < nq; i += KD_NT) {
        perm[i] = (uint16_t)i;
        nid[i] = 0;
    }
    if (tid == 0) {
        n_start[0] = 0;
        n_size[0] = nq;
        s_nn = 1;
        s_split = nq > G;
    }
    __syncthreads();
    const int per = (nq + KD_NT - 1) / KD_NT, p0 = tid * per;
    while (s_split) {
        const int nn = s_nn;
        // coordinate ranges of the splitting nodes
        for (int i = tid; i < nn * PD_P; i += KD_NT) {
            n_mn[i / PD_P][i % PD_P] = 0xFFFFFFFFu;
            n_mx[i / PD_P][i % PD_P] = 0u;
        }
        __syncthreads();
        // (lanes hold consecutive positions, mostly of one node: reduced over the
        // warp per node, then one atomic per node and coordinate)
        for (int i0 = 0; i0 < nq; i0 += KD_NT) {
            const int i = i0 + tid;
            int n = 0;
            bool act = false;
            unsigned k[PD_P];
            if (i < nq) {
                n = nid[i];
                act = n_size[n] > G;
            }
            if (act) {
                const float4 y = Y[perm[i]];
#pragma unroll
                for (int j = 0; j < PD_P; ++j) k[j] = pd_key(pd_comp(y, j));
            }
            unsigned pending = __ballot_sync(0xffffffffu, act);
            while (pending) {
                const int src = __ffs(pending) - 1;
                const int tn = __shfl_sync(0xffffffffu, n, src);
                const bool mine = act && n == tn;
#pragma unroll
                for (int j = 0; j < PD_P; ++j) {
                    const unsigned mn = __reduce_min_sync(0xffffffffu, mine ? k[j] : 0xFFFFFFFFu);
                    const unsigned mx = __reduce_max_sync(0xffffffffu, mine ? k[j] : 0u);
                    if ((tid & 31) == src) {
                        atomicMin(&n_mn[tn][j], mn);
                        atomicMax(&n_mx[tn][j], mx);
                    }
                }
                pending &= ~__ballot_sync(0xffffffffu, mine);
            }
        }
        __syncthreads();
        for (int n = tid; n < nn; n += KD_NT) {
            if (n_size[n] <= G) continue;
            int best = 0;
            float bw = -1.0f;
            for (int j = 0; j < PD_P; ++j) {
                const float w = pd_unkey(n_mx[n][j]) - pd_unkey(n_mn[n][j]);
                if (w > bw) {
                    bw = w;
                    best = j;
                }
            }
            n_dim[n] = best;
            n_h[n] = (n_size[n] / 2 + G - 1) / G * G;
            n_need[n] = n_h[n];
            n_pref[n] = 0u;
        }
        __syncthreads();
        for (int i = tid; i < nq; i += KD_NT) {
            const int n = nid[i];
            keys[i] = n_size[n] > G ? pd_key(pd_comp(Y[perm[i]], n_dim[n])) : 0u;
        }
        // radix select, 4 bits a pass: the n_h-th smallest key of each splitting node
        unsigned mask = 0u;
        for (int shift = 28; shift >= 0; shift -= 4) {
            for (int i = tid; i < nn * 16; i += KD_NT) hist[i] = 0u;
            __syncthreads();
            // lanes with the same (node, digit) add once, by their lowest lane
            for (int i0 = 0; i0 < nq; i0 += KD_NT) {
                const int i = i0 + tid;
                unsigned bin = 0xFFFFFFFFu;
                if (i < nq) {
                    const int n = nid[i];
                    const unsigned k = keys[i];
                    if (n_size[n] > G && (k & mask) == n_pref[n]) bin = (unsigned)n * 16u + ((k >> shift) & 15u);
                }
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (bin != 0xFFFFFFFFu && __ffs(peers) - 1 == (tid & 31)) atomicAdd(&hist[bin], (unsigned)__popc(peers));
            }
            __syncthreads();
            for (int n = tid; n < nn; n += KD_NT) {
                if (n_size[n] <= G) continue;
                int cum = 0, b = 0;
                for (; b < 15; ++b) {
                    const int c = (int)hist[n * 16 + b];
                    if (cum + c >= n_need[n]) break;
                    cum += c;
                }
                n_pref[n] |= (unsigned)b << shift;
                n_need[n] -= cum;
            }
            mask |= 15u << shift;
            __syncthreads();
        }
        // stable partition: keys below the pivot, then the first n_need equal
        // keys, go to [start, start + h); the rest to [start + h, start + size)
        unsigned f[KD_PER];
        unsigned tot = 0u;
#pragma unroll
        for (int u = 0; u < KD_PER; ++u) {
            const int i = p0 + u;
            unsigned v = 0u;
            if (u < per && i < nq) {
                const int n = nid[i];
                if (n_size[n] > G) {
                    const unsigned k = keys[i];
                    v = (k < n_pref[n] ? 1u : 0u) | (k == n_pref[n] ? 0x10000u : 0u);
                }
            }
            f[u] = v;
            tot += v;
        }
        long long all;
        const unsigned excl = (unsigned)tr_block_scan<KD_NT>((long long)tot, scan_ws, &all);
        unsigned run = excl;
#pragma unroll
        for (int u = 0; u < KD_PER; ++u) {
            const int i = p0 + u;
            if (u < per && i < nq && (i == 0 || nid[i] != nid[i - 1])) n_base[nid[i]] = run;
            run += f[u];
        }
        __syncthreads();
        run = excl;
#pragma unroll
        for (int u = 0; u < KD_PER; ++u) {
            const int i = p0 + u;
            if (u < per && i < nq) {
                const int n = nid[i];
                if (n_size[n] > G) {
                    const unsigned b = n_base[n];
                    const int lt_b = (int)((run & 0xFFFFu) - (b & 0xFFFFu));
                    const int eq_b = (int)((run >> 16) - (b >> 16));
                    const int need = n_need[n];
                    const bool left = (f[u] & 1u) || ((f[u] >> 16) && eq_b < need);
                    const int lb = lt_b + (eq_b < need ? eq_b : need);
                    const int dst = left ? n_start[n] + lb : n_start[n] + n_h[n] + (i - n_start[n] - lb);
                    perm2[dst] = perm[i];
                } else {
                    perm2[i] = perm[i];
                }
            }
            run += f[u];
        }
        __syncthreads();
        uint16_t *tp = perm;
        perm = perm2;
        perm2 = tp;
        // the children
        if (tid == 0) {
            int m = 0, more = 0;
            for (int n = 0; n < nn; ++n) {
                if (n_size[n] > G) {
                    t_start[m] = n_start[n];
                    t_size[m++] = n_h[n];
                    t_start[m] = n_start[n] + n_h[n];
                    t_size[m++] = n_size[n] - n_h[n];
                    more |= n_h[n] > G || n_size[n] - n_h[n] > G;
                } else {
                    t_start[m] = n_start[n];
                    t_size[m++] = n_size[n];
                }
            }
            for (int n = 0; n < m; ++n) {
                n_start[n] = t_start[n];
                n_size[n] = t_size[n];
            }
            s_nn = m;
            s_split = more;
        }
        __syncthreads();
        const int nn2 = s_nn;
        for (int i = tid; i < nq; i += KD_NT) {
            int lo = 0, hi = nn2 - 1;          // last node with start <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (n_start[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            nid[i] = (uint8_t)lo;
        }
        __syncthreads();
    }
    for (int i = tid; i < nq; i += KD_NT) qord[i] = perm[i];
}

constexpr size_t kd_smem_bytes() { return (size_t)CRISP_GROUP_MAXQ * (4 + 2 + 2 + 1); }

// Groups smaller than KD_LEAF: each k-d leaf of KD_LEAF positions (the last one
// may be shorter) is split further, down to G, the same way (widest coordinate
// range, group-aligned median, ties by position).  One thread per leaf.
constexpr int KD_LEAF = 64;
__global__ void k_kd_leaf(const float4 *__restrict__ Y, int nq, int G, int *__restrict__ qord) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int s0 = l * KD_LEAF;
    if (s0 >= nq) return;
    const int n = nq - s0 < KD_LEAF ? nq - s0 : KD_LEAF;
    int idx[KD_LEAF];
    for (int i = 0; i < n; ++i) idx[i] = qord[s0 + i];
    int ns_[KD_LEAF], nz_[KD_LEAF], nn = 1;     // nodes of the current level
    ns_[0] = 0;
    nz_[0] = n;
    bool more = n > G;
    while (more) {
        int ts[KD_LEAF], tz[KD_LEAF], m = 0;
        more = false;
        for (int k = 0; k < nn; ++k) {
            const int a = ns_[k], z = nz_[k];
            if (z <= G) {
                ts[m] = a;
                tz[m++] = z;
                continue;
            }
            float lo[PD_P], hi[PD_P];
            for (int j = 0; j < PD_P; ++j) lo[j] = hi[j] = pd_comp(Y[idx[a]], j);
            for (int i = a + 1; i < a + z; ++i) {
                const float4 y = Y[idx[i]];
                for (int j = 0; j < PD_P; ++j) {
                    lo[j] = fminf(lo[j], pd_comp(y, j));
                    hi[j] = fmaxf(hi[j], pd_comp(y, j));
                }
            }
            int d = 0;
            for (int j = 1; j < PD_P; ++j)
                if (hi[j] - lo[j] > hi[d] - lo[d]) d = j;
            for (int i = a + 1; i < a + z; ++i) {       // stable insertion sort by coordinate d
                const int v = idx[i];
                const unsigned kv = pd_key(pd_comp(Y[v], d));
                int t = i - 1;
                while (t >= a && pd_key(pd_comp(Y[idx[t]], d)) > kv) {
                    idx[t + 1] = idx[t];
                    --t;
                }
                idx[t + 1] = v;
            }
            const int h = (z / 2 + G - 1) / G * G;
            ts[m] = a;
            tz[m++] = h;
            ts[m] = a + h;
            tz[m++] = z - h;
            more |= h > G || z - h > G;
        }
        for (int k = 0; k < m; ++k) {
            ns_[k] = ts[k];
            nz_[k] = tz[k];
        }
        nn = m;
    }
    for (int i = 0; i < n; ++i) qord[s0 + i] = idx[i];
}

}  // namespace

// The k-d order of a batch's queries for groups of G (qord), from their rows
// Qr [nq][Dp] (see the k-d partition above).  Scratch: V [Dp] float4,
// mu [Dp], part [PD_CH][Dp] float4, Y [max(nq, PD_NS)] float4 (the sizes
// crisp_query_order_scratch gives).
size_t crisp_query_order_scratch(int nq, int Dp) {
    auto r = [](size_t b) { return (b + 255) / 256 * 256; };
    return r(sizeof(float4) * (size_t)Dp) + r(sizeof(float) * (size_t)Dp) + r(sizeof(float4) * (size_t)PD_CH * Dp) +
           r(sizeof(float4) * (size_t)std::max(nq, PD_NS));
}

crisp_status crisp_run_query_order(const float *Qr, int nq, int Dp, int G, void *scratch, int *qord, cudaStream_t st) {
    if (nq <= 0) return CRISP_OK;
    const int Gt = G < KD_LEAF ? KD_LEAF : G;          // the tree's leaves
    CRISP_REQUIRE(G >= 1 && nq <= CRISP_GROUP_MAXQ && (nq + Gt - 1) / Gt <= KD_MAXN,
                  "query order: at most %d queries", CRISP_GROUP_MAXQ);
    auto r = [](size_t b) { return (b + 255) / 256 * 256; };
    uint8_t *sp = (uint8_t *)scratch;
    float4 *V = (float4 *)sp;
    float *mu = (float *)(sp + r(sizeof(float4) * (size_t)Dp));
    float4 *part = (float4 *)((uint8_t *)mu + r(sizeof(float) * (size_t)Dp));
    float4 *Y = (float4 *)((uint8_t *)part + r(sizeof(float4) * (size_t)PD_CH * Dp));
    const int ns = nq < PD_NS ? nq : PD_NS;
    const dim3 gb((unsigned)((Dp + PD_NT - 1) / PD_NT), PD_CH);
    k_pd_back<<<gb, PD_NT, 0, st>>>(Qr, nq, Dp, ns, nullptr, nullptr, part);
    CRISP_COUNT_LAUNCH();
    k_pd_finish<<<1, 1024, 0, st>>>(part, Dp, ns, 0, mu, V);
    CRISP_COUNT_LAUNCH();
    for (int it = 0; it < PD_IT; ++it) {
        k_pd_proj<<<(unsigned)((ns + 7) / 8), 256, 0, st>>>(Qr, nq, Dp, ns, mu, V, Y);
        CRISP_COUNT_LAUNCH();
        k_pd_back<<<gb, PD_NT, 0, st>>>(Qr, nq, Dp, ns, mu, Y, part);
        CRISP_COUNT_LAUNCH();
        k_pd_finish<<<1, 1024, 0, st>>>(part, Dp, ns, 1, mu, V);
        CRISP_COUNT_LAUNCH();
    }
    k_pd_proj<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(Qr, nq, Dp, nq, mu, V, Y);
    CRISP_COUNT_LAUNCH();
    CRISP_CK(cudaFuncSetAttribute(k_kd_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kd_smem_bytes()));
    k_kd_order<<<1, KD_NT, kd_smem_bytes(), st>>>(Y, nq, Gt, qord);
    CRISP_COUNT_LAUNCH();
    if (G < KD_LEAF) {
        const int nl = (nq + KD_LEAF - 1) / KD_LEAF;
        k_kd_leaf<<<(unsigned)((nl + 127) / 128), 128, 0, st>>>(Y, nq, G, qord);
        CRISP_COUNT_LAUNCH();
    }
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

namespace {

struct TileMeta {
    int g;                          // query group of the tile
    int count;                      // rows in use (< 0: no more tiles)
    int rid[TR_ROWS];               // per row: row id (rows past count repeat row 0)
    unsigned long long mask[TR_ROWS][TGW];   // per row: members that need it
    int pb[TR_ROWS];                // per row: first pair slot
    int off[TR_ROWS];               // per row: its first pair in spos
    float nx[TR_ROWS];              // per row: |x|^2
    int spos[TR_PMAX];              // list positions of the tile's first TR_PMAX pairs, rows in order
    int gq[TG];                     // per member: query number (-1 past nq)
    float gn2[TG], gn1[TG];         // per member: |q|^2, |q|
};

struct TrArgs {
    int nk;                         // 128-byte k-blocks per row (Dp / 32 FP32, ceil(Dp / 64) BF16)
    int Dp, ngroups, R;
    int bf16;                       // 1: BF16 rows and queries (kind::f16), 0: FP32 rows (kind::tf32)
    int row_bytes;                  // bytes of a stored row (Dp x 4 or Dp x 2)
    long long items;                // ngroups * ceil(R / TR_RB)
    long long stride;               // candidate list stride of ub / lb
    const uint8_t *X;               // [N][Dp] rows scored: the FP32 rows or their BF16 copy
    const int *gq;
    const float *gn2, *gn1;         // per group slot: |q|^2, |q|
    const int *ent_row;
    const unsigned long long *ent_mask;
    const int *ent_pb;
    const float *ent_nx;
    const int *pair_pos;
    const int2 *items_arr;          // [ngroups][R]
    unsigned long long *counter;    // work-item counter
    float *ub, *lb;                 // [nq][stride] upper / lower bound of each pair's CR32 distance
    float c1, c2, c3, c4, gam;      // error-bound constants (file comment)
};

constexpr int TR_MAXSEG = TR_RB;    // a tile holds consecutive entries of at most TR_RB ranges
constexpr int TR_NBAR = 3 * TR_NS + 4 * TR_NB + 1;
__host__ __device__ constexpr size_t tr_smem_bytes() {
    return 1024 + (size_t)TR_NS * TR_STAGE + sizeof(TileMeta) * TR_NB + sizeof(int) * 4 * TR_MAXSEG +
           sizeof(uint64_t) * TR_NBAR + 32;
}
static_assert(tr_smem_bytes() <= 227 * 1024, "the stages and tile buffers must fit one CTA's shared memory");

// 16 bytes, of which the first n (0 or 16) come from src and the rest are zeros.
__device__ __forceinline__ void cp_async16_n(uint32_t dst, const void *src, uint32_t n) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

// Arrive on the mbarrier once every cp.async this thread has issued so far has
// landed (the barrier's count includes this arrival).
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Persistent: one CTA per SM (its shared memory fills the SM, so its 512
// tensor-memory columns are always free).  Work items are (block of TR_RB id
// ranges, group), range-block-major, so the CTAs in flight fetch rows of the
// same ranges for different groups and most fetches hit L2.  Roles:
//  - tile preparation (warp 12): cuts each item's rows into tiles of up to 256
//    and stages every tile's per-row data and the list positions of its pairs
//    (consecutive union entries own consecutive pair slots, so a tile's
//    positions are at most TR_MAXSEG contiguous runs), up to TR_NB tiles ahead;
//  - copies (warps 8-11): the tile's 256 rows, TR_KB 32-float k-blocks a
//    stage, with 16-byte cp.async (thread t moves chunk t & 7 of rows t / 8 +
//    16 i; the 128-byte swizzled layout puts chunk c of row r at c ^ (r & 7)),
//    and the group's 64 query rows by one TMA tile load per k-block;
//  - MMA issue (warp 13, one thread): per k-block 2 x 4 MMAs (M = 128, N = 64,
//    K = 8) into the tile's two accumulators;
//  - epilogue (warps 0-7, a TMEM lane quarter and one of the two accumulators
//    each): per row and member pair the bounds of the CR32 distance, written to
//    the member's list slot.
__global__ void __launch_bounds__(TR_NT, 1) k_rerank_tc(const __grid_constant__ CUtensorMap tmQ, TrArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);   // swizzled tiles need 1024-byte alignment
    uint8_t *stages = sm;
    TileMeta *meta = reinterpret_cast<TileMeta *>(sm + (size_t)TR_NS * TR_STAGE);
    int *sseg = reinterpret_cast<int *>(meta + TR_NB);      // preparation scratch: (first row, rows, first entry) per segment
    uint64_t *bars = reinterpret_cast<uint64_t *>(sseg + 4 * TR_MAXSEG);
    const uint32_t full0 = smem_addr(bars), qfull0 = full0 + 8u * TR_NS, empty0 = qfull0 + 8u * TR_NS,
                   mfull0 = empty0 + 8u * TR_NS, mempty0 = mfull0 + 8u * TR_NB, afull0 = mempty0 + 8u * TR_NB,
                   aempty0 = afull0 + 8u * TR_NB, done = aempty0 + 8u * TR_NB;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + TR_NBAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < TR_NS; ++i) {
            mbar_init(full0 + 8u * i, TR_LT);   // one cp.async arrival per copy thread
            mbar_init(qfull0 + 8u * i, 1);      // the query tile (TMA, counted in bytes)
            mbar_init(empty0 + 8u * i, 1);      // the stage's MMAs have completed
        }
        for (int i = 0; i < TR_NB; ++i) {
            mbar_init(mfull0 + 8u * i, 1);      // a tile's per-row data is staged
            mbar_init(mempty0 + 8u * i, 8);     // the eight epilogue warps are done with it
            mbar_init(afull0 + 8u * i, 1);      // the tile's MMAs have completed
            mbar_init(aempty0 + 8u * i, 8);     // the epilogue warps have read the accumulators
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == TR_WM) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(4 * 128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    long long issued = 0;           // copy threads: k-blocks issued

    // lane 0 waits, the warp follows its verdict (warp-uniform control flow)
    auto warp_wait = [&](uint32_t bar, uint32_t parity, unsigned site) -> bool {
        int ok = 1;
        if (lane == 0) {
            ok = mbar_wait(bar, parity) ? 1 : 0;
            if (!ok) {
                tr_error(site);
                *abort_flag = 1;
            }
        }
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    if (warp == TR_WP) {
        // ---------------------------------------------------- tile preparation
        int t = 0, b = 0, fill = 0, nseg = 0;
        auto emit = [&](int g) -> bool {
            if (t >= TR_NB && !warp_wait(mempty0 + 8u * b, (uint32_t)((t / TR_NB) - 1) & 1u, 0)) return false;
            TileMeta &mt = meta[b];
            const int count = fill;
            // the tile's rows are consecutive union entries, segment by segment, so
            // their data are contiguous runs of the entry arrays: fetched with
            // asynchronous copies, one wait for all of them
            for (int sg = 0; sg < nseg; ++sg) {
                const int r0 = sseg[3 * sg], n = sseg[3 * sg + 1], e0 = sseg[3 * sg + 2];
                for (int i = lane; i < n; i += 32) {
                    cp_async4(smem_addr(&mt.rid[r0 + i]), a.ent_row + e0 + i);
#pragma unroll
                    for (int w = 0; w < TGW; ++w)
                        cp_async8(smem_addr(&mt.mask[r0 + i][w]), a.ent_mask + (long long)(e0 + i) * TGW + w);
                    cp_async4(smem_addr(&mt.pb[r0 + i]), a.ent_pb + e0 + i);
                    cp_async4(smem_addr(&mt.nx[r0 + i]), a.ent_nx + e0 + i);
                }
            }
            for (int j = lane; j < TG; j += 32) {
                cp_async4(smem_addr(&mt.gq[j]), a.gq + g * TG + j);
                cp_async4(smem_addr(&mt.gn2[j]), a.gn2 + g * TG + j);
                cp_async4(smem_addr(&mt.gn1[j]), a.gn1 + g * TG + j);
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            for (int r = count + lane; r < TR_ROWS; r += 32) mt.rid[r] = mt.rid[0];   // padding rows repeat row 0
            // pairs: each segment's slots are one contiguous run starting at the
            // pair base of its first row
            int base = 0;
            for (int sg = 0; sg < nseg; ++sg) {
                const int r0 = sseg[3 * sg], n = sseg[3 * sg + 1];
                int lastc = 0;
#pragma unroll
                for (int w = 0; w < TGW; ++w) lastc += __popcll(mt.mask[r0 + n - 1][w]);
                const int pb0 = mt.pb[r0], len = mt.pb[r0 + n - 1] + lastc - pb0;
                for (int r = r0 + lane; r < r0 + n; r += 32) mt.off[r] = base + mt.pb[r] - pb0;
                const int lim = base + len < TR_PMAX ? len : TR_PMAX - base;
                for (int p = lane; p < lim; p += 32) cp_async4(smem_addr(&mt.spos[base + p]), a.pair_pos + pb0 + p);
                base += len;
                if (base > TR_PMAX) base = TR_PMAX + 1;   // the rest read their positions from global memory
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            if (lane == 0) {
                mt.g = g;
                mt.count = count;
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) mbar_arrive(mfull0 + 8u * b);
            ++t;
            b = t % TR_NB;
            fill = 0;
            nseg = 0;
            return true;
        };
        bool ok = true;
        for (;;) {
            unsigned long long it = 0;
            if (lane == 0) it = atomicAdd(a.counter, 1ull);
            it = __shfl_sync(0xffffffffu, it, 0);
            if ((long long)it >= a.items || __shfl_sync(0xffffffffu, *abort_flag, 0)) break;
            const int g = (int)(it % (unsigned long long)a.ngroups), rb = (int)(it / (unsigned long long)a.ngroups);
            const int r_end = (rb + 1) * TR_RB < a.R ? (rb + 1) * TR_RB : a.R;
            for (int r = rb * TR_RB; r < r_end && ok; ++r) {
                const int2 itm = a.items_arr[(long long)g * a.R + r];
                for (int got = 0; got < itm.y;) {
                    const int take = TR_ROWS - fill < itm.y - got ? TR_ROWS - fill : itm.y - got;
                    if (lane == 0) {
                        sseg[3 * nseg] = fill;
                        sseg[3 * nseg + 1] = take;
                        sseg[3 * nseg + 2] = itm.x + got;
                    }
                    ++nseg;
                    fill += take;
                    got += take;
                    __syncwarp();
                    if (fill == TR_ROWS && !(ok = emit(g))) break;
                }
            }
            if (!ok) break;
            if (fill > 0 && !(ok = emit(g))) break;
        }
        // no more tiles (after an abort the other roles stop by themselves)
        if (ok && !__shfl_sync(0xffffffffu, *abort_flag, 0) &&
            (t < TR_NB || warp_wait(mempty0 + 8u * b, (uint32_t)((t / TR_NB) - 1) & 1u, 0))) {
            if (lane == 0) {
                meta[b].count = -1;
                __threadfence_block();
                mbar_arrive(mfull0 + 8u * b);
            }
        }
    } else if (warp >= TR_WC && warp < TR_WC + TR_LT / 32) {
        // -------------------------------------------------------------- copies
        // each copy warp waits by itself (lane 0 polls, the warp follows); the
        // stage completes once all 128 copy threads' copies have landed
        const int lt = threadIdx.x - 32 * TR_WC;
        const int c = lt & 7, r0 = lt >> 3;
        const uint32_t swz = (uint32_t)((c ^ (r0 & 7)) << 4);
        const int nst = (a.nk + TR_KB - 1) / TR_KB;      // stages per tile
        for (int t = 0;; ++t) {
            const int b = t % TR_NB;
            if (!warp_wait(mfull0 + 8u * b, (uint32_t)(t / TR_NB) & 1u, 1)) break;
            const TileMeta &mt = meta[b];
            if (mt.count < 0) break;
            const int g = mt.g;
            int id[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) id[i] = mt.rid[r0 + 16 * i];
            bool ok = true;
            for (int si = 0; si < nst; ++si, ++issued) {
                const int s = (int)(issued % TR_NS);
                if (issued >= TR_NS && !warp_wait(empty0 + 8u * s, (uint32_t)((issued / TR_NS) - 1) & 1u, 2)) {
                    ok = false;
                    break;
                }
                const int k0 = si * TR_KB, nkb = a.nk - k0 < TR_KB ? a.nk - k0 : TR_KB;
                const uint32_t sa = smem_addr(stages + (size_t)s * TR_STAGE), sq = sa + TR_KB * 2 * TR_A_BYTES;
                if (lt == 0) {
                    mbar_expect_tx(qfull0 + 8u * s, (uint32_t)nkb * TR_B_BYTES);
                    for (int kb = 0; kb < nkb; ++kb)
                        tma_load_2d(sq + (uint32_t)kb * TR_B_BYTES, &tmQ, (a.bf16 ? 64 : 32) * (k0 + kb), TG * g,
                                    qfull0 + 8u * s);
                }
                for (int kb = 0; kb < nkb; ++kb) {
                    // chunk c of the k-block: bytes 128 (k0 + kb) + 16 c of the row; a BF16
                    // row of Dp = 64 j + 32 ends halfway through its last k-block (zeros after)
                    const int cb = 128 * (k0 + kb) + 16 * c;
                    const uint32_t n = cb < a.row_bytes ? 16u : 0u;
                    const uint8_t *col = a.X + (n ? cb : 0);      // an empty copy still names its own row
                    const uint32_t da = sa + (uint32_t)kb * 2 * TR_A_BYTES + swz;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        cp_async16_n(da + (uint32_t)((r0 + 16 * i) * 128), col + (long long)id[i] * a.row_bytes, n);
                }
                cp_async_arrive(full0 + 8u * s);
            }
            if (!ok) break;
        }
    } else if (warp == TR_WM) {
        // ------------------------------------------------------------- MMA issue
        if (lane == 0) {
            const bool bf = a.bf16 != 0;
            const uint32_t idesc = bf ? bf16_idesc(TG, 128) : tf32_idesc(TG, 128);
            long long c = 0;
            for (int t = 0;; ++t) {
                const int b = t % TR_NB;
                if (!mbar_wait(mfull0 + 8u * b, (uint32_t)(t / TR_NB) & 1u)) {
                    tr_error(3);
                    *abort_flag = 1;
                    break;
                }
                if (meta[b].count < 0 || *abort_flag) break;
                if (t >= TR_NB && !mbar_wait(aempty0 + 8u * b, (uint32_t)((t / TR_NB) - 1) & 1u)) {
                    tr_error(4);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + (uint32_t)(2 * TG) * b, d1 = d0 + (uint32_t)TG;
                bool bad = false;
                const int nst = (a.nk + TR_KB - 1) / TR_KB;
                for (int si = 0; si < nst; ++si, ++c) {
                    const int s = (int)(c % TR_NS);
                    const uint32_t ph = (uint32_t)(c / TR_NS) & 1u;
                    if (!mbar_wait(full0 + 8u * s, ph) || !mbar_wait(qfull0 + 8u * s, ph)) {
                        bad = true;
                        break;
                    }
                    // the rows were written through the generic proxy (cp.async); the MMA reads them
                    // through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc_fence_after();
                    const int k0 = si * TR_KB, nkb = a.nk - k0 < TR_KB ? a.nk - k0 : TR_KB;
                    const uint32_t sa0 = smem_addr(stages + (size_t)s * TR_STAGE), sq0 = sa0 + TR_KB * 2 * TR_A_BYTES;
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint32_t sa = sa0 + (uint32_t)kb * 2 * TR_A_BYTES, sq = sq0 + (uint32_t)kb * TR_B_BYTES;
                        if (bf) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {   // UMMA K = 16 BF16 = 32 bytes
                                const uint32_t o = 32u * j, acc = (k0 + kb + j) != 0;
                                mma_bf16(d0, sw128_desc(sa + o), sw128_desc(sq + o), idesc, acc);
                                mma_bf16(d1, sw128_desc(sa + TR_A_BYTES + o), sw128_desc(sq + o), idesc, acc);
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {   // UMMA K = 8 floats = 32 bytes
                                const uint32_t o = 32u * j, acc = (k0 + kb + j) != 0;
                                mma_tf32(d0, sw128_desc(sa + o), sw128_desc(sq + o), idesc, acc);
                                mma_tf32(d1, sw128_desc(sa + TR_A_BYTES + o), sw128_desc(sq + o), idesc, acc);
                            }
                        }
                    }
                    mma_commit(empty0 + 8u * s);
                }
                if (bad) {
                    tr_error(5);
                    *abort_flag = 1;
                    break;
                }
                mma_commit(afull0 + 8u * b);
            }
            mma_commit(done);       // completes once every MMA issued above has
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        // warps w and w + 4 read TMEM lane quarter w & 3; warp w < 4 takes the
        // tile's first accumulator (rows 0-127), w >= 4 the second
        const int qd = warp & 3, h = warp >> 2;
        for (int t = 0;; ++t) {
            const int b = t % TR_NB;
            if (!warp_wait(mfull0 + 8u * b, (uint32_t)(t / TR_NB) & 1u, 6)) break;
            const TileMeta &mt = meta[b];
            const int count = mt.count;
            if (count < 0) break;
            if (!warp_wait(afull0 + 8u * b, (uint32_t)(t / TR_NB) & 1u, 7)) break;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(2 * TG) * b + (uint32_t)TG * h;
            const int row = 32 * qd + lane + 128 * h;
            const bool valid = row < count;
            unsigned long long mw[TGW];
#pragma unroll
            for (int w = 0; w < TGW; ++w) mw[w] = valid ? mt.mask[row][w] : 0ull;
            const int pb = valid ? mt.pb[row] : 0, po = valid ? mt.off[row] : 0;
            const float nx = valid ? mt.nx[row] : 0.0f, rx = sqrtf(nx), c1rx = a.c1 * rx;
#pragma unroll 1
            for (int cb = 0; cb < TG / 16; ++cb) {
                uint32_t v[16];
                tmem_ld16(ta + 16u * cb, v);               // warp-collective: every lane takes part
                const unsigned long long m = mw[cb >> 2];                  // the word holding members 16 cb ..
                const int sh = 16 * (cb & 3);
                const unsigned sub = (unsigned)(m >> sh) & 0xFFFFu;
                int rank0 = __popcll(m & ((1ull << sh) - 1ull));
                if (TGW > 1 && cb >= 4) rank0 += __popcll(mw[0]);
                int pos[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {          // list positions for members 16 cb + jj
                    const int rk = rank0 + __popc(sub & ((1u << jj) - 1u));
                    pos[jj] = !((sub >> jj) & 1u) ? 0 : po + rk < TR_PMAX ? mt.spos[po + rk] : a.pair_pos[pb + rk];
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    if ((sub >> jj) & 1u) {
                        const int j = 16 * cb + jj;
                        const float ss = nx + mt.gn2[j];
                        const float dt = ss - 2.0f * __uint_as_float(v[jj]);
                        const float E = mt.gn1[j] * c1rx + a.c2 * ss + (a.c3 * (rx + mt.gn1[j]) + a.c4);
                        const float E2 = E + a.gam * (fabsf(dt) + E);
                        const long long at = (long long)mt.gq[j] * a.stride + pos[jj];
                        a.ub[at] = fmaxf(dt + E2, 0.0f);
                        a.lb[at] = dt - E2;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(aempty0 + 8u * b);
                mbar_arrive(mempty0 + 8u * b);
            }
        }
    }

    // ---------------------------------------------------------------- teardown
    if (warp == TR_WM && lane == 0 && !mbar_wait(done, 0)) tr_error(8);
    if (warp >= TR_WC && warp < TR_WC + TR_LT / 32) {
        // every copy still in flight lands before the CTA's shared memory goes away
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (threadIdx.x == 32 * TR_WC)
            for (long long c = issued - TR_NS < 0 ? 0 : issued - TR_NS; c < issued; ++c)
                if (!mbar_wait(qfull0 + 8u * (c % TR_NS), (uint32_t)(c / TR_NS) & 1u)) tr_error(9);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == TR_WM) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * 128) : "memory");
    }
}

// Profiling records (crisp_rerank_profile_*): events around each scoring
// launch and a pinned copy of its work counters.
struct ProfRec {
    cudaEvent_t a = nullptr, b = nullptr;
    unsigned long long *host = nullptr;   // pinned [2]: entries, pairs
    int Dp = 0;
    int elem_bytes = 4;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;

}  // namespace

extern "C" crisp_status crisp_query_order(const float *Qr, int32_t nq, int32_t Dp, int32_t G, int32_t *qord,
                                          void *stream) {
    CRISP_REQUIRE(nq >= 0 && Dp >= 1 && G >= 1, "crisp_query_order: nq = %d, Dp = %d, G = %d", nq, Dp, G);
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Qr && qord, "crisp_query_order: null pointer");
    const int Gt = G < KD_LEAF ? KD_LEAF : G;
    CRISP_REQUIRE(nq <= CRISP_GROUP_MAXQ && (nq + Gt - 1) / Gt <= KD_MAXN,
                  "crisp_query_order: at most %d queries and %d groups of max(G, 64)", CRISP_GROUP_MAXQ, KD_MAXN);
    cudaStream_t st = (cudaStream_t)stream;
    void *buf = nullptr;
    CRISP_CK(crisp_scratch_alloc(&buf, crisp_query_order_scratch(nq, Dp), st));
    const crisp_status s = crisp_run_query_order(Qr, nq, Dp, G, buf, qord, st);
    crisp_scratch_free(buf, st);
    return s;
}

extern "C" crisp_status crisp_rerank_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return CRISP_OK;
}

extern "C" crisp_status crisp_rerank_profile_read(crisp_rerank_profile *out) {
    CRISP_REQUIRE(out, "crisp_rerank_profile_read: null output");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    crisp_rerank_profile r = {};
    r.group = TG;
    crisp_status s = CRISP_OK;
    for (ProfRec &p : g_prof_recs) {
        cudaError_t e = cudaEventSynchronize(p.b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess && s == CRISP_OK) s = crisp_cuda_fail(e, "crisp_rerank_profile_read", __FILE__, __LINE__);
        r.launches += 1;
        r.ms += ms;
        r.rows += (int64_t)p.host[0];
        r.pairs += (int64_t)p.host[1];
        r.Dp = p.Dp;
        r.elem_bytes = p.elem_bytes;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
        cudaFreeHost(p.host);
    }
    g_prof_recs.clear();
    *out = r;
    return s;
}

// What a tensor-core batch computes after its bounds: the exact FP32 top-k
// (ids, d2: [nq][ko]), or the shortlist of the S smallest BF16 coarse scores
// (out: [nq][out_stride], nout) for the coarse-scoring and learned paths.
struct TcTask {
    bool coarse;
    int32_t k;                      // exact: k; coarse: S (per query: S_per_query, else qp S)
    const int64_t *S_per_query;
    const QParam *qp;
    int32_t ko;
    int64_t *ids;
    float *d2;
    int32_t *out;
    int64_t out_stride;
    int64_t *nout;
};

// One batch of TR_MINQ to CRISP_GROUP_MAXQ queries whose pairs fit 32-bit
// slots.  dbuf: [nq][stride] floats of scratch.
static crisp_status rerank_tc_batch(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                    int64_t stride, const int64_t *ncand, const TcTask &task, float *dbuf,
                                    cudaStream_t st);

// Batches of TR_MINQ to CRISP_GROUP_MAXQ queries whose candidate lists may hold
// 2,048 or more ids; *done = false (nothing run) for other batches, which the
// caller streams.
static crisp_status run_tc(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand, int64_t stride,
                           const int64_t *ncand, const TcTask &task, float *dbuf, cudaStream_t st, bool *done) {
    *done = false;
    if (nq < TR_MINQ || nq > CRISP_GROUP_MAXQ || stride < 2048) return CRISP_OK;
    // pair slots are 32-bit: batches whose lists could hold more pairs run in
    // equal sub-batches (the kernels have no minimum batch size)
    const long long per_q = std::min<int64_t>(stride, ix->N);
    const long long sub = 0x7FFFFFFFLL / per_q;
    if (sub < 512) return CRISP_OK;
    const int32_t nb = (int32_t)((nq + sub - 1) / sub), each = (nq + nb - 1) / nb;
    for (int32_t q0 = 0; q0 < nq; q0 += each) {
        const int32_t n = std::min(each, nq - q0);
        TcTask t = task;
        if (t.qp) t.qp += q0;
        if (t.S_per_query) t.S_per_query += q0;
        if (t.coarse) {
            t.out += (int64_t)q0 * t.out_stride;
            t.nout += q0;
        } else {
            t.ids += (int64_t)q0 * t.ko;
            t.d2 += (int64_t)q0 * t.ko;
        }
        crisp_status s = rerank_tc_batch(ix, Qr + (int64_t)q0 * ix->Dp, n, cand + (int64_t)q0 * stride, stride,
                                         ncand + q0, t, dbuf + (int64_t)q0 * stride, st);
        if (s) return s;
    }
    *done = true;
    return CRISP_OK;
}

crisp_status crisp_run_rerank_tc(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                 int64_t stride, const int64_t *ncand, int32_t k, const QParam *qp, int32_t ko,
                                 float *dbuf, int64_t *ids, float *d2, cudaStream_t st, bool *done) {
    TcTask t{false, k, nullptr, qp, ko, ids, d2, nullptr, 0, nullptr};
    return run_tc(ix, Qr, nq, cand, stride, ncand, t, dbuf, st, done);
}

// The BF16 coarse-score shortlist (precision 1, learned depths) of large
// batches: one BF16 pass bounds every pair's coarse score (the CR32 distance
// of the FP32 query to the widened BF16 row), the candidates whose lower bound
// reaches the S-th smallest upper bound are scored exactly, and the S best by
// (score, id) are kept, in ascending id.
crisp_status crisp_run_shortlist_tc(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                    int64_t stride, const int64_t *ncand, int32_t S, const int64_t *S_per_query,
                                    const QParam *qp, float *dbuf, int32_t *out, int64_t out_stride, int64_t *nout,
                                    cudaStream_t st, bool *done) {
    *done = false;
    if (!ix->Xb || !ix->xbn2) return CRISP_OK;
    TcTask t{true, S, S_per_query, qp, 0, nullptr, nullptr, out, out_stride, nout};
    return run_tc(ix, Qr, nq, cand, stride, ncand, t, dbuf, st, done);
}

static crisp_status rerank_tc_batch(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                    int64_t stride, const int64_t *ncand, const TcTask &task, float *dbuf,
                                    cudaStream_t st) {
    const int Dp = ix->Dp;
    const int R = (int)((ix->N + TSPAN - 1) / TSPAN);
    const int ngroups = (nq + TG - 1) / TG, nslots = ngroups * TG;
    const long long pcap = (long long)nq * std::min<int64_t>(stride, ix->N);
    const long long ecap = std::min<long long>(pcap, (long long)ngroups * R * TSPAN);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    // the BF16 copy, when the index keeps one, halves the bytes of every row fetch
    // (CRISP_RERANK_TF32=1 keeps the FP32 rows)
    const char *force_tf32 = getenv("CRISP_RERANK_TF32");
    const bool bf = task.coarse || (ix->Xb != nullptr && !(force_tf32 && atoi(force_tf32) != 0));
    const int Dp64 = (Dp + 63) / 64 * 64;
    const size_t o_cnt = take(4 * sizeof(unsigned long long)), o_qord = take(sizeof(int) * nq), o_pos = take(sizeof(int) * (size_t)nq * (R + 1)),
                 o_ord = take(crisp_query_order_scratch(nq, Dp)),
                 o_gq = take(sizeof(int) * nslots), o_gn2 = take(sizeof(float) * nslots),
                 o_gn1 = take(sizeof(float) * nslots), o_qg = take(sizeof(float) * (size_t)nslots * Dp),
                 o_qgb = take(bf ? sizeof(uint16_t) * (size_t)nslots * Dp64 : 0),
                 o_items = take(sizeof(int2) * (size_t)ngroups * R), o_row = take(sizeof(int) * (size_t)ecap),
                 o_mask = take(sizeof(unsigned long long) * TGW * (size_t)ecap), o_pb = take(sizeof(int) * (size_t)ecap),
                 o_enx = take(sizeof(float) * (size_t)ecap),
                 o_pp = take(sizeof(int) * (size_t)pcap), o_ub = take(sizeof(float) * (size_t)nq * stride),
                 o_lb = take(sizeof(float) * (size_t)nq * stride),
                 o_rc = take(sizeof(int) * (size_t)nq * stride), o_nr = take(sizeof(int64_t) * nq);
    uint8_t *buf = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&buf, off, st));
    unsigned long long *counts = (unsigned long long *)(buf + o_cnt);
    int *qord = (int *)(buf + o_qord), *pos = (int *)(buf + o_pos), *gq = (int *)(buf + o_gq);
    float *gn2 = (float *)(buf + o_gn2), *gn1 = (float *)(buf + o_gn1), *Qg = (float *)(buf + o_qg);
    uint16_t *Qgb = bf ? (uint16_t *)(buf + o_qgb) : nullptr;
    float *ub = (float *)(buf + o_ub), *lb = (float *)(buf + o_lb);
    int32_t *rc = (int32_t *)(buf + o_rc);
    int64_t *nr = (int64_t *)(buf + o_nr);
    TUnion u;
    u.gq = gq;
    u.pos = pos;
    u.ent_row = (int *)(buf + o_row);
    u.ent_mask = (unsigned long long *)(buf + o_mask);
    u.ent_pb = (int *)(buf + o_pb);
    u.ent_nx = (float *)(buf + o_enx);
    u.xn2 = task.coarse ? ix->xbn2 : ix->xn2;   // |x|^2 of the rows the exact value is measured on
    u.pair_pos = (int *)(buf + o_pp);
    u.items = (int2 *)(buf + o_items);
    u.counts = counts;
    u.ecap = ecap;
    u.pcap = pcap;
    u.R = R;
    crisp_status s = CRISP_OK;
    do {
        cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__); break; }
        unsigned *err_word = nullptr;
        e = cudaGetSymbolAddress((void **)&err_word, g_tr_error);
        if (e == cudaSuccess) e = cudaMemsetAsync(err_word, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "error word", __FILE__, __LINE__); break; }
        s = crisp_run_query_order(Qr, nq, Dp, TG, buf + o_ord, qord, st);
        if (s) break;
        s = crisp_run_group_pos(cand, stride, ncand, nq, R, pos, st);
        if (s) break;
        k_group_queries<<<(nslots + 7) / 8, 256, 0, st>>>(Qr, nq, Dp, qord, nslots, Qg, Qgb, Dp64, gq, gn2, gn1);
        CRISP_COUNT_LAUNCH();
        const size_t usmem = sizeof(unsigned long long) * TSPAN * TGW + sizeof(int) * TSPAN;
        e = cudaFuncSetAttribute(k_union, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__); break; }
        k_union<<<dim3(R, ngroups), TU_NT, usmem, st>>>(cand, (long long)stride, u);
        CRISP_COUNT_LAUNCH();
        CUtensorMap mq;
        if (bf ? !crisp_make_map_bf16(&mq, Qgb, nslots, Dp64, Dp64, TG) : !crisp_make_map_f32(&mq, Qg, nslots, Dp, Dp, TG)) {
            crisp_set_error("tensor-core re-rank: tensor map encoding failed");
            s = CRISP_ECUDA;
            break;
        }
        TrArgs ta;
        ta.nk = bf ? Dp64 / 64 : Dp / 32;
        ta.Dp = Dp;
        ta.bf16 = bf ? 1 : 0;
        ta.row_bytes = Dp * (bf ? 2 : 4);
        ta.X = bf ? (const uint8_t *)ix->Xb : (const uint8_t *)ix->Xr;
        ta.ngroups = ngroups;
        ta.R = R;
        ta.items = (long long)ngroups * ((R + TR_RB - 1) / TR_RB);
        ta.stride = stride;
        ta.gq = gq;
        ta.gn2 = gn2;
        ta.gn1 = gn1;
        ta.ent_row = u.ent_row;
        ta.ent_mask = u.ent_mask;
        ta.ent_pb = u.ent_pb;
        ta.ent_nx = u.ent_nx;
        ta.pair_pos = u.pair_pos;
        ta.items_arr = u.items;
        ta.counter = counts + 2;
        ta.ub = ub;
        ta.lb = lb;
        const int K = bf ? 16 : 8;
        const double eps_acc = (double)(Dp / K + 1) * (K + 1) * std::ldexp(1.0, -22);
        // coarse scores are of the BF16 rows themselves: only the query is rounded
        const double eps_mul = task.coarse ? std::ldexp(1.0, -9) + std::ldexp(1.0, -18)
                               : bf        ? std::ldexp(1.0, -8) + std::ldexp(1.0, -18)
                                           : std::ldexp(1.0, -9) + std::ldexp(1.0, -20);
        ta.c1 = (float)(2.0 * (eps_mul + eps_acc) * 1.01);
        ta.c2 = (float)std::ldexp(1.0, -19);
        ta.c3 = (float)std::ldexp(1.0, -110);
        ta.c4 = (float)std::ldexp(1.0, -100);
        ta.gam = (float)((Dp / 32 + 12) * std::ldexp(1.0, -23) + std::ldexp(1.0, -20));
        const size_t smem = tr_smem_bytes();
        e = cudaFuncSetAttribute(k_rerank_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__); break; }
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ProfRec rec;
        {
            std::lock_guard<std::mutex> lk(g_prof_mu);
            if (g_prof_on) {
                rec.Dp = Dp;
                rec.elem_bytes = bf ? 2 : 4;
                if (cudaEventCreate(&rec.a) != cudaSuccess || cudaEventCreate(&rec.b) != cudaSuccess ||
                    cudaMallocHost((void **)&rec.host, 2 * sizeof(unsigned long long)) != cudaSuccess) {
                    s = crisp_cuda_fail(cudaGetLastError(), "profiling record", __FILE__, __LINE__);
                    break;
                }
                cudaEventRecord(rec.a, st);
            }
        }
        k_rerank_tc<<<sms, TR_NT, smem, st>>>(mq, ta);
        CRISP_COUNT_LAUNCH();
        e = cudaGetLastError();
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_rerank_tc", __FILE__, __LINE__); break; }
        if (rec.a) {
            cudaEventRecord(rec.b, st);
            cudaMemcpyAsync(rec.host, counts, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
            std::lock_guard<std::mutex> lk(g_prof_mu);
            g_prof_recs.push_back(rec);
        }
        s = crisp_run_bound_select(nq, cand, stride, ncand, task.k, task.qp, task.coarse ? 1 : 0, task.S_per_query,
                                   ub, lb, err_word, rc, nr, st);
        if (s) break;
        if (task.coarse)   // the kept candidates' exact coarse scores (streaming) -> the S best
            s = crisp_run_shortlist(ix, Qr, nq, rc, stride, nr, 1, task.k, dbuf, task.out, task.out_stride, task.nout,
                                    st, task.S_per_query, task.qp, false);
        else               // the kept candidates, measured exactly (streaming CR32) -> top-k
            s = crisp_run_rerank(ix, Qr, nq, rc, stride, nr, task.k, dbuf, task.ids, task.d2, st, false, false,
                                 task.qp, task.ko);
    } while (0);
    crisp_scratch_free(buf, st);
    return s;
}
