// Optimized-mode verification (§4.3.2 Stages 2-3, Eq. 2) for sm_103a.
//
// One CTA per query.  The candidates (ascending ids) are ordered by
// (Hamming(b(q), b(x)), id) with a shared-memory bitonic sort of 32-bit keys
// (ham << 15 | list position; positions ascend with ids).  They are then
// verified in chunks of 32, one 8-lane group per candidate: each group walks
// its row 32 dims at a time in the CR32 order, keeping every checkpoint sum
// d_t, and stops early once d_t > fl(r2_start * f_t), r2_start being the k-th
// distance at the start of the chunk.  The sequential walk of the method can
// only hold a smaller or equal k-th distance at any candidate of the chunk, so
// it prunes no later than the group stopped and every value it would read has
// been computed.  Warp 0 then replays the chunk in order, exactly: prune
// decisions for all 32 candidates are evaluated in parallel under the current
// r_k, the first candidate that enters the top-k is found by a ballot, the
// top-k and the patience counter are updated, and the remaining lanes are
// re-evaluated under the new r_k.  The walk ends when the counter reaches P.
#include <float.h>
#include <limits.h>
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int VO_NT = 256;                 // 32 groups of 8 lanes
constexpr int VO_CHUNK = VO_NT / 8;

__device__ __forceinline__ float cr32_block_v(float4 x, float4 qv, unsigned gmask) {
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

struct VoShared {
    float tk_d[CRISP_KOUT_MAX];
    int tk_id[CRISP_KOUT_MAX];
    int tk_n;
    long long counter, processed, nfull;
    int done;
    int stop_b[VO_CHUNK];      // blocks computed by the group (nb = full row)
    unsigned long long nblk;
    float full[VO_CHUNK];
    int cid[VO_CHUNK];
    float r2_start;
};

// Smallest checkpoint b < nb_chk, b < stop with cs[b] > r2 * ft[b]; -1 if none.
__device__ __forceinline__ int first_prune(const float *cs, const float *ft, int nb_chk, int stop, float r2) {
    int lim = stop < nb_chk ? stop : nb_chk;
    for (int b = 0; b < lim; ++b)
        if (cs[b] > r2 * ft[b]) return b;
    return -1;
}

__global__ void __launch_bounds__(VO_NT) k_verify_opt(IxView ix, const float *__restrict__ Qr, int nq,
                                                      const int *__restrict__ cand, long long stride,
                                                      const long long *__restrict__ ncand, int kk, float eps0,
                                                      long long patience, int order, const QParam *__restrict__ qp,
                                                      int ko, int cap_keys,
                                                      long long *__restrict__ out_ids, float *__restrict__ out_d,
                                                      long long *__restrict__ out_nver, long long *__restrict__ out_nfull,
                                                      long long *__restrict__ out_nblk) {
    extern __shared__ __align__(16) float smv[];
    __shared__ VoShared S;
    const int q = blockIdx.x, tid = threadIdx.x;
    if (qp) {                           // per-query parameters
        kk = qp[q].k;
        eps0 = qp[q].eps0;
        patience = qp[q].patience;
        order = qp[q].order;
    }
    const int Dp = ix.Dp, nb = Dp / 32, W = Dp / 32, D = ix.D;
    float *qs = smv;                                        // [Dp]
    float *ft = qs + Dp;                                    // [nb]
    uint32_t *qc = reinterpret_cast<uint32_t *>(ft + nb);   // [W]
    float *cs = reinterpret_cast<float *>(qc + W);          // [VO_CHUNK][nb]
    uint32_t *keys = reinterpret_cast<uint32_t *>(cs + VO_CHUNK * nb);   // [cap_keys]
    long long n = ncand[q];
    if (n > stride) n = stride;
    if (n > cap_keys) n = cap_keys;                        // the launcher guarantees n <= cap_keys
    const int *candq = cand + (long long)q * stride;
    // number of checkpoints: t = 32 (b+1) < D
    const int nb_chk = (D - 1) / 32 < nb ? (D - 1) / 32 : nb;

    for (int d = tid; d < Dp; d += VO_NT) qs[d] = Qr[(long long)q * Dp + d];
    for (int b = tid; b < nb; b += VO_NT) {
        int t = 32 * (b + 1);
        double a = 1.0 + (double)eps0 / sqrt((double)t);
        ft[b] = t < D ? (float)(((double)t / (double)D) * (a * a)) : 0.0f;
    }
    __syncthreads();
    for (int w = tid; w < W; w += VO_NT) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) v |= (qs[32 * w + b] > 0.0f ? 1u : 0u) << b;
        qc[w] = v;
    }
    if (tid == 0) {
        S.tk_n = 0; S.counter = 0; S.processed = 0; S.nfull = 0; S.done = 0; S.nblk = 0;
    }
    __syncthreads();

    // Stage 2: Hamming distances, key = ham << 15 | position
    const int lane = tid & 31, g = tid >> 3, l = tid & 7;
    const unsigned gmask = 0xFFu << (lane & 24);
    int npow = 1;
    while (npow < n) npow <<= 1;
    for (long long i0 = 0; i0 < n; i0 += VO_CHUNK) {
        long long i = i0 + g;
        if (i < n) {
            const uint32_t *row = ix.codes + (long long)candq[i] * W;
            int h = 0;
            for (int w = l; w < W; w += 8) h += __popc(__ldg(row + w) ^ qc[w]);
            h += __shfl_xor_sync(gmask, h, 4);
            h += __shfl_xor_sync(gmask, h, 2);
            h += __shfl_xor_sync(gmask, h, 1);
            if (l == 0) keys[i] = ((uint32_t)(order ? 0 : h) << 15) | (uint32_t)i;   // order 1: ids only
        }
    }
    for (long long i = n + tid; i < npow; i += VO_NT) keys[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (int size = 2; size <= npow; size <<= 1) {
        for (int sd = size >> 1; sd > 0; sd >>= 1) {
            for (int i = tid; i < npow; i += VO_NT) {
                int j = i ^ sd;
                if (j > i) {
                    uint32_t a = keys[i], b = keys[j];
                    bool up = (i & size) == 0;
                    if ((a > b) == up) { keys[i] = b; keys[j] = a; }
                }
            }
            __syncthreads();
        }
    }

    // Stage 3: chunked ADSampling + patience with exact replay
    for (long long pos = 0; pos < n; pos += VO_CHUNK) {
        if (S.done) break;                                  // block-uniform (read after a barrier)
        const int chunk = (int)(n - pos < VO_CHUNK ? n - pos : VO_CHUNK);
        const float r2s = S.tk_n == kk ? S.tk_d[kk - 1] : INFINITY;
        if (g < chunk) {
            int p = (int)(keys[pos + g] & 0x7FFFu);
            int id = candq[p];
            const float4 *row = reinterpret_cast<const float4 *>(ix.Xr + (long long)id * Dp) + l;
            float *csg = cs + g * nb;
            float acc = 0.0f;
            int stop = nb;
            constexpr int U = 4;
            int b_read = 0;
            for (int b0 = 0; b0 < nb && stop == nb; b0 += U) {
                b_read = b0 + U;
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (b0 + u < nb) v[u] = __ldcs(row + 8 * (b0 + u));
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    int b = b0 + u;
                    if (b < nb && stop == nb) {
                        float4 qv = *reinterpret_cast<const float4 *>(qs + 32 * b + 4 * l);
                        acc = acc + cr32_block_v(v[u], qv, gmask);
                        if (l == 0) csg[b] = acc;
                        if (b < nb_chk && acc > r2s * ft[b]) stop = b + 1;
                    }
                }
            }
            if (l == 0) {
                int rd = b_read < nb ? b_read : nb;
                atomicAdd(&S.nblk, (unsigned long long)rd);
                S.stop_b[g] = stop;
                S.full[g] = acc;
                S.cid[g] = id;
            }
        }
        __syncthreads();
        if (tid < 32) {
            // warp 0 replays candidates pos .. pos+chunk-1 in order
            int j0 = 0;
            while (j0 < chunk) {
                const bool full_tk = S.tk_n == kk;
                const float r2 = full_tk ? S.tk_d[kk - 1] : INFINITY;
                const int wid = full_tk ? S.tk_id[kk - 1] : INT_MAX;
                bool ins = false;
                if (lane >= j0 && lane < chunk) {
                    int pb = full_tk ? first_prune(cs + lane * nb, ft, nb_chk, S.stop_b[lane], r2) : -1;
                    if (pb < 0) {
                        float d = S.full[lane];
                        ins = !full_tk || d < r2 || (d == r2 && S.cid[lane] < wid);
                    }
                }
                unsigned bal = __ballot_sync(0xffffffffu, ins);
                int jins = bal ? __ffs(bal) - 1 : chunk;    // first lane that changes the top-k
                // candidates j0 .. jins-1 leave the top-k unchanged
                long long cnt0 = S.counter;
                int stop_at = -1;
                if (patience > 0 && cnt0 + (jins - j0) >= patience) stop_at = j0 + (int)(patience - cnt0) - 1;
                // count full distances among the unchanged ones (not pruned)
                int upto = stop_at >= 0 ? stop_at + 1 : jins;
                bool unpruned = false;
                if (lane >= j0 && lane < upto) {
                    int pb = full_tk ? first_prune(cs + lane * nb, ft, nb_chk, S.stop_b[lane], r2) : -1;
                    unpruned = pb < 0;
                }
                int nf = __popc(__ballot_sync(0xffffffffu, unpruned));
                if (stop_at >= 0) {
                    if (lane == 0) {
                        S.processed += upto - j0;
                        S.nfull += nf;
                        S.counter = cnt0 + (upto - j0);
                        S.done = 1;
                    }
                    __syncwarp();
                    break;
                }
                if (lane == 0) {
                    S.processed += jins - j0;
                    S.nfull += nf;
                    S.counter = cnt0 + (jins - j0);
                }
                __syncwarp();
                if (jins >= chunk) break;
                // candidate jins enters the top-k (full distance computed)
                if (lane == 0) {
                    float d = S.full[jins];
                    int id = S.cid[jins];
                    int p = S.tk_n == kk ? kk - 1 : S.tk_n;
                    while (p > 0 && (S.tk_d[p - 1] > d || (S.tk_d[p - 1] == d && S.tk_id[p - 1] > id))) {
                        S.tk_d[p] = S.tk_d[p - 1];
                        S.tk_id[p] = S.tk_id[p - 1];
                        --p;
                    }
                    S.tk_d[p] = d;
                    S.tk_id[p] = id;
                    if (S.tk_n < kk) S.tk_n++;
                    S.processed += 1;
                    S.nfull += 1;
                    S.counter = 0;
                }
                __syncwarp();
                j0 = jins + 1;
            }
        }
        __syncthreads();
    }
    for (int r = tid; r < ko; r += VO_NT) {          // rows of ko >= kk entries, padded -1 / +inf
        bool ok = r < S.tk_n && r < kk;
        out_ids[(long long)q * ko + r] = ok ? (long long)S.tk_id[r] : -1LL;
        out_d[(long long)q * ko + r] = ok ? S.tk_d[r] : INFINITY;
    }
    if (tid == 0) {
        if (out_nver) out_nver[q] = S.processed;
        if (out_nfull) out_nfull[q] = S.nfull;
        if (out_nblk) out_nblk[q] = (long long)S.nblk;
    }
}

int next_pow2(long long n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

size_t vo_smem(const crisp_index *ix, int cap_keys) {
    int nb = ix->Dp / 32;
    return sizeof(float) * ((size_t)ix->Dp + nb + nb + (size_t)VO_CHUNK * nb) + sizeof(uint32_t) * (size_t)cap_keys;
}

}  // namespace

crisp_status crisp_run_verify_opt(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                  int64_t stride, const int64_t *ncand, int32_t k, float eps0, int64_t patience,
                                  int32_t order,
                                  int64_t *ids, float *d2, int64_t *nver, int64_t *nfull, int64_t *nblk,
                                  cudaStream_t st, const QParam *qp, int32_t ko) {
    if (nq <= 0) return CRISP_OK;
    if (ko <= 0) ko = k;
    int64_t cap = stride;
    if (cap > CRISP_OPT_MAX_CAND) {
        // only the real candidate counts matter: read them back (one small copy)
        int64_t *h = new int64_t[nq];
        cudaError_t e = cudaMemcpyAsync(h, ncand, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { delete[] h; return crisp_cuda_fail(e, "ncand readback", __FILE__, __LINE__); }
        int64_t mx = 0;
        for (int32_t i = 0; i < nq; ++i) mx = h[i] > mx ? h[i] : mx;
        delete[] h;
        if (mx > CRISP_OPT_MAX_CAND) {
            crisp_set_error("Optimized mode: a query has %lld candidates (> %d); set max_candidates", (long long)mx,
                            CRISP_OPT_MAX_CAND);
            return CRISP_EUNSUPPORTED;
        }
        cap = mx;
    }
    int cap_keys = next_pow2(cap < 1 ? 1 : cap);
    size_t smem = vo_smem(ix, cap_keys);
    CRISP_CK(cudaFuncSetAttribute(k_verify_opt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_verify_opt<<<nq, VO_NT, smem, st>>>(ix_view(ix), Qr, nq, cand, (long long)stride, (const long long *)ncand, k,
                                          eps0, (long long)patience, order, qp, ko, cap_keys, (long long *)ids, d2,
                                          (long long *)nver, (long long *)nfull, (long long *)nblk);
    CRISP_COUNT_LAUNCH();
    CRISP_CK_LAUNCH();
    return CRISP_OK;
}

extern "C" crisp_status crisp_verify_opt(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                         int64_t cand_stride, const int64_t *ncand, int32_t k, float eps0,
                                         int64_t patience, int32_t order, int64_t *ids, float *sqdist,
                                         int64_t *n_verified, int64_t *n_full, int64_t *n_blocks, void *stream) {
    CRISP_REQUIRE(ix != nullptr, "null index");
    CRISP_REQUIRE(nq >= 0 && k >= 1 && k <= CRISP_KOUT_MAX, "crisp_verify_opt: bad nq or k");
    CRISP_REQUIRE(nq == 0 || (Qr && cand && ncand && ids && sqdist), "crisp_verify_opt: null pointer");
    CRISP_REQUIRE(cand_stride >= 1, "crisp_verify_opt: cand_stride < 1");
    CRISP_REQUIRE(order == 0 || order == 1, "crisp_verify_opt: order must be 0 (Hamming) or 1 (id)");
    return crisp_run_verify_opt(ix, Qr, nq, cand, cand_stride, ncand, k, eps0, patience, order, ids, sqdist, n_verified,
                                n_full, n_blocks, as_stream(stream), nullptr, k);
}
