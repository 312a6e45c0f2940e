// C ABI of the CRISP GB300 library: errors, index lifetime, import/export, and
// the batched search (Algorithm 1) that chains the query kernels on one stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

// launchers defined in query.cu / verify.cu
crisp_status crisp_run_activate(const crisp_index *ix, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, cudaStream_t st,
                                float *cost_first, float *cost_last);
crisp_status crisp_run_count_cut(const crisp_index *ix, const int32_t *act, const int32_t *nact, int32_t nq,
                                 int32_t tau, int32_t k, int64_t cap, int32_t *cand, int64_t stride, int64_t *ncand,
                                 uint8_t *score, int32_t *how, cudaStream_t st);
crisp_status crisp_run_rerank(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                              int64_t stride, const int64_t *ncand, int32_t k, float *dbuf, int64_t *ids, float *d2,
                              cudaStream_t st, bool no_alloc = false, bool may_group = true);
crisp_status crisp_run_shortlist(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                 int64_t stride, const int64_t *ncand, int32_t precision, int32_t S, float *dbuf,
                                 int32_t *out, int64_t out_stride, int64_t *nout, cudaStream_t st,
                                 const int64_t *S_per_query);
crisp_status crisp_run_verify_opt(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                  int64_t stride, const int64_t *ncand, int32_t k, float eps0, int64_t patience,
                                  int32_t order, int64_t *ids, float *d2, int64_t *nver, int64_t *nfull, int64_t *nblk,
                                  cudaStream_t st);

crisp_status crisp_run_features(const crisp_index *ix, const int32_t *cand, int64_t stride, const int64_t *ncand,
                                const uint8_t *score, const float *cfirst, const float *clast, int32_t nq, int32_t k,
                                int32_t tau, float *feats, cudaStream_t st);
crisp_status crisp_run_mlp_depth(const crisp_index *ix, const float *feats, int32_t nq, const int64_t *ncand,
                                 int64_t stride, int32_t k, float mV, float mS, int64_t *dV, int64_t *dS,
                                 cudaStream_t st);
crisp_status crisp_run_select_score(const int32_t *cand, int64_t stride, const int64_t *ncand, const uint8_t *score,
                                    const int64_t *depth, int32_t nq, int32_t *out, int64_t *nout, cudaStream_t st);
crisp_status crisp_run_labels_v(const int32_t *cand, int64_t stride, const int64_t *ncand, const uint8_t *score,
                                const int64_t *top, int32_t k, int32_t nq, int64_t *dV, cudaStream_t st);
crisp_status crisp_run_labels_s(const int32_t *P, int64_t stride, const int64_t *nP, const float *dist,
                                const int64_t *top, int32_t k, int32_t nq, int64_t *dS, cudaStream_t st);
crisp_status crisp_run_log2_targets(const int64_t *dV, const int64_t *dS, int32_t nq, int64_t *labels, float *targets,
                                    cudaStream_t st);

// ------------------------------------------------------------ scratch pool
#include <mutex>
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static bool g_pool_ok[64];

static cudaMemPool_t scratch_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_pool_ok[dev]) {
        cudaMemPoolProps pp = {};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        if (cudaMemPoolCreate(&g_pool[dev], &pp) != cudaSuccess) return nullptr;
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool_ok[dev] = true;
    }
    return g_pool[dev];
}

cudaError_t crisp_scratch_alloc(void **p, size_t bytes, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = scratch_pool(dev);
    if (!pool) return cudaMallocAsync(p, bytes, st);
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void crisp_scratch_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void crisp_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

crisp_status crisp_cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    crisp_set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? CRISP_ENOMEM : CRISP_ECUDA;
}

extern "C" const char *crisp_last_error(void) { return g_err; }

std::atomic<unsigned long long> g_crisp_launches{0};

extern "C" uint64_t crisp_kernel_launches(void) { return g_crisp_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------- readings
int32_t crisp_tau(double alpha, int32_t M) { return (int32_t)ceil(alpha * (double)M - 1e-9); }

int64_t crisp_budget(double rho, int64_t N) {
    int64_t b = (int64_t)ceil(rho * (double)N - 1e-9);
    return b < 1 ? 1 : b;
}

void crisp_subspace(int32_t D, int32_t M, int32_t m, int32_t *lo, int32_t *hl, int32_t *hr) {
    int32_t a = (int32_t)(((int64_t)m * D) / M), b = (int32_t)(((int64_t)(m + 1) * D) / M);
    int32_t d = b - a;
    *lo = a;
    *hl = d / 2;
    *hr = d - d / 2;
}

// ------------------------------------------------------------ lifetime
static void free_index_arrays(crisp_index *ix) {
    cudaFree(ix->R32);
    cudaFree(ix->cent);
    cudaFree(ix->offsets);
    cudaFree(ix->ids);
    cudaFree(ix->tile_off);
    cudaFree(ix->Xr);
    cudaFree(ix->codes);
    cudaFree(ix->Xb);
    cudaFree(ix->X8);
    cudaFree(ix->S8);
    cudaFree(ix->xn2);
    cudaFree(ix->mlp);
}

extern "C" void crisp_free(crisp_index *ix) {
    if (!ix) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ix->device);
    cudaDeviceSynchronize();
    free_index_arrays(ix);
    cudaSetDevice(cur);
    delete ix;
}

// Allocate the arrays of an index whose sizes are already set.
crisp_status crisp_alloc_index(crisp_index *ix) {
    const int64_t K2 = (int64_t)ix->K * ix->K;
    ix->T = (int32_t)((ix->N + CRISP_TILE - 1) / CRISP_TILE);
    struct A { void **p; size_t n; } arrs[] = {
        {(void **)&ix->cent, sizeof(float) * (size_t)ix->M * 2 * ix->K * ix->H},
        {(void **)&ix->offsets, sizeof(int32_t) * (size_t)ix->M * (K2 + 1)},
        {(void **)&ix->ids, sizeof(int32_t) * (size_t)ix->M * ix->N},
        {(void **)&ix->tile_off, sizeof(int32_t) * (size_t)ix->M * K2 * (ix->T + 1)},
        {(void **)&ix->Xr, sizeof(float) * (size_t)ix->N * ix->Dp},
        {(void **)&ix->codes, sizeof(uint32_t) * (size_t)ix->N * (ix->Dp / 32)},
        {(void **)&ix->R32, ix->rotated ? sizeof(float) * (size_t)ix->D * ix->D : 0},
        {(void **)&ix->xn2, sizeof(float) * (size_t)ix->N},
    };
    ix->bytes = 0;
    for (auto &a : arrs) {
        if (!a.n) continue;
        CRISP_CK(cudaMalloc(a.p, a.n));
        ix->bytes += (int64_t)a.n;
    }
    return CRISP_OK;
}

// Derived tables: per-tile positions inside every cell list, largest cell.
crisp_status crisp_finish_index(crisp_index *ix, cudaStream_t st) {
    crisp_status s = launch_tile_offsets(ix, st);
    if (!s) s = launch_row_norms(ix, st);
    if (s) return s;
    const int64_t K2 = (int64_t)ix->K * ix->K;
    std::vector<int32_t> off((size_t)ix->M * (K2 + 1));
    CRISP_CK(cudaMemcpyAsync(off.data(), ix->offsets, sizeof(int32_t) * off.size(), cudaMemcpyDeviceToHost, st));
    CRISP_CK(cudaStreamSynchronize(st));
    int32_t mx = 0;
    for (int32_t m = 0; m < ix->M; ++m)
        for (int64_t c = 0; c < K2; ++c) mx = std::max(mx, off[m * (K2 + 1) + c + 1] - off[m * (K2 + 1) + c]);
    ix->max_cell = mx;
    return CRISP_OK;
}

extern "C" crisp_status crisp_index_get_info(const crisp_index *ix, crisp_index_info *o) {
    CRISP_REQUIRE(ix && o, "crisp_index_get_info: null pointer");
    memset(o, 0, sizeof *o);
    o->N = ix->N; o->D = ix->D; o->Dp = ix->Dp; o->M = ix->M; o->K = ix->K; o->H = ix->H;
    o->rotated = ix->rotated; o->cev = ix->cev; o->max_cell = ix->max_cell;
    o->id_tile_log2 = CRISP_TILE_LOG2; o->device_bytes = ix->bytes;
    o->R32 = ix->R32; o->cent = ix->cent; o->offsets = ix->offsets; o->ids = ix->ids; o->Xr = ix->Xr;
    o->codes = ix->codes;
    o->Xb = ix->Xb; o->X8 = ix->X8; o->S8 = ix->S8;
    return CRISP_OK;
}

// ------------------------------------------------------- blob format
static const char kMagic[8] = {'C', 'R', 'I', 'S', 'P', 'I', 'X', '1'};

struct BlobLayout {
    size_t off[6], len[6], total;   // R32, cent, offsets, ids, Xr, codes
};

static BlobLayout blob_layout(int64_t N, int32_t D, int32_t Dp, int32_t M, int32_t K, int32_t H, int32_t rot) {
    BlobLayout L;
    size_t K2 = (size_t)K * K;
    size_t lens[6] = {rot ? sizeof(float) * (size_t)D * D : 0, sizeof(float) * (size_t)M * 2 * K * H,
                      sizeof(int32_t) * (size_t)M * (K2 + 1), sizeof(int32_t) * (size_t)M * N,
                      sizeof(float) * (size_t)N * Dp, sizeof(uint32_t) * (size_t)N * (Dp / 32)};
    size_t pos = 256;
    for (int i = 0; i < 6; ++i) {
        L.off[i] = pos;
        L.len[i] = lens[i];
        pos += lens[i];
        pos = (pos + 255) / 256 * 256;
    }
    L.total = pos;
    return L;
}

extern "C" crisp_status crisp_index_export(const crisp_index *ix, void *host_buf, size_t *bytes) {
    CRISP_REQUIRE(ix && bytes, "crisp_index_export: null pointer");
    BlobLayout L = blob_layout(ix->N, ix->D, ix->Dp, ix->M, ix->K, ix->H, ix->rotated);
    if (!host_buf) { *bytes = L.total; return CRISP_OK; }
    CRISP_REQUIRE(*bytes >= L.total, "crisp_index_export: buffer of %zu bytes, need %zu", *bytes, L.total);
    uint8_t *b = (uint8_t *)host_buf;
    memset(b, 0, L.total);
    memcpy(b, kMagic, 8);
    int64_t h[8] = {1, ix->N, ix->D, ix->Dp, ix->M, ix->K, ix->H, ix->rotated};
    memcpy(b + 8, h, sizeof h);
    memcpy(b + 72, &ix->cev, sizeof(double));
    const void *src[6] = {ix->R32, ix->cent, ix->offsets, ix->ids, ix->Xr, ix->codes};
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ix->device);
    CRISP_CK(cudaDeviceSynchronize());
    for (int i = 0; i < 6; ++i)
        if (L.len[i]) CRISP_CK(cudaMemcpy(b + L.off[i], src[i], L.len[i], cudaMemcpyDeviceToHost));
    cudaSetDevice(cur);
    *bytes = L.total;
    return CRISP_OK;
}

extern "C" crisp_status crisp_index_import(const void *host_buf, size_t bytes, void *stream, crisp_index **out) {
    CRISP_REQUIRE(host_buf && out, "crisp_index_import: null pointer");
    CRISP_REQUIRE(bytes >= 256 && memcmp(host_buf, kMagic, 8) == 0, "crisp_index_import: not a CRISP index blob");
    const uint8_t *b = (const uint8_t *)host_buf;
    int64_t h[8];
    memcpy(h, b + 8, sizeof h);
    double cev;
    memcpy(&cev, b + 72, sizeof cev);
    CRISP_REQUIRE(h[0] == 1, "crisp_index_import: unsupported version %lld", (long long)h[0]);
    int64_t N = h[1];
    int32_t D = (int32_t)h[2], Dp = (int32_t)h[3], M = (int32_t)h[4], K = (int32_t)h[5], H = (int32_t)h[6];
    int32_t rot = (int32_t)h[7];
    CRISP_REQUIRE(N >= 1 && N < (1LL << 31) && D >= 2 && Dp == (D + 31) / 32 * 32 && M >= 1 && 2 * M <= D,
                  "crisp_index_import: inconsistent header");
    CRISP_REQUIRE(K >= 2 && K <= CRISP_KMAX, "crisp_index_import: K = %d outside [2, %d]", K, CRISP_KMAX);
    int32_t hmax = 0;
    for (int32_t m = 0; m < M; ++m) {
        int32_t lo, hl, hr;
        crisp_subspace(D, M, m, &lo, &hl, &hr);
        hmax = std::max(hmax, std::max(hl, hr));
    }
    CRISP_REQUIRE(H == hmax, "crisp_index_import: H = %d, expected %d", H, hmax);
    BlobLayout L = blob_layout(N, D, Dp, M, K, H, rot);
    CRISP_REQUIRE(bytes >= L.total, "crisp_index_import: blob of %zu bytes, need %zu", bytes, L.total);
    crisp_index *ix = new crisp_index();
    ix->N = N; ix->D = D; ix->Dp = Dp; ix->M = M; ix->K = K; ix->H = H; ix->rotated = rot != 0; ix->cev = cev;
    cudaGetDevice(&ix->device);
    cudaStream_t st = as_stream(stream);
    crisp_status s = crisp_alloc_index(ix);
    void *dst[6] = {ix->R32, ix->cent, ix->offsets, ix->ids, ix->Xr, ix->codes};
    for (int i = 0; i < 6 && s == CRISP_OK; ++i) {
        if (!L.len[i]) continue;
        cudaError_t e = cudaMemcpyAsync(dst[i], b + L.off[i], L.len[i], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = crisp_cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    }
    if (s == CRISP_OK) s = crisp_finish_index(ix, st);
    if (s != CRISP_OK) {
        free_index_arrays(ix);
        delete ix;
        return s;
    }
    *out = ix;
    return CRISP_OK;
}

// --------------------------------------------------------------- search
struct SearchPlan {
    int32_t tau, phi, k, prec, S;
    bool learned;
    int64_t budget, cap, stride;
    int32_t chunk;
    size_t per_query;
};

static crisp_status plan_search(const crisp_index *ix, int32_t nq, const crisp_search_params *p, SearchPlan *pl) {
    CRISP_REQUIRE(ix && p, "crisp_search: null index or params");
    CRISP_REQUIRE(nq >= 0, "crisp_search: nq < 0");
    CRISP_REQUIRE(p->k >= 1 && p->k <= CRISP_KOUT_MAX && p->k <= ix->N, "crisp_search: k = %d outside [1, min(256, N)]",
                  p->k);
    CRISP_REQUIRE(p->mode >= 0 && p->mode <= 2, "crisp_search: mode must be 0, 1 or 2");
    if (p->mode == 2) {
        CRISP_REQUIRE(ix->mlp, "crisp_search: learned mode needs a model (crisp_index_set_model)");
        CRISP_REQUIRE(ix->Xb, "crisp_search: learned mode needs the BF16 copy (crisp_index_add_copies)");
    }
    CRISP_REQUIRE(p->rho > 0.0 && p->rho <= 1.0, "crisp_search: rho outside (0, 1]");
    CRISP_REQUIRE(p->alpha >= 0.0 && p->alpha <= 1.0, "crisp_search: alpha outside [0, 1]");
    CRISP_REQUIRE(p->max_candidates == 0 || p->max_candidates >= p->k, "crisp_search: 0 < max_candidates < k");
    CRISP_REQUIRE(p->verify_order == 0 || p->verify_order == 1, "crisp_search: verify_order must be 0 or 1");
    CRISP_REQUIRE(p->reserved == 0, "crisp_search: reserved must be 0");
    CRISP_REQUIRE(p->max_candidates >= 0, "crisp_search: max_candidates < 0");
    CRISP_REQUIRE(p->precision >= 0 && p->precision <= 2, "crisp_search: precision must be 0, 1 or 2");
    if (p->precision > 0) {
        CRISP_REQUIRE(p->mode == 0, "crisp_search: coarse scoring (precision > 0) runs in Guaranteed mode");
        CRISP_REQUIRE(p->shortlist >= p->k, "crisp_search: shortlist < k");
        CRISP_REQUIRE(p->precision != 1 || ix->Xb, "crisp_search: the index has no BF16 copy (crisp_index_add_copies)");
        CRISP_REQUIRE(p->precision != 2 || ix->X8, "crisp_search: the index has no FP8 copy (crisp_index_add_copies)");
    }
    if (ix->M > 127) { crisp_set_error("crisp_search: M > 127 is not supported"); return CRISP_EUNSUPPORTED; }
    pl->tau = crisp_tau(p->alpha, ix->M);
    pl->budget = crisp_budget(p->rho, ix->N);
    pl->phi = p->mode == 1 ? 1 : 0;
    pl->learned = p->mode == 2;
    pl->k = p->k;
    pl->cap = p->max_candidates;
    pl->prec = p->precision;
    pl->S = p->precision > 0 ? p->shortlist : 0;
    // Every candidate needs V >= tau and the scores sum to at most w * (ids
    // retrieved), each subspace retrieving fewer than budget + largest cell:
    // |C| <= w M (budget + max_cell) / tau; the fallback returns at most k.
    int64_t bound = ix->N;
    if (pl->tau > 0) {
        int64_t w = p->mode == 1 ? 2 : 1;
        int64_t votes = w * (int64_t)ix->M * (pl->budget + ix->max_cell);
        bound = std::min<int64_t>(ix->N, std::max<int64_t>((votes + pl->tau - 1) / pl->tau, p->k));
    }
    pl->stride = p->max_candidates > 0 ? std::min<int64_t>(p->max_candidates, bound) : bound;
    if (pl->cap > pl->stride) pl->cap = 0;   // the cap can never bind
    pl->stride = std::max<int64_t>(pl->stride, 1);
    const int64_t K2 = (int64_t)ix->K * ix->K;
    pl->per_query = sizeof(float) * ix->Dp + sizeof(int32_t) * ix->M * K2 + sizeof(int32_t) * ix->M +
                    sizeof(int64_t) * ix->M + sizeof(int32_t) * pl->stride * 2 + sizeof(int32_t) * pl->S + 64;
    if (pl->learned)   // scores, traversal costs, features, selected list
        pl->per_query += pl->stride + sizeof(float) * (2 * ix->M + 2 * ix->M + 68) + sizeof(int32_t) * pl->stride + 64;
    size_t budget_bytes = (size_t)16 << 30;
    if (const char *e = getenv("CRISP_SCRATCH_MB")) budget_bytes = (size_t)atoll(e) << 20;
    int64_t chunk = (int64_t)(budget_bytes / pl->per_query);
    chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, CRISP_GROUP_MAXQ));   // chunks stay groupable
    pl->chunk = (int32_t)std::min<int64_t>(chunk, std::max<int32_t>(nq, 1));
    return CRISP_OK;
}

extern "C" crisp_status crisp_search_scratch_bytes(const crisp_index *ix, int32_t nq, const crisp_search_params *p,
                                                   size_t *bytes) {
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, p, &pl);
    if (s) return s;
    CRISP_REQUIRE(bytes, "crisp_search_scratch_bytes: null output");
    *bytes = pl.per_query * (size_t)pl.chunk;
    return CRISP_OK;
}

template <class T>
static T *carve(uint8_t *&p, size_t n) {
    T *r = reinterpret_cast<T *>(p);
    p += (sizeof(T) * n + 255) / 256 * 256;
    return r;
}

static crisp_status search_device(const crisp_index *ix, const float *Q, int32_t nq, const crisp_search_params *p,
                                  int64_t *ids, float *d2, crisp_query_stats *stats, cudaStream_t st) {
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, p, &pl);
    if (s) return s;
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Q && ids && d2, "crisp_search: null pointer");
    const int64_t K2 = (int64_t)ix->K * ix->K;
    const int32_t C = pl.chunk, M = ix->M;
    size_t total = 0;
    {
        size_t parts[] = {sizeof(float) * (size_t)C * ix->Dp, sizeof(int32_t) * (size_t)C * M * K2,
                          sizeof(int32_t) * (size_t)C * M, sizeof(int64_t) * (size_t)C * M,
                          sizeof(int32_t) * (size_t)C * pl.stride, sizeof(float) * (size_t)C * pl.stride,
                          sizeof(int64_t) * (size_t)C, sizeof(int32_t) * (size_t)C, sizeof(int64_t) * (size_t)C,
                          sizeof(int64_t) * (size_t)C, sizeof(int32_t) * (size_t)C * pl.S,
                          sizeof(int64_t) * (size_t)C,
                          pl.learned ? (size_t)C * pl.stride : 0, pl.learned ? sizeof(float) * (size_t)C * M : 0,
                          pl.learned ? sizeof(float) * (size_t)C * M : 0,
                          pl.learned ? sizeof(float) * (size_t)C * (2 * M + 68) : 0, sizeof(int64_t) * (size_t)C,
                          sizeof(int64_t) * (size_t)C, pl.learned ? sizeof(int32_t) * (size_t)C * pl.stride : 0,
                          sizeof(int64_t) * (size_t)C};
        for (size_t x : parts) total += (x + 255) / 256 * 256;
    }
    uint8_t *base = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&base, total, st));
    uint8_t *cur = base;
    float *Qr = carve<float>(cur, (size_t)C * ix->Dp);
    int32_t *act = carve<int32_t>(cur, (size_t)C * M * K2);
    int32_t *nact = carve<int32_t>(cur, (size_t)C * M);
    int64_t *retr = carve<int64_t>(cur, (size_t)C * M);
    int32_t *cand = carve<int32_t>(cur, (size_t)C * pl.stride);
    float *dist = carve<float>(cur, (size_t)C * pl.stride);
    int64_t *ncand = carve<int64_t>(cur, C);
    int32_t *how = carve<int32_t>(cur, C);
    int64_t *nver = carve<int64_t>(cur, C);
    int64_t *nfull = carve<int64_t>(cur, C);
    int32_t *shortl = carve<int32_t>(cur, (size_t)C * pl.S);
    int64_t *nshort = carve<int64_t>(cur, C);
    uint8_t *score = pl.learned ? carve<uint8_t>(cur, (size_t)C * pl.stride) : nullptr;
    float *cfirst = pl.learned ? carve<float>(cur, (size_t)C * M) : nullptr;
    float *clast = pl.learned ? carve<float>(cur, (size_t)C * M) : nullptr;
    float *feats = pl.learned ? carve<float>(cur, (size_t)C * (2 * M + 68)) : nullptr;
    int64_t *dV = pl.learned ? carve<int64_t>(cur, C) : nullptr;
    int64_t *dS = pl.learned ? carve<int64_t>(cur, C) : nullptr;
    int32_t *selV = pl.learned ? carve<int32_t>(cur, (size_t)C * pl.stride) : nullptr;
    int64_t *nsel = pl.learned ? carve<int64_t>(cur, C) : nullptr;
    for (int32_t c0 = 0; c0 < nq && s == CRISP_OK; c0 += C) {
        int32_t nc = std::min(C, nq - c0);
        const float *Qc = Q + (int64_t)c0 * ix->D;
        if (ix->rotated) s = crisp_rotate_rows(Qc, nc, ix->D, ix->D, ix->R32, Qr, ix->Dp, st);
        else s = launch_pad_rows(Qc, nc, ix->D, ix->D, Qr, ix->Dp, st);
        if (!s) s = crisp_run_activate(ix, Qr, nc, pl.phi, pl.k, pl.budget, act, nact, retr, st, cfirst, clast);
        if (!s) s = crisp_run_count_cut(ix, act, nact, nc, pl.tau, pl.k, pl.cap, cand, pl.stride, ncand, score, how, st);
        int64_t *ids_c = ids + (int64_t)c0 * pl.k;
        float *d2_c = d2 + (int64_t)c0 * pl.k;
        if (!s && pl.learned) {
            // F1: features -> MLP depths -> score prefix -> BF16 shortlist -> FP32 re-rank
            s = crisp_run_features(ix, cand, pl.stride, ncand, score, cfirst, clast, nc, pl.k, pl.tau, feats, st);
            if (!s) s = crisp_run_mlp_depth(ix, feats, nc, ncand, pl.stride, pl.k, p->depth_margin, p->short_margin, dV,
                                            dS, st);
            if (!s) s = crisp_run_select_score(cand, pl.stride, ncand, score, dV, nc, selV, nsel, st);
            if (!s) s = crisp_run_shortlist(ix, Qr, nc, selV, pl.stride, nsel, 1, 1, dist, cand, pl.stride, nshort, st,
                                            dS);
            // shortlists are short whatever the list stride: stream them per query
            if (!s) s = crisp_run_rerank(ix, Qr, nc, cand, pl.stride, nshort, pl.k, dist, ids_c, d2_c, st, false, false);
            if (!s && stats)
                s = launch_write_stats(nc, ncand, how, retr, M, nsel, nshort, pl.tau, stats + c0, st);
        } else if (!s && p->mode == 0 && pl.prec > 0) {
            // F2: coarse-score every candidate on the low-precision rows, then the
            // FP32 re-rank of the shortlist
            s = crisp_run_shortlist(ix, Qr, nc, cand, pl.stride, ncand, pl.prec, pl.S, dist, shortl, pl.S, nshort, st,
                                    nullptr);
            if (!s) s = crisp_run_rerank(ix, Qr, nc, shortl, pl.S, nshort, pl.k, dist, ids_c, d2_c, st);
            if (!s && stats)
                s = launch_write_stats(nc, ncand, how, retr, M, ncand, nshort, pl.tau, stats + c0, st);
        } else if (!s && p->mode == 0) {
            s = crisp_run_rerank(ix, Qr, nc, cand, pl.stride, ncand, pl.k, dist, ids_c, d2_c, st);
            if (!s && stats)
                s = launch_write_stats(nc, ncand, how, retr, M, nullptr, nullptr, pl.tau, stats + c0, st);
        } else if (!s) {
            int64_t P = p->patience_factor > 0 ? (int64_t)p->patience_factor * pl.k : 0;
            s = crisp_run_verify_opt(ix, Qr, nc, cand, pl.stride, ncand, pl.k, p->eps0, P, p->verify_order, ids_c,
                                     d2_c, nver, nfull, nullptr, st);
            if (!s && stats) s = launch_write_stats(nc, ncand, how, retr, M, nver, nfull, pl.tau, stats + c0, st);
        }
    }
    crisp_scratch_free(base, st);
    return s;
}

extern "C" crisp_status crisp_search(const crisp_index *ix, const float *Q, int32_t nq, const crisp_search_params *p,
                                     int64_t *ids, float *sqdist, crisp_query_stats *stats, void *stream) {
    return search_device(ix, Q, nq, p, ids, sqdist, stats, as_stream(stream));
}

extern "C" crisp_status crisp_search_host(const crisp_index *ix, const float *Q, int32_t nq,
                                          const crisp_search_params *p, int64_t *ids, float *sqdist,
                                          crisp_query_stats *stats, void *stream) {
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, p, &pl);
    if (s) return s;
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Q && ids && sqdist, "crisp_search_host: null pointer");
    cudaStream_t st = as_stream(stream);
    size_t qb = sizeof(float) * (size_t)nq * ix->D, ib = sizeof(int64_t) * (size_t)nq * p->k,
           db = sizeof(float) * (size_t)nq * p->k, sb = stats ? sizeof(crisp_query_stats) * (size_t)nq : 0;
    uint8_t *buf = nullptr;
    size_t tot = (qb + 255) / 256 * 256 + (ib + 255) / 256 * 256 + (db + 255) / 256 * 256 + (sb + 255) / 256 * 256;
    CRISP_CK(crisp_scratch_alloc((void **)&buf, tot, st));
    uint8_t *cur = buf;
    float *dQ = carve<float>(cur, (size_t)nq * ix->D);
    int64_t *dI = carve<int64_t>(cur, (size_t)nq * p->k);
    float *dD = carve<float>(cur, (size_t)nq * p->k);
    crisp_query_stats *dS = stats ? carve<crisp_query_stats>(cur, nq) : nullptr;
    cudaError_t e = cudaMemcpyAsync(dQ, Q, qb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = crisp_cuda_fail(e, "cudaMemcpyAsync(Q)", __FILE__, __LINE__);
    if (!s) s = search_device(ix, dQ, nq, p, dI, dD, dS, st);
    if (!s) {
        e = cudaMemcpyAsync(ids, dI, ib, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sqdist, dD, db, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && stats) e = cudaMemcpyAsync(stats, dS, sb, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) s = crisp_cuda_fail(e, "cudaMemcpyAsync(out)", __FILE__, __LINE__);
    }
    crisp_scratch_free(buf, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (!s && e2 != cudaSuccess) s = crisp_cuda_fail(e2, "cudaStreamSynchronize", __FILE__, __LINE__);
    return s;
}

// ------------------------------------------------------- learned training data
extern "C" crisp_status crisp_learned_data(const crisp_index *ix, const float *Q, int32_t nq,
                                           const crisp_search_params *p, float *features, int64_t *labels,
                                           float *targets, void *stream) {
    CRISP_REQUIRE(ix && p, "crisp_learned_data: null index or params");
    CRISP_REQUIRE(ix->Xb, "crisp_learned_data: the index needs the BF16 copy (crisp_index_add_copies)");
    crisp_search_params g = *p;
    g.mode = 0;
    g.precision = 0;
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, &g, &pl);
    if (s) return s;
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Q && features && labels, "crisp_learned_data: null pointer");
    cudaStream_t st = as_stream(stream);
    const int64_t K2 = (int64_t)ix->K * ix->K;
    const int32_t M = ix->M, F = 2 * M + 68, k = pl.k;
    int64_t per = pl.per_query + pl.stride * 5 + sizeof(float) * (4 * M + 2 * k) + 256;
    int32_t C = (int32_t)std::max<int64_t>(1, std::min<int64_t>(pl.chunk, ((int64_t)16 << 30) / per));
    C = std::min(C, nq);
    size_t parts[] = {sizeof(float) * (size_t)C * ix->Dp, sizeof(int32_t) * (size_t)C * M * K2,
                      sizeof(int32_t) * (size_t)C * M, sizeof(int64_t) * (size_t)C * M, sizeof(float) * (size_t)C * M,
                      sizeof(float) * (size_t)C * M, sizeof(int32_t) * (size_t)C * pl.stride, (size_t)C * pl.stride,
                      sizeof(float) * (size_t)C * pl.stride, sizeof(int64_t) * (size_t)C, sizeof(int32_t) * (size_t)C,
                      sizeof(int64_t) * (size_t)C * k, sizeof(float) * (size_t)C * k, sizeof(int64_t) * (size_t)C,
                      sizeof(int64_t) * (size_t)C, sizeof(int32_t) * (size_t)C * pl.stride, sizeof(int64_t) * (size_t)C,
                      sizeof(int64_t) * (size_t)C};
    size_t total = 0;
    for (size_t x : parts) total += (x + 255) / 256 * 256;
    uint8_t *base = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&base, total, st));
    uint8_t *cur = base;
    float *Qr = carve<float>(cur, (size_t)C * ix->Dp);
    int32_t *act = carve<int32_t>(cur, (size_t)C * M * K2);
    int32_t *nact = carve<int32_t>(cur, (size_t)C * M);
    int64_t *retr = carve<int64_t>(cur, (size_t)C * M);
    float *cfirst = carve<float>(cur, (size_t)C * M);
    float *clast = carve<float>(cur, (size_t)C * M);
    int32_t *cand = carve<int32_t>(cur, (size_t)C * pl.stride);
    uint8_t *score = carve<uint8_t>(cur, (size_t)C * pl.stride);
    float *dist = carve<float>(cur, (size_t)C * pl.stride);
    int64_t *ncand = carve<int64_t>(cur, C);
    int32_t *how = carve<int32_t>(cur, C);
    int64_t *top = carve<int64_t>(cur, (size_t)C * k);
    float *topd = carve<float>(cur, (size_t)C * k);
    int64_t *dV = carve<int64_t>(cur, C);
    int64_t *dS = carve<int64_t>(cur, C);
    int32_t *selV = carve<int32_t>(cur, (size_t)C * pl.stride);
    int64_t *nsel = carve<int64_t>(cur, C);
    int64_t *nshort = carve<int64_t>(cur, C);
    for (int32_t c0 = 0; c0 < nq && s == CRISP_OK; c0 += C) {
        int32_t nc = std::min(C, nq - c0);
        const float *Qc = Q + (int64_t)c0 * ix->D;
        if (ix->rotated) s = crisp_rotate_rows(Qc, nc, ix->D, ix->D, ix->R32, Qr, ix->Dp, st);
        else s = launch_pad_rows(Qc, nc, ix->D, ix->D, Qr, ix->Dp, st);
        if (!s) s = crisp_run_activate(ix, Qr, nc, 0, k, pl.budget, act, nact, retr, st, cfirst, clast);
        if (!s) s = crisp_run_count_cut(ix, act, nact, nc, pl.tau, k, pl.cap, cand, pl.stride, ncand, score, how, st);
        if (!s) s = crisp_run_features(ix, cand, pl.stride, ncand, score, cfirst, clast, nc, k, pl.tau,
                                       features + (int64_t)c0 * F, st);
        if (!s) s = crisp_run_rerank(ix, Qr, nc, cand, pl.stride, ncand, k, dist, top, topd, st);
        if (!s) s = crisp_run_labels_v(cand, pl.stride, ncand, score, top, k, nc, dV, st);
        if (!s) s = crisp_run_select_score(cand, pl.stride, ncand, score, dV, nc, selV, nsel, st);
        // coarse distances of the whole prefix (keep all of it), then the coarse label
        if (!s) s = crisp_run_shortlist(ix, Qr, nc, selV, pl.stride, nsel, 1, 1, dist, cand, pl.stride, nshort, st,
                                        nsel);
        if (!s) s = crisp_run_labels_s(selV, pl.stride, nsel, dist, top, k, nc, dS, st);
        if (!s) s = crisp_run_log2_targets(dV, dS, nc, labels + 2 * (int64_t)c0,
                                           targets ? targets + 2 * (int64_t)c0 : nullptr, st);
    }
    crisp_scratch_free(base, st);
    return s;
}
