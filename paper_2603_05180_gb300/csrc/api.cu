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

// launchers defined in query.cu / verify.cu / learned.cu
crisp_status crisp_run_activate(const crisp_index *ix, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, cudaStream_t st,
                                float *cost_first, float *cost_last, const QParam *qp = nullptr);
crisp_status crisp_run_count_cut(const crisp_index *ix, const int32_t *act, const int32_t *nact, int32_t nq,
                                 int32_t tau, int32_t k, int64_t cap, int32_t *cand, int64_t stride, int64_t *ncand,
                                 uint8_t *score, int32_t *how, cudaStream_t st, const QParam *qp = nullptr);
crisp_status crisp_run_rerank(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                              int64_t stride, const int64_t *ncand, int32_t k, float *dbuf, int64_t *ids, float *d2,
                              cudaStream_t st, bool no_alloc = false, bool may_group = true,
                              const QParam *qp = nullptr, int32_t ko = 0);
crisp_status crisp_run_shortlist(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                 int64_t stride, const int64_t *ncand, int32_t precision, int32_t S, float *dbuf,
                                 int32_t *out, int64_t out_stride, int64_t *nout, cudaStream_t st,
                                 const int64_t *S_per_query, const QParam *qp = nullptr, bool may_group = true);
crisp_status crisp_run_verify_opt(const crisp_index *ix, const float *Qr, int32_t nq, const int32_t *cand,
                                  int64_t stride, const int64_t *ncand, int32_t k, float eps0, int64_t patience,
                                  int32_t order, int64_t *ids, float *d2, int64_t *nver, int64_t *nfull, int64_t *nblk,
                                  cudaStream_t st, const QParam *qp, int32_t ko);

crisp_status crisp_run_features(const crisp_index *ix, const int32_t *cand, int64_t stride, const int64_t *ncand,
                                const uint8_t *score, const float *cfirst, const float *clast, int32_t nq, int32_t k,
                                int32_t tau, float *feats, cudaStream_t st, const QParam *qp = nullptr);
crisp_status crisp_run_mlp_depth(const crisp_index *ix, const float *feats, int32_t nq, const int64_t *ncand,
                                 int64_t stride, int32_t k, float mV, float mS, int64_t *dV, int64_t *dS,
                                 cudaStream_t st, const QParam *qp = nullptr);
crisp_status crisp_run_select_score(const int32_t *cand, int64_t stride, const int64_t *ncand, const uint8_t *score,
                                    const int64_t *depth, int32_t nq, int32_t *out, int64_t *nout, cudaStream_t st);
crisp_status crisp_run_labels_v(const int32_t *cand, int64_t stride, const int64_t *ncand, const uint8_t *score,
                                const int64_t *top, int32_t k, int32_t nq, int64_t *dV, cudaStream_t st);
crisp_status crisp_run_labels_s(const int32_t *P, int64_t stride, const int64_t *nP, const float *dist,
                                const int64_t *top, int32_t k, int32_t nq, int64_t *dS, cudaStream_t st);
crisp_status crisp_run_log2_targets(const int64_t *dV, const int64_t *dS, int32_t nq, int64_t *labels, float *targets,
                                    cudaStream_t st);
crisp_status launch_gather_rows(const float *Q, int32_t D, const int32_t *perm, int32_t n, float *Y, cudaStream_t st);
crisp_status launch_scatter_results(const int64_t *ids_t, const float *d2_t, const crisp_query_stats *st_t, int32_t ko,
                                    const int32_t *perm, int32_t n, int64_t *ids, float *d2, crisp_query_stats *stats,
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
        // keep up to 64 GiB between calls (the largest default search scratch, so
        // repeated searches do not map and unmap it); what a larger search took
        // goes back to the device at its next synchronisation
        uint64_t keep = (uint64_t)64 << 30;
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

std::vector<int32_t> crisp_equal_bounds(int32_t D, int32_t M) {
    std::vector<int32_t> b((size_t)M + 1);
    for (int32_t m = 0; m <= M; ++m) b[m] = (int32_t)(((int64_t)m * D) / M);
    return b;
}

int32_t crisp_bounds_half_max(const int32_t *sub, int32_t M) {
    int32_t h = 0;
    for (int32_t m = 0; m < M; ++m) {
        const int32_t w = sub[m + 1] - sub[m];
        h = std::max(h, w - w / 2);
    }
    return h;
}

bool crisp_bounds_valid(const int32_t *sub, int32_t D, int32_t M, const char *who) {
    if (!sub || sub[0] != 0 || sub[M] != D) {
        crisp_set_error("%s: subspace boundaries must run from 0 to D = %d", who, D);
        return false;
    }
    for (int32_t m = 0; m < M; ++m) {
        const int32_t w = sub[m + 1] - sub[m];
        if (w < 2 || w > 256) {
            crisp_set_error("%s: subspace %d has %d dims (need 2..256)", who, m, w);
            return false;
        }
    }
    return true;
}

// Variance-aware boundaries (§7 Adaptive Subspace Decomposition): contiguous
// subspaces with near-equal shares of the total variance.  V_j is the running
// FP64 sum of var[0..j-1]; boundary m is the last j with V_j <= m V_D / M,
// then held to [b_{m-1} + 2, b_{m-1} + 256] and to what leaves every later
// subspace 2..256 dims.  Zero total variance gives the equal split.
extern "C" crisp_status crisp_adaptive_bounds(const double *var, int32_t D, int32_t M, int32_t *bounds) {
    CRISP_REQUIRE(var && bounds, "crisp_adaptive_bounds: null pointer");
    CRISP_REQUIRE(M >= 1 && 2 * (int64_t)M <= D && D <= 256 * (int64_t)M,
                  "crisp_adaptive_bounds: need 2M <= D <= 256M (D = %d, M = %d)", D, M);
    std::vector<double> V((size_t)D + 1, 0.0);
    for (int32_t d = 0; d < D; ++d) V[d + 1] = V[d] + var[d];
    const double tot = V[D];
    bounds[0] = 0;
    int32_t j = 0;
    for (int32_t m = 1; m < M; ++m) {
        int32_t want;
        if (tot > 0.0) {
            const double t = (double)m * tot / (double)M;
            while (j < D && V[j + 1] <= t) ++j;   // targets grow with m: the scan resumes
            want = j;
        } else {
            want = (int32_t)(((int64_t)m * D) / M);
        }
        const int32_t prev = bounds[m - 1];
        const int32_t lo = std::max(prev + 2, D - 256 * (M - m)), hi = std::min(prev + 256, D - 2 * (M - m));
        bounds[m] = std::min(std::max(want, lo), hi);
    }
    bounds[M] = D;
    return CRISP_OK;
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
    cudaFree(ix->xbn2);
    cudaFree(ix->mlp);
    cudaFree(ix->sub);
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

// Allocate the arrays of an index whose sizes are already set (the centroids
// only once H is known: an index build with variance-aware boundaries sets H
// after the rows are stored).
crisp_status crisp_alloc_index(crisp_index *ix) {
    const int64_t K2 = (int64_t)ix->K * ix->K;
    ix->T = (int32_t)((ix->N + CRISP_TILE - 1) / CRISP_TILE);
    struct A { void **p; size_t n; } arrs[] = {
        {(void **)&ix->cent, sizeof(float) * (size_t)ix->M * 2 * ix->K * ix->H},   // 0 while H = 0
        {(void **)&ix->offsets, sizeof(int32_t) * (size_t)ix->M * (K2 + 1)},
        // + 4 entries: the count kernel reads the ids as aligned 16-byte quads,
        // the last of which may reach 3 entries past the end (masked out)
        {(void **)&ix->ids, sizeof(int32_t) * ((size_t)ix->M * ix->N + 4)},
        {(void **)&ix->tile_off, sizeof(int32_t) * (size_t)ix->M * K2 * (ix->T + 1)},
        {(void **)&ix->Xr, sizeof(float) * (size_t)ix->N * ix->Dp},
        {(void **)&ix->codes, sizeof(uint32_t) * (size_t)ix->N * (ix->Dp / 32)},
        {(void **)&ix->R32, ix->rotated ? sizeof(float) * (size_t)ix->D * ix->D : 0},
        {(void **)&ix->xn2, sizeof(float) * (size_t)ix->N},
        {(void **)&ix->sub, sizeof(int32_t) * ((size_t)ix->M + 1)},
    };
    ix->bytes = 0;
    for (auto &a : arrs) {
        if (!a.n) continue;
        CRISP_CK(cudaMalloc(a.p, a.n));
        ix->bytes += (int64_t)a.n;
    }
    CRISP_CK(cudaMemset(ix->ids + (size_t)ix->M * ix->N, 0, 4 * sizeof(int32_t)));
    return CRISP_OK;
}

// Derived tables: per-tile positions inside every cell list, largest cell;
// the subspace boundaries (host copy, the equal split if unset) go to the device.
crisp_status crisp_finish_index(crisp_index *ix, cudaStream_t st) {
    if (ix->sub_h.empty()) ix->sub_h = crisp_equal_bounds(ix->D, ix->M);
    CRISP_CK(cudaMemcpyAsync(ix->sub, ix->sub_h.data(), sizeof(int32_t) * ix->sub_h.size(), cudaMemcpyHostToDevice,
                             st));
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
    o->sub = ix->sub; o->block_dims = ix->block_dims; o->rotated_blocks = ix->rotated_blocks;
    return CRISP_OK;
}

extern "C" crisp_status crisp_index_get_bounds(const crisp_index *ix, int32_t *bounds) {
    CRISP_REQUIRE(ix && bounds, "crisp_index_get_bounds: null pointer");
    std::copy(ix->sub_h.begin(), ix->sub_h.end(), bounds);
    return CRISP_OK;
}

// ------------------------------------------------------- blob format
static const char kMagic[8] = {'C', 'R', 'I', 'S', 'P', 'I', 'X', '1'};

struct BlobLayout {
    size_t off[7], len[7], total;   // R32, cent, offsets, ids, Xr, codes, boundaries (version 2)
};

static BlobLayout blob_layout(int64_t N, int32_t D, int32_t Dp, int32_t M, int32_t K, int32_t H, int32_t rot,
                              int64_t version) {
    BlobLayout L;
    size_t K2 = (size_t)K * K;
    size_t lens[7] = {rot ? sizeof(float) * (size_t)D * D : 0, sizeof(float) * (size_t)M * 2 * K * H,
                      sizeof(int32_t) * (size_t)M * (K2 + 1), sizeof(int32_t) * (size_t)M * N,
                      sizeof(float) * (size_t)N * Dp, sizeof(uint32_t) * (size_t)N * (Dp / 32),
                      version >= 2 ? sizeof(int32_t) * ((size_t)M + 1) : 0};
    size_t pos = 256;
    for (int i = 0; i < 7; ++i) {
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
    // version 1 holds the equal split; other boundaries need version 2
    const int64_t version = ix->sub_h == crisp_equal_bounds(ix->D, ix->M) ? 1 : 2;
    BlobLayout L = blob_layout(ix->N, ix->D, ix->Dp, ix->M, ix->K, ix->H, ix->rotated, version);
    if (!host_buf) { *bytes = L.total; return CRISP_OK; }
    CRISP_REQUIRE(*bytes >= L.total, "crisp_index_export: buffer of %zu bytes, need %zu", *bytes, L.total);
    uint8_t *b = (uint8_t *)host_buf;
    memset(b, 0, L.total);
    memcpy(b, kMagic, 8);
    int64_t h[8] = {version, ix->N, ix->D, ix->Dp, ix->M, ix->K, ix->H, ix->rotated};
    memcpy(b + 8, h, sizeof h);
    memcpy(b + 72, &ix->cev, sizeof(double));
    const void *src[6] = {ix->R32, ix->cent, ix->offsets, ix->ids, ix->Xr, ix->codes};
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ix->device);
    CRISP_CK(cudaDeviceSynchronize());
    for (int i = 0; i < 6; ++i)
        if (L.len[i]) CRISP_CK(cudaMemcpy(b + L.off[i], src[i], L.len[i], cudaMemcpyDeviceToHost));
    if (L.len[6]) memcpy(b + L.off[6], ix->sub_h.data(), L.len[6]);
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
    CRISP_REQUIRE(h[0] == 1 || h[0] == 2, "crisp_index_import: unsupported version %lld", (long long)h[0]);
    int64_t N = h[1];
    int32_t D = (int32_t)h[2], Dp = (int32_t)h[3], M = (int32_t)h[4], K = (int32_t)h[5], H = (int32_t)h[6];
    int32_t rot = (int32_t)h[7];
    CRISP_REQUIRE(N >= 1 && N < (1LL << 31) && D >= 2 && Dp == (D + 31) / 32 * 32 && M >= 1 && 2 * M <= D,
                  "crisp_index_import: inconsistent header");
    CRISP_REQUIRE(K >= 2 && K <= CRISP_KMAX, "crisp_index_import: K = %d outside [2, %d]", K, CRISP_KMAX);
    BlobLayout L = blob_layout(N, D, Dp, M, K, H, rot, h[0]);
    CRISP_REQUIRE(bytes >= L.total, "crisp_index_import: blob of %zu bytes, need %zu", bytes, L.total);
    std::vector<int32_t> sub = crisp_equal_bounds(D, M);
    if (L.len[6]) {
        memcpy(sub.data(), b + L.off[6], L.len[6]);
        if (!crisp_bounds_valid(sub.data(), D, M, "crisp_index_import")) return CRISP_EINVAL;
    }
    const int32_t hmax = crisp_bounds_half_max(sub.data(), M);
    CRISP_REQUIRE(H == hmax, "crisp_index_import: H = %d, expected %d", H, hmax);
    CRISP_REQUIRE(H <= 128, "crisp_index_import: subspace halves wider than 128 dims");
    crisp_index *ix = new crisp_index();
    ix->sub_h = sub;
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
extern "C" int32_t crisp_search_tau(double alpha, int32_t M) { return crisp_tau(alpha, M); }
extern "C" int64_t crisp_search_budget(double rho, int64_t N) { return crisp_budget(rho, N); }

// Stage-3 class of a parameter set: Guaranteed with FP32 re-rank (0), with
// BF16 (1) or FP8 (2) coarse scores, Optimized (3), Learned (4).
static int stage_class(const crisp_search_params *p) { return p->mode == 1 ? 3 : p->mode == 2 ? 4 : p->precision; }

// Validate one parameter set; derive what the kernels read and the candidate
// list bound of a query using it.
static crisp_status check_params(const crisp_index *ix, const crisp_search_params *p, QParam *qp, int64_t *bound) {
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
    qp->k = p->k;
    qp->phi = p->mode == 1 ? 1 : 0;
    qp->tau = crisp_tau(p->alpha, ix->M);
    qp->order = p->verify_order;
    qp->budget = crisp_budget(p->rho, ix->N);
    qp->patience = p->patience_factor > 0 ? (int64_t)p->patience_factor * p->k : 0;
    qp->eps0 = p->eps0;
    qp->mV = p->depth_margin;
    qp->mS = p->short_margin;
    qp->S = p->precision > 0 ? p->shortlist : 0;
    // Every candidate needs V >= tau and the scores sum to at most w * (ids
    // retrieved), each subspace retrieving fewer than budget + largest cell:
    // |C| <= w M (budget + max_cell) / tau; the fallback returns at most k.
    int64_t b = ix->N;
    if (qp->tau > 0) {
        const int64_t w = p->mode == 1 ? 2 : 1;
        const int64_t votes = w * (int64_t)ix->M * (qp->budget + ix->max_cell);
        b = std::min<int64_t>(ix->N, std::max<int64_t>((votes + qp->tau - 1) / qp->tau, p->k));
    }
    if (p->max_candidates > 0) b = std::min<int64_t>(p->max_candidates, b);
    qp->cap = p->max_candidates > b ? 0 : p->max_candidates;   // a cap at or above the bound never binds
    *bound = std::max<int64_t>(b, 1);
    return CRISP_OK;
}

struct SearchPlan {
    bool shared;            // one parameter set for every query
    QParam q0;              // the shared set (shared)
    int cls0;               // its class (shared)
    int64_t stride;         // candidate list stride: the largest bound
    int32_t kmax;           // output row length
    int32_t Smax;           // largest shortlist of a coarse-scored query
    bool any_learned;
    int32_t chunk;
    size_t per_query;
    std::vector<QParam> qp; // per query, in the original order (not shared)
    std::vector<int> cls;   // per query (not shared)
};

static crisp_status plan_search(const crisp_index *ix, int32_t nq, const crisp_search_params *p, int32_t p_count,
                                int32_t kmax, SearchPlan *pl) {
    CRISP_REQUIRE(ix && p, "crisp_search: null index or params");
    CRISP_REQUIRE(nq >= 0, "crisp_search: nq < 0");
    CRISP_REQUIRE(p_count == 1 || p_count == nq, "crisp_search: p_count must be 1 or nq (%d), not %d", nq, p_count);
    if (ix->M > 127) { crisp_set_error("crisp_search: M > 127 is not supported"); return CRISP_EUNSUPPORTED; }
    pl->shared = p_count == 1;
    pl->stride = 1;
    pl->Smax = 0;
    pl->any_learned = false;
    int32_t kbig = 0;
    if (!pl->shared) {
        pl->qp.resize((size_t)nq);
        pl->cls.resize((size_t)nq);
    }
    for (int32_t i = 0; i < p_count; ++i) {
        QParam q;
        int64_t b;
        crisp_status s = check_params(ix, &p[i], &q, &b);
        if (s) return s;
        pl->stride = std::max(pl->stride, b);
        pl->Smax = std::max(pl->Smax, q.S);
        pl->any_learned = pl->any_learned || p[i].mode == 2;
        kbig = std::max(kbig, q.k);
        if (pl->shared) {
            pl->q0 = q;
            pl->cls0 = stage_class(&p[i]);
        } else {
            pl->qp[i] = q;
            pl->cls[i] = stage_class(&p[i]);
        }
    }
    pl->kmax = kmax <= 0 ? kbig : kmax;
    CRISP_REQUIRE(pl->kmax >= kbig, "crisp_search: kmax = %d < the largest k (%d)", kmax, kbig);
    const int64_t K2 = (int64_t)ix->K * ix->K;
    const int64_t st = pl->stride;
    pl->per_query = sizeof(float) * ix->Dp + sizeof(float) * ix->D + sizeof(int32_t) * ix->M * K2 +
                    sizeof(int32_t) * ix->M + sizeof(int64_t) * ix->M + sizeof(int32_t) * st * 2 +
                    sizeof(int32_t) * pl->Smax + sizeof(QParam) + (sizeof(int64_t) + sizeof(float)) * pl->kmax +
                    sizeof(crisp_query_stats) + 64;
    if (pl->any_learned)   // scores, traversal costs, features, selected list
        pl->per_query += st + sizeof(float) * (2 * ix->M + 2 * ix->M + 68) + sizeof(int32_t) * st + 64;
    // batches of 1,024 queries or more re-rank on the tensor cores, with bounds, kept lists and pair slots
    pl->per_query += sizeof(float) * 2 * st + sizeof(int32_t) * st + sizeof(int32_t) * st;
    // default budget: half the device memory free now, between 16 and 64 GiB (a
    // chunk large enough to re-rank in query groups when candidate lists are
    // long, and no larger than what the scratch pool keeps between calls)
    size_t budget_bytes = (size_t)16 << 30, free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
        budget_bytes = std::min<size_t>(std::max(budget_bytes, free_b / 2), (size_t)64 << 30);
    else cudaGetLastError();
    if (const char *e = getenv("CRISP_SCRATCH_MB")) budget_bytes = (size_t)atoll(e) << 20;
    int64_t chunk = (int64_t)(budget_bytes / pl->per_query);
    chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, CRISP_GROUP_MAXQ));   // chunks stay groupable
    pl->chunk = (int32_t)std::min<int64_t>(chunk, std::max<int32_t>(nq, 1));
    return CRISP_OK;
}

extern "C" crisp_status crisp_search_scratch_bytes(const crisp_index *ix, int32_t nq, const crisp_search_params *p,
                                                   int32_t p_count, size_t *bytes) {
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, p, p_count, 0, &pl);
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
                                  int32_t p_count, int64_t *ids, float *d2, int32_t kmax, crisp_query_stats *stats,
                                  cudaStream_t st) {
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, p, p_count, kmax, &pl);
    if (s) return s;
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Q && ids && d2, "crisp_search: null pointer");
    const int64_t K2 = (int64_t)ix->K * ix->K;
    const int32_t C = pl.chunk, M = ix->M, KO = pl.kmax, F = 2 * M + 68;
    const int64_t ST = pl.stride;
    // per-query batches run class by class: the queries are ordered by class
    // (stably), searched in that order, and their results put back in place
    std::vector<int32_t> perm;
    std::vector<int> pcls;            // class of each position of the ordered batch
    bool mixed = false;
    if (!pl.shared) {
        perm.resize((size_t)nq);
        for (int32_t i = 0; i < nq; ++i) perm[i] = i;
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) { return pl.cls[x] < pl.cls[y]; });
        pcls.resize((size_t)nq);
        for (int32_t i = 0; i < nq; ++i) {
            pcls[i] = pl.cls[perm[i]];
            mixed = mixed || perm[i] != i;
        }
    }
    const bool learned = pl.any_learned;
    std::vector<size_t> parts = {
        sizeof(float) * (size_t)C * ix->Dp, sizeof(int32_t) * (size_t)C * M * K2, sizeof(int32_t) * (size_t)C * M,
        sizeof(int64_t) * (size_t)C * M, sizeof(int32_t) * (size_t)C * ST, sizeof(float) * (size_t)C * ST,
        sizeof(int64_t) * (size_t)C, sizeof(int32_t) * (size_t)C, sizeof(int64_t) * (size_t)C,
        sizeof(int64_t) * (size_t)C, sizeof(int32_t) * (size_t)C * std::max(pl.Smax, 1), sizeof(int64_t) * (size_t)C,
        learned ? (size_t)C * ST : 0, learned ? sizeof(float) * (size_t)C * M : 0,
        learned ? sizeof(float) * (size_t)C * M : 0, learned ? sizeof(float) * (size_t)C * F : 0,
        sizeof(int64_t) * (size_t)C, sizeof(int64_t) * (size_t)C, learned ? sizeof(int32_t) * (size_t)C * ST : 0,
        sizeof(int64_t) * (size_t)C,
        pl.shared ? 0 : sizeof(QParam) * (size_t)nq, pl.shared ? 0 : sizeof(int32_t) * (size_t)nq,
        mixed ? sizeof(float) * (size_t)C * ix->D : 0, mixed ? sizeof(int64_t) * (size_t)C * KO : 0,
        mixed ? sizeof(float) * (size_t)C * KO : 0, mixed && stats ? sizeof(crisp_query_stats) * (size_t)C : 0};
    size_t total = 0;
    for (size_t x : parts) total += (x + 255) / 256 * 256;
    uint8_t *base = nullptr;
    CRISP_CK(crisp_scratch_alloc((void **)&base, total, st));
    uint8_t *cur = base;
    float *Qr = carve<float>(cur, (size_t)C * ix->Dp);
    int32_t *act = carve<int32_t>(cur, (size_t)C * M * K2);
    int32_t *nact = carve<int32_t>(cur, (size_t)C * M);
    int64_t *retr = carve<int64_t>(cur, (size_t)C * M);
    int32_t *cand = carve<int32_t>(cur, (size_t)C * ST);
    float *dist = carve<float>(cur, (size_t)C * ST);
    int64_t *ncand = carve<int64_t>(cur, C);
    int32_t *how = carve<int32_t>(cur, C);
    int64_t *nver = carve<int64_t>(cur, C);
    int64_t *nfull = carve<int64_t>(cur, C);
    const int32_t SM = std::max(pl.Smax, 1);
    int32_t *shortl = carve<int32_t>(cur, (size_t)C * SM);
    int64_t *nshort = carve<int64_t>(cur, C);
    uint8_t *score = learned ? carve<uint8_t>(cur, (size_t)C * ST) : nullptr;
    float *cfirst = learned ? carve<float>(cur, (size_t)C * M) : nullptr;
    float *clast = learned ? carve<float>(cur, (size_t)C * M) : nullptr;
    float *feats = learned ? carve<float>(cur, (size_t)C * F) : nullptr;
    int64_t *dV = carve<int64_t>(cur, C);
    int64_t *dS = carve<int64_t>(cur, C);
    int32_t *selV = learned ? carve<int32_t>(cur, (size_t)C * ST) : nullptr;
    int64_t *nsel = carve<int64_t>(cur, C);
    QParam *qp_d = pl.shared ? nullptr : carve<QParam>(cur, (size_t)nq);
    int32_t *perm_d = pl.shared ? nullptr : carve<int32_t>(cur, (size_t)nq);
    float *Qg = mixed ? carve<float>(cur, (size_t)C * ix->D) : nullptr;
    int64_t *ids_t = mixed ? carve<int64_t>(cur, (size_t)C * KO) : nullptr;
    float *d2_t = mixed ? carve<float>(cur, (size_t)C * KO) : nullptr;
    crisp_query_stats *st_t = mixed && stats ? carve<crisp_query_stats>(cur, C) : nullptr;
    std::vector<QParam> qp_perm;
    if (!pl.shared) {
        qp_perm.resize((size_t)nq);
        for (int32_t i = 0; i < nq; ++i) qp_perm[i] = pl.qp[perm[i]];
        cudaError_t e = cudaMemcpyAsync(qp_d, qp_perm.data(), sizeof(QParam) * nq, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(perm_d, perm.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st);
        // the host vectors are read by the copies: wait for them before returning
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = crisp_cuda_fail(e, "per-query parameters", __FILE__, __LINE__);
    }
    const QParam &q0 = pl.q0;   // scalars of the shared case (per-query batches read qp instead)
    for (int32_t c0 = 0; c0 < nq && s == CRISP_OK; c0 += C) {
        const int32_t nc = std::min(C, nq - c0);
        const QParam *qpc = pl.shared ? nullptr : qp_d + c0;
        const float *Qc = Q + (int64_t)c0 * ix->D;
        if (mixed) {
            s = launch_gather_rows(Q, ix->D, perm_d + c0, nc, Qg, st);
            Qc = Qg;
        }
        if (!s) {
            if (ix->rotated) s = crisp_rotate_rows(Qc, nc, ix->D, ix->D, ix->R32, Qr, ix->Dp, st);
            else s = launch_pad_rows(Qc, nc, ix->D, ix->D, Qr, ix->Dp, st);
        }
        if (!s) s = crisp_run_activate(ix, Qr, nc, q0.phi, q0.k, q0.budget, act, nact, retr, st, cfirst, clast, qpc);
        if (!s) s = crisp_run_count_cut(ix, act, nact, nc, q0.tau, q0.k, q0.cap, cand, ST, ncand, score, how, st, qpc);
        int64_t *ids_o = mixed ? ids_t : ids + (int64_t)c0 * KO;
        float *d2_o = mixed ? d2_t : d2 + (int64_t)c0 * KO;
        crisp_query_stats *st_o = stats ? (mixed ? st_t : stats + c0) : nullptr;
        // stage 3, one run per class segment of the chunk
        for (int32_t a = 0; a < nc && s == CRISP_OK;) {
            const int cls = pl.shared ? pl.cls0 : pcls[c0 + a];
            int32_t b = a + 1;
            if (pl.shared) b = nc;
            else while (b < nc && pcls[c0 + b] == cls) ++b;
            const int32_t n = b - a;
            const QParam *qa = qpc ? qpc + a : nullptr;
            const float *Qra = Qr + (int64_t)a * ix->Dp;
            const int32_t *ca = cand + (int64_t)a * ST;
            const int64_t *na = ncand + a;
            float *da = dist + (int64_t)a * ST;
            int64_t *io = ids_o + (int64_t)a * KO;
            float *dout = d2_o + (int64_t)a * KO;
            crisp_query_stats *so = st_o ? st_o + a : nullptr;
            if (cls == 4) {
                // F1: features -> MLP depths -> score prefix -> BF16 shortlist -> FP32 re-rank
                const uint8_t *sa = score + (int64_t)a * ST;
                s = crisp_run_features(ix, ca, ST, na, sa, cfirst + (int64_t)a * M, clast + (int64_t)a * M, n, q0.k,
                                       q0.tau, feats + (int64_t)a * F, st, qa);
                if (!s) s = crisp_run_mlp_depth(ix, feats + (int64_t)a * F, n, na, ST, q0.k, q0.mV, q0.mS, dV + a,
                                                dS + a, st, qa);
                if (!s) s = crisp_run_select_score(ca, ST, na, sa, dV + a, n, selV + (int64_t)a * ST, nsel + a, st);
                if (!s) s = crisp_run_shortlist(ix, Qra, n, selV + (int64_t)a * ST, ST, nsel + a, 1, 1, da,
                                                cand + (int64_t)a * ST, ST, nshort + a, st, dS + a, nullptr);
                // shortlists are short whatever the list stride: stream them per query
                if (!s) s = crisp_run_rerank(ix, Qra, n, cand + (int64_t)a * ST, ST, nshort + a, q0.k, da, io, dout,
                                             st, false, false, qa, KO);
                if (!s && so)
                    s = launch_write_stats(n, na, how + a, retr + (int64_t)a * M, M, nsel + a, nshort + a, q0.tau, so,
                                           st, qa);
            } else if (cls == 1 || cls == 2) {
                // F2: coarse-score every candidate on the low-precision rows, then the
                // FP32 re-rank of the shortlist
                int32_t *sa = shortl + (int64_t)a * SM;
                s = crisp_run_shortlist(ix, Qra, n, ca, ST, na, cls, q0.S, da, sa, SM, nshort + a, st, nullptr, qa);
                if (!s) s = crisp_run_rerank(ix, Qra, n, sa, SM, nshort + a, q0.k, da, io, dout, st, false, true, qa, KO);
                if (!s && so)
                    s = launch_write_stats(n, na, how + a, retr + (int64_t)a * M, M, na, nshort + a, q0.tau, so, st, qa);
            } else if (cls == 0) {
                s = crisp_run_rerank(ix, Qra, n, ca, ST, na, q0.k, da, io, dout, st, false, true, qa, KO);
                if (!s && so)
                    s = launch_write_stats(n, na, how + a, retr + (int64_t)a * M, M, nullptr, nullptr, q0.tau, so, st,
                                           qa);
            } else {
                s = crisp_run_verify_opt(ix, Qra, n, ca, ST, na, q0.k, q0.eps0, q0.patience, q0.order, io, dout,
                                         nver + a, nfull + a, nullptr, st, qa, KO);
                if (!s && so)
                    s = launch_write_stats(n, na, how + a, retr + (int64_t)a * M, M, nver + a, nfull + a, q0.tau, so,
                                           st, qa);
            }
            a = b;
        }
        if (!s && mixed)
            s = launch_scatter_results(ids_t, d2_t, st_t, KO, perm_d + c0, nc, ids, d2, stats, st);
    }
    crisp_scratch_free(base, st);
    return s;
}

extern "C" crisp_status crisp_search(const crisp_index *ix, const float *Q, int32_t nq, const crisp_search_params *p,
                                     int32_t p_count, int64_t *ids, float *sqdist, int32_t kmax,
                                     crisp_query_stats *stats, void *stream) {
    return search_device(ix, Q, nq, p, p_count, ids, sqdist, kmax, stats, as_stream(stream));
}

extern "C" crisp_status crisp_search_host(const crisp_index *ix, const float *Q, int32_t nq,
                                          const crisp_search_params *p, int32_t p_count, int64_t *ids, float *sqdist,
                                          int32_t kmax, crisp_query_stats *stats, void *stream) {
    SearchPlan pl;
    crisp_status s = plan_search(ix, nq, p, p_count, kmax, &pl);
    if (s) return s;
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Q && ids && sqdist, "crisp_search_host: null pointer");
    cudaStream_t st = as_stream(stream);
    const int32_t KO = pl.kmax;
    size_t qb = sizeof(float) * (size_t)nq * ix->D, ib = sizeof(int64_t) * (size_t)nq * KO,
           db = sizeof(float) * (size_t)nq * KO, sb = stats ? sizeof(crisp_query_stats) * (size_t)nq : 0;
    uint8_t *buf = nullptr;
    size_t tot = (qb + 255) / 256 * 256 + (ib + 255) / 256 * 256 + (db + 255) / 256 * 256 + (sb + 255) / 256 * 256;
    CRISP_CK(crisp_scratch_alloc((void **)&buf, tot, st));
    uint8_t *cur = buf;
    float *dQ = carve<float>(cur, (size_t)nq * ix->D);
    int64_t *dI = carve<int64_t>(cur, (size_t)nq * KO);
    float *dD = carve<float>(cur, (size_t)nq * KO);
    crisp_query_stats *dS = stats ? carve<crisp_query_stats>(cur, nq) : nullptr;
    cudaError_t e = cudaMemcpyAsync(dQ, Q, qb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = crisp_cuda_fail(e, "cudaMemcpyAsync(Q)", __FILE__, __LINE__);
    if (!s) s = search_device(ix, dQ, nq, p, p_count, dI, dD, KO, dS, st);
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
    crisp_status s = plan_search(ix, nq, &g, 1, 0, &pl);
    if (s) return s;
    const QParam &q0 = pl.q0;
    if (nq == 0) return CRISP_OK;
    CRISP_REQUIRE(Q && features && labels, "crisp_learned_data: null pointer");
    cudaStream_t st = as_stream(stream);
    const int64_t K2 = (int64_t)ix->K * ix->K;
    const int32_t M = ix->M, F = 2 * M + 68, k = q0.k;
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
        if (!s) s = crisp_run_activate(ix, Qr, nc, 0, k, q0.budget, act, nact, retr, st, cfirst, clast);
        if (!s) s = crisp_run_count_cut(ix, act, nact, nc, q0.tau, k, q0.cap, cand, pl.stride, ncand, score, how, st);
        if (!s) s = crisp_run_features(ix, cand, pl.stride, ncand, score, cfirst, clast, nc, k, q0.tau,
                                       features + (int64_t)c0 * F, st);
        if (!s) s = crisp_run_rerank(ix, Qr, nc, cand, pl.stride, ncand, k, dist, top, topd, st);
        if (!s) s = crisp_run_labels_v(cand, pl.stride, ncand, score, top, k, nc, dV, st);
        if (!s) s = crisp_run_select_score(cand, pl.stride, ncand, score, dV, nc, selV, nsel, st);
        // coarse distances of the whole prefix (keep all of it), then the coarse label
        if (!s) s = crisp_run_shortlist(ix, Qr, nc, selV, pl.stride, nsel, 1, 1, dist, cand, pl.stride, nshort, st,
                                        nsel, nullptr);
        if (!s) s = crisp_run_labels_s(selV, pl.stride, nsel, dist, top, k, nc, dS, st);
        if (!s) s = crisp_run_log2_targets(dV, dS, nc, labels + 2 * (int64_t)c0,
                                           targets ? targets + 2 * (int64_t)c0 : nullptr, st);
    }
    crisp_scratch_free(base, st);
    return s;
}
