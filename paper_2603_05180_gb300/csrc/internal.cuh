// Internal declarations of the CRISP GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "crisp.h"

// Ids per counting tile: the per-query collision counters of one tile live in
// shared memory as bytes, so a tile of 2^16 ids takes 64 KB.
#define CRISP_TILE_LOG2 16
#define CRISP_TILE (1 << CRISP_TILE_LOG2)
#define CRISP_KMAX 64
#define CRISP_KOUT_MAX 256
#define CRISP_OPT_MAX_CAND 32768
#define CRISP_GROUP_MAXQ 16384   // largest batch the grouped scorers order (one CTA sorts its keys)

struct crisp_index {
    int64_t N = 0;
    int32_t D = 0, Dp = 0, M = 0, K = 0, H = 0, rotated = 0;
    double cev = 0.0;
    int32_t max_cell = 0;
    int32_t T = 0;                 // number of id tiles
    float *R32 = nullptr;          // [D][D]
    float *cent = nullptr;         // [M][2][K][H]
    int32_t *offsets = nullptr;    // [M][K*K+1]
    int32_t *ids = nullptr;        // [M][N] (+ 4 zero entries: 16-byte quad reads)
    int32_t *tile_off = nullptr;   // [M][K*K][T+1]
    float *Xr = nullptr;           // [N][Dp]
    uint32_t *codes = nullptr;     // [N][Dp/32]
    uint16_t *Xb = nullptr;        // [N][Dp] BF16 bits (optional)
    uint8_t *X8 = nullptr;         // [N][Dp] FP8 E4M3 codes (optional)
    float *S8 = nullptr;           // [N] FP8 row scales (optional)
    float *xn2 = nullptr;          // [N] |x|^2 of the stored rows, FP64 sum rounded to FP32
    float *xbn2 = nullptr;         // [N] |xb|^2 of the BF16 copy (widened), FP64 sum rounded to FP32
    float *mlp = nullptr;          // learned-depth model (F = 2M + 68 -> H -> H -> 2), optional
    int32_t mlp_H = 0;
    int32_t *sub = nullptr;        // [M+1] subspace boundaries (device)
    std::vector<int32_t> sub_h;    // the same boundaries on the host
    int32_t block_dims = 0;        // block-wise rotation: block width (0: global test)
    int32_t rotated_blocks = 0;    // blocks rotated by the block-wise test
    int device = 0;
    int64_t bytes = 0;
};

// Plain-old-data view of an index handed to kernels by value.
struct IxView {
    int64_t N;
    int32_t D, Dp, M, K, H, T;
    const float *cent;
    const int32_t *offsets;
    const int32_t *ids;
    const int32_t *tile_off;
    const float *Xr;
    const uint32_t *codes;
    const uint16_t *Xb;
    const uint8_t *X8;
    const float *S8;
    const float *xn2;
    const int32_t *sub;
};

static inline IxView ix_view(const crisp_index *ix) {
    IxView v;
    v.N = ix->N; v.D = ix->D; v.Dp = ix->Dp; v.M = ix->M; v.K = ix->K; v.H = ix->H; v.T = ix->T;
    v.cent = ix->cent; v.offsets = ix->offsets; v.ids = ix->ids; v.tile_off = ix->tile_off;
    v.Xr = ix->Xr; v.codes = ix->codes;
    v.Xb = ix->Xb; v.X8 = ix->X8; v.S8 = ix->S8;
    v.xn2 = ix->xn2;
    v.sub = ix->sub;
    return v;
}

// Search parameters of one query as the kernels read them (per-query batches:
// crisp_search with p_count = nq).  Kernels given a null QParam array use their
// scalar arguments for every query.
struct QParam {
    int32_t k;          // neighbours (k_size)
    int32_t phi;        // 1: rank weights of Optimized mode
    int32_t tau;        // collision threshold
    int32_t order;      // Optimized verification order (0 Hamming, 1 id)
    int64_t budget;     // ids retrieved per subspace
    int64_t cap;        // candidate cap (0: none)
    int64_t patience;   // Optimized: P = patience_factor k (0: never stop)
    float eps0;         // Optimized: ADSampling margin
    float mV, mS;       // Learned: depth margins
    int32_t S;          // coarse scoring: shortlist size
};

// ------------------------------------------------------- launch accounting
extern std::atomic<unsigned long long> g_crisp_launches;
#define CRISP_COUNT_LAUNCH() g_crisp_launches.fetch_add(1, std::memory_order_relaxed)

// ---------------------------------------------------------------- errors
void crisp_set_error(const char *fmt, ...);
crisp_status crisp_cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define CRISP_CK(call)                                                          \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) return crisp_cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define CRISP_CK_LAUNCH() CRISP_CK(cudaGetLastError())

#define CRISP_REQUIRE(cond, ...)                                                \
    do {                                                                        \
        if (!(cond)) { crisp_set_error(__VA_ARGS__); return CRISP_EINVAL; }     \
    } while (0)

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------- host-side readings
int32_t crisp_tau(double alpha, int32_t M);
int64_t crisp_budget(double rho, int64_t N);
void crisp_subspace(int32_t D, int32_t M, int32_t m, int32_t *lo, int32_t *hl, int32_t *hr);
// Boundaries of the equal split, sub[m] = floor(mD/M), sub[M] = D.
std::vector<int32_t> crisp_equal_bounds(int32_t D, int32_t M);
// Widest half over the subspaces [sub[m], sub[m+1]) (half widths floor(w/2), w - floor(w/2)).
int32_t crisp_bounds_half_max(const int32_t *sub, int32_t M);
// False (with the error set) unless sub[0] = 0, sub[M] = D and every width is in [2, 256].
bool crisp_bounds_valid(const int32_t *sub, int32_t D, int32_t M, const char *who);

// ------------------------------------------ stream-ordered scratch memory
// A memory pool per device that keeps its memory between calls.
cudaError_t crisp_scratch_alloc(void **p, size_t bytes, cudaStream_t st);
void crisp_scratch_free(void *p, cudaStream_t st);

// ------------------------------------------------ internal launchers
// Tensor-core cell assignment (tc.cu): cells [M][N], or per-half centroid
// indices asg [2M][N] when asg is not null.  Synchronous on st.
// sub: host [M+1] subspace boundaries.
// Xb (optional): the BF16 copy of Xr; given, the scores come from one BF16 pass.
crisp_status crisp_tc_assign(const float *Xr, int64_t N, int32_t D, int32_t Dp, int32_t M, int32_t K, int32_t H,
                             const int32_t *sub, const float *cent, uint16_t *cells, int32_t *asg, cudaStream_t st,
                             const uint16_t *Xb = nullptr);
// X' = X R on the tensor cores writing only Y[:, 0:ncols] (ncols <= D rounded up to 32).
crisp_status crisp_rotate_rows_tc_cols(const float *X, int64_t N, int32_t D, int32_t ldx, const float *R, float *Y,
                                       int32_t ldy, int32_t ncols, cudaStream_t st);
crisp_status launch_pad_rows(const float *X, int64_t N, int32_t D, int32_t ldx, float *Y, int32_t ldy,
                             cudaStream_t st);
crisp_status launch_tile_offsets(crisp_index *ix, cudaStream_t st);
crisp_status launch_row_norms(crisp_index *ix, cudaStream_t st);
crisp_status launch_row_norms_bf16(crisp_index *ix, cudaStream_t st);
crisp_status launch_write_stats(int32_t nq, const int64_t *ncand, const int32_t *how, const int64_t *retrieved,
                                int32_t M, const int64_t *nver, const int64_t *nfull, int32_t tau,
                                crisp_query_stats *stats, cudaStream_t st, const QParam *qp = nullptr);
