// Tensor-core (tcgen05) contractions of the index build.
//
//   k_rotate_tc   B2  X' = X R (the adaptive rotation of §4.1 applied to every
//                     row), a dense N x D x D contraction on the 5th-generation
//                     tensor cores.  FP32 accuracy from the TF32 pipe by the
//                     three-product split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
//                     where a_hi is a with its low 13 mantissa bits cleared and
//                     a_lo = a - a_hi (exact in FP32).
//
// Data movement: the rows of X and of R^T (split into hi / lo once, D x D) are
// fetched by TMA (cp.async.bulk.tensor) as 128-row x 32-float boxes in the
// 128-byte swizzled layout that tcgen05.mma reads directly; the X tile is split
// in shared memory (hi in place, lo beside it) by the CTA's threads.  One
// thread issues the MMAs into a 128 x BN FP32 accumulator in tensor memory
// (TMEM) and signals stage reuse through tcgen05.commit -> mbarrier; the four
// warps then read their 32 TMEM lanes (one output row per thread) with
// tcgen05.ld and store the rows.  Every mbarrier wait is bounded in time: a
// wait that gives up records an error word, the CTA skips the rest of its
// work, waits (bounded) for what it still has in flight, frees its TMEM and
// returns, and the host reports CRISP_ECUDA.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched from the driver at run time)

#include <mutex>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace {

constexpr int TC_BM = 128;      // output rows per tile = UMMA M
constexpr int TC_BK = 32;       // floats per k-block: one 128-byte swizzle row
constexpr int TC_NT = 128;      // four warps
constexpr int TC_TMEM_COLS = 256;

__device__ unsigned int g_tc_error;   // first failing wait: 1 + its site code

__device__ __forceinline__ void record_error(unsigned int site) { atomicCAS(&g_tc_error, 0u, 1u + site); }

struct RotArgs {
    long long N;      // rows of X and Y
    int nk;           // k-blocks of 32 over the contraction (ceil(D / 32))
    int BN;           // output columns per tile (multiple of 16, <= 256)
    int nt;           // column tiles
    int ncols;        // output columns written (Y[:, 0:ncols])
    int ldy;
    int vec;          // 1: Y rows 16-byte aligned (float4 stores)
    float *Y;
};

// One CTA per (128-row tile, column tile); column tiles of a row tile are
// adjacent in launch order so the X tile is read from HBM about once.
__global__ void __launch_bounds__(TC_NT, 1) k_rotate_tc(const __grid_constant__ CUtensorMap tmX,
                                                        const __grid_constant__ CUtensorMap tmBh,
                                                        const __grid_constant__ CUtensorMap tmBl, RotArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    const uint32_t A_BYTES = TC_BM * 128, B_BYTES = (uint32_t)a.BN * 128;
    const uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
    uint64_t *bars = (uint64_t *)(sm + 2 * STAGE);     // full[2], empty[2], done
    uint32_t *tmem_slot = (uint32_t *)(bars + 5);
    int *abort_flag = (int *)(bars + 6);
    auto sA = [&](int s) { return sm + s * STAGE; };
    auto sAlo = [&](int s) { return sm + s * STAGE + A_BYTES; };
    auto sBh = [&](int s) { return sm + s * STAGE + 2 * A_BYTES; };
    auto sBl = [&](int s) { return sm + s * STAGE + 2 * A_BYTES + B_BYTES; };
    const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[2]), done = smem_addr(&bars[4]);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ct = (int)(blockIdx.x % (unsigned)a.nt);
    const long long row0 = (long long)(blockIdx.x / (unsigned)a.nt) * TC_BM;
    const int col0 = ct * a.BN;
    const int nk = a.nk;

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(smem_addr(&bars[i]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // loads issued / consumed (thread 0 keeps the count of issued ones)
    int issued = 0;
    auto issue = [&](int kb) {
        const int s = kb & 1;
        const uint32_t fb = full0 + 8u * s;
        mbar_expect_tx(fb, A_BYTES + 2 * B_BYTES);
        tma_load_2d(smem_addr(sA(s)), &tmX, kb * TC_BK, (int)row0, fb);
        tma_load_2d(smem_addr(sBh(s)), &tmBh, kb * TC_BK, col0, fb);
        tma_load_2d(smem_addr(sBl(s)), &tmBl, kb * TC_BK, col0, fb);
    };
    if (tid == 0)
        for (; issued < 2 && issued < nk; ++issued) issue(issued);

    const uint32_t idesc = tf32_idesc(a.BN, TC_BM);
    int consumed = 0;
    for (int kb = 0; kb < nk; ++kb) {
        const int s = kb & 1;
        const uint32_t ph = (uint32_t)(kb >> 1) & 1u;
        if (!mbar_wait(full0 + 8u * s, ph)) {
            record_error(0);
            *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) break;
        consumed = kb + 1;
        // split the X tile: hi (low 13 mantissa bits cleared) in place, lo = x - hi beside it
        float4 *pa = (float4 *)sA(s);
        float4 *pl = (float4 *)sAlo(s);
#pragma unroll 4
        for (int i = tid; i < TC_BM * TC_BK / 4; i += TC_NT) {
            float4 v = pa[i], h;
            h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
            h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
            h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
            h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
            pl[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            pa[i] = h;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 32) {
            tc_fence_after();
            const uint32_t ah = smem_addr(sA(s)), al = smem_addr(sAlo(s)), bh = smem_addr(sBh(s)),
                           bl = smem_addr(sBl(s));
#pragma unroll
            for (int j = 0; j < TC_BK / 8; ++j) {   // UMMA K = 8 floats = 32 bytes
                const uint32_t o = 32u * j;
                mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bh + o), idesc, (kb | j) != 0);
                mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1);
                mma_tf32(tmem, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1);
            }
            mma_commit(empty0 + 8u * s);
        }
        if (tid == 0 && issued < nk) {
            // stage s is free again once the MMAs just issued have read it
            if (mbar_wait(empty0 + 8u * s, ph)) {
                issue(issued);
                ++issued;
            } else {
                record_error(1);
                *abort_flag = 1;
            }
        }
    }
    // every MMA issued so far completes before the accumulator is read or freed
    if (tid == 32) mma_commit(done);
    if (!mbar_wait(done, 0)) {
        record_error(2);
        *abort_flag = 1;
    }
    __syncthreads();
    const bool ok = !*abort_flag;   // the same for every thread: tcgen05.ld below is warp-collective
    tc_fence_after();
    if (ok) {
        const long long r = row0 + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < a.BN; c += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + (uint32_t)c, v);        // all 32 lanes of the warp take part
            const int gc = col0 + c;
            if (r >= a.N || gc >= a.ncols) continue;
            float *y = a.Y + r * (long long)a.ldy + gc;
            if (a.vec && gc + 16 <= a.ncols) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    reinterpret_cast<float4 *>(y)[q] =
                        make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                    __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            } else {
                for (int q = 0; q < 16 && gc + q < a.ncols; ++q) y[q] = __uint_as_float(v[q]);
            }
        }
    }
    // loads still in flight after an abort land before the CTA's shared memory goes away
    if (tid == 0)
        for (int kb = consumed; kb < issued; ++kb)
            if (!mbar_wait(full0 + 8u * (kb & 1), (uint32_t)(kb >> 1) & 1u)) record_error(3);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// BT_hi / BT_lo [Dp][Dp]: BT[n][k] = R[k][n] split into hi + lo, zero outside D x D.
__global__ void k_split_rt(const float *__restrict__ R, int D, int Dp, float *__restrict__ hi, float *__restrict__ lo) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Dp * Dp) return;
    int n = (int)(e / Dp), k = (int)(e % Dp);
    float v = (n < D && k < D) ? R[(long long)k * D + n] : 0.0f;
    float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    hi[e] = h;
    lo[e] = v - h;
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

// 2-D FP32 map over rows x cols (row pitch ld floats), box 32 floats x box_rows,
// 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap *m, const float *base, long long rows, int cols, int ld, int box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// 2-D FP32 tensor map for other translation units (box 32 floats x box_rows,
// 128-byte swizzle): the tensor-core re-rank fetches its rows and queries with it.
bool crisp_make_map_f32(CUtensorMap *m, const float *base, long long rows, int cols, int ld, int box_rows) {
    return make_map(m, base, rows, cols, ld, box_rows);
}

// 2-D BF16 tensor map over rows x cols (row pitch ld elements), box 64
// elements (128 bytes) x box_rows, 128-byte swizzle, zero fill outside.
bool crisp_make_map_bf16(CUtensorMap *m, const uint16_t *base, long long rows, int cols, int ld, int box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(uint16_t)};
    cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

size_t rot_smem(int BN) { return 1024 + 2 * (2 * (size_t)TC_BM * 128 + 2 * (size_t)BN * 128) + 64; }

}  // namespace

extern "C" crisp_status crisp_rotate_rows_tc(const float *X, int64_t N, int32_t D, int32_t ldx, const float *R, float *Y,
                                             int32_t ldy, void *stream) {
    return crisp_rotate_rows_tc_cols(X, N, D, ldx, R, Y, ldy, -1, as_stream(stream));
}

// ncols < 0: Y[:, 0:min(ldy, Dp)] with columns D.. zero; else Y[:, 0:ncols] only
// (a block of columns inside a wider row).
crisp_status crisp_rotate_rows_tc_cols(const float *X, int64_t N, int32_t D, int32_t ldx, const float *R, float *Y,
                                       int32_t ldy, int32_t ncols_req, cudaStream_t st) {
    CRISP_REQUIRE(N >= 0 && D >= 1 && ldx >= D && ldy >= D, "crisp_rotate_rows_tc: bad sizes");
    CRISP_REQUIRE(N == 0 || (X && R && Y), "crisp_rotate_rows_tc: null pointer");
    CRISP_REQUIRE((const void *)X != (const void *)Y, "crisp_rotate_rows_tc: Y overlaps X");
    CRISP_REQUIRE(((uintptr_t)X % 16) == 0 && ((size_t)ldx * sizeof(float)) % 16 == 0,
                  "crisp_rotate_rows_tc: X must be 16-byte aligned with a row pitch of a multiple of 4 floats");
    if (N == 0) return CRISP_OK;
    const int Dp = (D + TC_BK - 1) / TC_BK * TC_BK;
    const int ncols = ncols_req >= 0 ? std::min(ncols_req, ldy < Dp ? ldy : Dp)
                                     : (ldy < Dp ? ldy : Dp);   // columns D..ncols-1 come out zero
    if (ncols <= 0) return CRISP_OK;
    const int nt = (ncols + 255) / 256;
    const int BN = ((ncols + nt - 1) / nt + 15) / 16 * 16;
    float *bt = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&bt, sizeof(float) * 2 * (size_t)Dp * Dp, st));
    crisp_status s = CRISP_OK;
    do {
        k_split_rt<<<(unsigned)(((long long)Dp * Dp + 255) / 256), 256, 0, st>>>(R, D, Dp, bt, bt + (size_t)Dp * Dp);
        CRISP_COUNT_LAUNCH();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_split_rt", __FILE__, __LINE__); break; }
        CUtensorMap mx, mh, ml;
        if (!make_map(&mx, X, N, D, ldx, TC_BM) || !make_map(&mh, bt, Dp, Dp, Dp, BN) ||
            !make_map(&ml, bt + (size_t)Dp * Dp, Dp, Dp, Dp, BN)) {
            crisp_set_error("crisp_rotate_rows_tc: tensor map encoding failed");
            s = CRISP_ECUDA;
            break;
        }
        const size_t smem = rot_smem(BN);
        e = cudaFuncSetAttribute(k_rotate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__); break; }
        unsigned int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "reset error word", __FILE__, __LINE__); break; }
        RotArgs a;
        a.N = N;
        a.nk = Dp / TC_BK;
        a.BN = BN;
        a.nt = nt;
        a.ncols = ncols;
        a.ldy = ldy;
        a.vec = ((uintptr_t)Y % 16 == 0) && (ldy % 4 == 0);
        a.Y = Y;
        const long long tiles = (N + TC_BM - 1) / TC_BM * nt;
        if (tiles > 0x7FFFFFFFLL) {
            crisp_set_error("crisp_rotate_rows_tc: too many rows");
            s = CRISP_EINVAL;
            break;
        }
        k_rotate_tc<<<(unsigned)tiles, TC_NT, smem, st>>>(mx, mh, ml, a);
        CRISP_COUNT_LAUNCH();
        e = cudaGetLastError();
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_rotate_tc", __FILE__, __LINE__); break; }
        if (ncols_req < 0 && ldy > ncols) {   // full rows: the columns past the output are zeroed
            e = cudaMemset2DAsync(Y + ncols, sizeof(float) * (size_t)ldy, 0, sizeof(float) * (size_t)(ldy - ncols),
                                  (size_t)N, st);
            if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaMemset2DAsync", __FILE__, __LINE__); break; }
        }
        unsigned int err = 0;
        e = cudaMemcpyFromSymbolAsync(&err, g_tc_error, sizeof err, 0, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_rotate_tc", __FILE__, __LINE__); break; }
        if (err) {
            crisp_set_error("crisp_rotate_rows_tc: a pipeline wait timed out (site %u)", err - 1);
            s = CRISP_ECUDA;
        }
    } while (0);
    cudaFreeAsync(bt, st);
    return s;
}

// ============================================================================
//   k_assign_tc   B3  u_m(x) = Combine(argmin_left, argmin_right) for every row
//                     and subspace (§3 IMI cells).  The tensor cores (TF32, one
//                     pass) give every row its scores s_c = |c|^2 - 2 x.c against
//                     the K centroids of both halves; each score is within a
//                     proven bound E_c of the exact |x - c|^2 - |x|^2, so only
//                     centroids with s_c - E_c <= min(s + E) can be the argmin.
//                     Those few are re-measured with the FP32 SEQ distance (an
//                     fmaf chain over the half's dims, ties to the lowest index),
//                     which makes the result identical to crisp_assign_cells.
//
// Operand layout: the subspace's columns of Xr come by TMA as 32-float k-blocks
// starting at the 32-aligned column below the subspace; the centroids sit in a
// prepared matrix whose row c (one per centroid, 64 rows per half) holds c at
// the same columns and zeros elsewhere, so columns outside a half contribute
// nothing.  Two 128 x 64 FP32 accumulators (left, right) live in TMEM.
namespace {

constexpr int AS_KPAD = 64;     // centroid rows per half (K <= 64)

struct AsgArgs {
    long long N;
    int D, Dp, M, K, H, KB;
    const float *Xr;
    const int32_t *sub;     // [M+1] subspace boundaries
    const float *cent;      // [M][2][K][H]
    const float *cn2;       // [M][2][64] |c|^2 (FP32)
    const float *cn;        // [M][2][64] |c|
    uint16_t *cells;        // [M][N] cell ids, or (when asg is set)
    int *asg;               // [2M][N] per-half centroid indices (k-means)
};

// TF32 score error bound (both operands truncated to 10 mantissa bits, FP32
// accumulation) plus the FP32 rounding of the exact distances, generously.
template <bool BF>
__device__ __forceinline__ float asg_bound(float nx, float nx2, float c, float c2) {
    // BF16 (both operands rounded to nearest, 2^-9 each): each product within
    // (2^-8 + 2^-18) |x_i c_i|, the FP32 accumulation of h <= 128 dims in K = 16
    // steps within 3.6e-5 |x| |c|: |score~ - score| <= 7.9e-3 |x| |c|; 1.2e-2
    // with margin, plus the same rounding term as TF32
    if (BF) return 1.2e-2f * nx * c + 1e-4f * (nx2 + c2) + 1e-30f;
    return 6e-3f * nx * c + 1e-4f * (nx2 + c2);
}

// Dynamic shared memory: two 32 KB stages (X tile, left and right centroid
// tiles), the subspace's centroids [2][K][HS], |c|^2 and |c| [2][64], barriers.
__host__ __device__ constexpr uint32_t asg_stage_bytes() { return TC_BM * 128 + 2 * AS_KPAD * 128; }
__host__ __device__ inline size_t asg_smem_bytes(int K, int HS) {
    return 1024 + 2 * (size_t)asg_stage_bytes() + sizeof(float) * (2 * (size_t)K * HS + 4 * AS_KPAD) + 64;
}

// BF = false: one TF32 pass over the FP32 rows (k-blocks of 32 floats);
// BF = true: one BF16 pass over the rows' BF16 copy against BF16 centroids
// (k-blocks of 64 elements).  The exact re-measure reads the FP32 rows either way.
template <bool BF>
__global__ void __launch_bounds__(TC_NT) k_assign_tc(const __grid_constant__ CUtensorMap tmX,
                                                     const __grid_constant__ CUtensorMap tmB, AsgArgs a) {
    constexpr int KE = BF ? 64 : TC_BK;                               // elements per 128-byte k-block
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    uint8_t *sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);   // swizzled tiles need 1024-byte alignment
    constexpr uint32_t A_BYTES = TC_BM * 128, B_BYTES = AS_KPAD * 128, STAGE = asg_stage_bytes();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = (int)(blockIdx.x % (unsigned)a.M);
    const long long row0 = (long long)(blockIdx.x / (unsigned)a.M) * TC_BM;
    const int lo = a.sub[m], hi_ = a.sub[m + 1];
    const int hl = (hi_ - lo) / 2, hr = (hi_ - lo) - hl, HS = hr;     // hr >= hl
    const int base = lo & ~(KE - 1);
    const int nk = (hi_ - base + KE - 1) / KE;
    float *sC = (float *)(sm + 2 * STAGE);                             // [2][K][HS]
    float *sN2 = sC + 2 * a.K * HS, *sN1 = sN2 + 2 * AS_KPAD;           // [2][64] each
    uint64_t *bars = (uint64_t *)(sN1 + 2 * AS_KPAD);                  // full[2], empty[2], done
    uint32_t *tmem_slot = (uint32_t *)(bars + 5);
    int *abort_flag = (int *)(bars + 6);
    const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[2]), done = smem_addr(&bars[4]);

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(smem_addr(&bars[i]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(2 * AS_KPAD)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int last_use[2] = {-1, -1};   // producer: last k-block loaded into each stage
    auto issue = [&](int kb) {
        const int s = kb & 1;
        const uint32_t fb = full0 + 8u * s;
        uint8_t *st = sm + s * STAGE;
        mbar_expect_tx(fb, STAGE);
        tma_load_2d(smem_addr(st), &tmX, base + kb * KE, (int)row0, fb);
        tma_load_2d(smem_addr(st + A_BYTES), &tmB, kb * KE, (m * 2 + 0) * AS_KPAD, fb);
        tma_load_2d(smem_addr(st + A_BYTES + B_BYTES), &tmB, kb * KE, (m * 2 + 1) * AS_KPAD, fb);
        last_use[s] = kb;
    };
    if (tid == 0) {
        int issued = 0;
        for (; issued < 2 && issued < nk; ++issued) issue(issued);
        for (int kb = 0; issued < nk; ++kb, ++issued) {
            // reuse stage kb & 1 once the MMAs of k-block kb have read it
            if (!mbar_wait(empty0 + 8u * (kb & 1), (uint32_t)(kb >> 1) & 1u)) {
                record_error(10);
                break;
            }
            issue(issued);
        }
    } else if (tid == 32) {
        const uint32_t idesc = BF ? bf16_idesc(AS_KPAD, TC_BM) : tf32_idesc(AS_KPAD, TC_BM);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb & 1;
            if (!mbar_wait(full0 + 8u * s, (uint32_t)(kb >> 1) & 1u)) {
                record_error(11);
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_addr(sm + s * STAGE), sl = sa + A_BYTES, sr = sa + A_BYTES + B_BYTES;
#pragma unroll
            for (int j = 0; j < 4; ++j) {   // four 32-byte K steps per 128-byte k-block
                const uint32_t o = 32u * j, acc = (kb | j) != 0;
                if (BF) {
                    mma_bf16(tmem, sw128_desc(sa + o), sw128_desc(sl + o), idesc, acc);
                    mma_bf16(tmem + AS_KPAD, sw128_desc(sa + o), sw128_desc(sr + o), idesc, acc);
                } else {
                    mma_tf32(tmem, sw128_desc(sa + o), sw128_desc(sl + o), idesc, acc);
                    mma_tf32(tmem + AS_KPAD, sw128_desc(sa + o), sw128_desc(sr + o), idesc, acc);
                }
            }
            mma_commit(empty0 + 8u * s);
        }
        mma_commit(done);
    }
    // while the tiles load: the subspace's centroids and their norms into shared memory
    for (int e = tid; e < 2 * a.K * HS; e += TC_NT) {
        const int half = e / (a.K * HS), rem = e % (a.K * HS), c = rem / HS, d = rem % HS;
        const int h = half ? hr : hl;
        sC[e] = d < h ? a.cent[(((long long)m * 2 + half) * a.K + c) * a.H + d] : 0.0f;
    }
    for (int e = tid; e < 2 * AS_KPAD; e += TC_NT) {
        sN2[e] = a.cn2[m * 2 * AS_KPAD + e];
        sN1[e] = a.cn[m * 2 * AS_KPAD + e];
    }
    if (!mbar_wait(done, 0)) {
        record_error(12);
        *abort_flag = 1;
    }
    __syncthreads();
    const bool ok = !*abort_flag;
    tc_fence_after();
    if (ok) {
        const int rl = warp * 32 + lane;                 // row within the tile = TMEM lane
        const long long r = row0 + rl;
        const bool live = r < a.N;
        // the row's subspace values: from the resident tiles when the subspace
        // spans at most the two stages, else from global memory
        const bool resident = !BF && nk <= 2;            // BF16 tiles: the FP32 values come from global memory
        const float *xg = a.Xr + (live ? r : 0) * (long long)a.Dp + lo;
        auto xval = [&](int j) -> float {               // j: column relative to lo
            if (!resident) return xg[j];
            const int jj = lo - base + j;
            const float *tile = (const float *)(sm + (jj >> 5) * STAGE);
            return tile[rl * 32 + ((((jj & 31) >> 2) ^ (rl & 7)) << 2) + (jj & 3)];
        };
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        int arg[2];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int off = half ? hl : 0, h = half ? hr : hl;
            const float *C = sC + half * a.K * HS;
            const float *c2 = sN2 + half * AS_KPAD, *c1 = sN1 + half * AS_KPAD;
            float nx2 = 0.0f;
            for (int d = 0; d < h; ++d) {
                const float t = xval(off + d);
                nx2 = fmaf(t, t, nx2);
            }
            const float nx = sqrtf(nx2);
            float U = INFINITY;
            for (int c0 = 0; c0 < AS_KPAD; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(lane_base + (uint32_t)(half * AS_KPAD + c0), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c0 + q;
                    if (c < a.K) {
                        const float sc = c2[c] - 2.0f * __uint_as_float(v[q]);
                        U = fminf(U, sc + asg_bound<BF>(nx, nx2, c1[c], c2[c]));
                    }
                }
            }
            float best = INFINITY;
            int bc = 0;
            for (int c0 = 0; c0 < AS_KPAD; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(lane_base + (uint32_t)(half * AS_KPAD + c0), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c0 + q;
                    if (c >= a.K) continue;
                    const float sc = c2[c] - 2.0f * __uint_as_float(v[q]);
                    if (!(sc - asg_bound<BF>(nx, nx2, c1[c], c2[c]) <= U)) continue;
                    const float *cc = C + c * HS;
                    float acc = 0.0f;
                    for (int d = 0; d < h; ++d) {
                        const float diff = xval(off + d) - cc[d];
                        acc = fmaf(diff, diff, acc);
                    }
                    if (acc < best) {   // ascending c: the first minimum wins ties
                        best = acc;
                        bc = c;
                    }
                }
            }
            arg[half] = bc;
        }
        if (live) {
            if (a.asg) {
                a.asg[(2LL * m) * a.N + r] = arg[0];
                a.asg[(2LL * m + 1) * a.N + r] = arg[1];
            } else {
                a.cells[(long long)m * a.N + r] = (uint16_t)(arg[0] * a.K + arg[1]);
            }
        }
    }
    if (tid == 0)
        for (int s = 0; s < 2; ++s)
            if (last_use[s] >= 0 && !mbar_wait(full0 + 8u * s, (uint32_t)(last_use[s] >> 1) & 1u)) record_error(13);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * AS_KPAD) : "memory");
    }
}

// Bm [M][2][64][KB*KE]: row c of half h holds centroid c at the Xr columns of
// that half (relative to the subspace's KE-aligned base column), zeros
// elsewhere, FP32 (KE = 32) or rounded to BF16 (KE = 64); cn2 / cn: |c|^2 and
// |c| of the FP32 centroids (zero rows past K).
template <bool BF>
__global__ void k_asg_prep(const float *__restrict__ cent, const int32_t *__restrict__ sub, int M, int K, int H, int KB,
                           void *__restrict__ Bm, float *__restrict__ cn2, float *__restrict__ cn) {
    constexpr int KE = BF ? 64 : TC_BK;
    const int W = KB * KE;
    const long long tot = (long long)M * 2 * AS_KPAD * W;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % W);
        const long long rowi = e / W;
        const int c = (int)(rowi % AS_KPAD), half = (int)((rowi / AS_KPAD) % 2), m = (int)(rowi / (2 * AS_KPAD));
        const int lo = sub[m], hi_ = sub[m + 1];
        const int hl = (hi_ - lo) / 2, hr = (hi_ - lo) - hl;
        const int start = lo + (half ? hl : 0) - (lo & ~(KE - 1)), h = half ? hr : hl;
        float v = 0.0f;
        if (c < K && j >= start && j < start + h) v = cent[(((long long)m * 2 + half) * K + c) * H + (j - start)];
        if (BF) reinterpret_cast<uint16_t *>(Bm)[e] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        else reinterpret_cast<float *>(Bm)[e] = v;
        if (j == 0) {
            float s = 0.0f;
            if (c < K)
                for (int d = 0; d < h; ++d) {
                    const float t = cent[(((long long)m * 2 + half) * K + c) * H + d];
                    s = fmaf(t, t, s);
                }
            cn2[rowi] = s;
            cn[rowi] = sqrtf(s);
        }
    }
}

}  // namespace

crisp_status crisp_tc_assign(const float *Xr, int64_t N, int32_t D, int32_t Dp, int32_t M, int32_t K, int32_t H,
                             const int32_t *sub, const float *cent, uint16_t *cells, int32_t *asg, cudaStream_t st,
                             const uint16_t *Xb) {
    CRISP_REQUIRE(Xr && sub && cent && (cells || asg), "crisp_assign_cells_tc: null pointer");
    CRISP_REQUIRE(K >= 2 && K <= AS_KPAD && M >= 1 && 2 * M <= D && Dp >= D && N >= 1 && H >= 1,
                  "crisp_assign_cells_tc: bad sizes");
    CRISP_REQUIRE(Dp % TC_BK == 0 && ((uintptr_t)Xr % 16) == 0 && ((uintptr_t)Xb % 16) == 0,
                  "crisp_assign_cells_tc: Xr (and Xb) must be 16-byte aligned with Dp a multiple of 32");
    CRISP_REQUIRE(crisp_bounds_valid(sub, D, M, "crisp_assign_cells_tc") && crisp_bounds_half_max(sub, M) <= H,
                  "crisp_assign_cells_tc: subspace boundaries do not fit H = %d", H);
    const bool bf = Xb != nullptr;
    const int KE = bf ? 64 : TC_BK;                 // elements per 128-byte k-block
    int KB = 1, HS = 1;
    for (int m = 0; m < M; ++m) {
        const int lo = sub[m], hi_ = sub[m + 1];
        KB = std::max(KB, (hi_ - (lo & ~(KE - 1)) + KE - 1) / KE);
        HS = std::max(HS, (hi_ - lo) - (hi_ - lo) / 2);
    }
    const size_t bm_n = (size_t)M * 2 * AS_KPAD * KB * KE, nn = (size_t)M * 2 * AS_KPAD;
    const size_t bm_bytes = (bm_n * (bf ? 2 : 4) + 255) / 256 * 256;
    uint8_t *buf = nullptr;
    CRISP_CK(cudaMallocAsync((void **)&buf, bm_bytes + sizeof(float) * 2 * nn + sizeof(int32_t) * ((size_t)M + 1), st));
    void *Bm = buf;
    float *cn2 = (float *)(buf + bm_bytes), *cn = cn2 + nn;
    int32_t *dsub = (int32_t *)(cn + nn);
    const std::vector<int32_t> hsub(sub, sub + M + 1);   // pageable: the copy is staged before return
    crisp_status s = CRISP_OK;
    do {
        cudaError_t e = cudaMemcpyAsync(dsub, hsub.data(), sizeof(int32_t) * hsub.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__); break; }
        const unsigned pg = (unsigned)std::min<size_t>((bm_n + 255) / 256, 4096);
        if (bf) k_asg_prep<true><<<pg, 256, 0, st>>>(cent, dsub, M, K, H, KB, Bm, cn2, cn);
        else k_asg_prep<false><<<pg, 256, 0, st>>>(cent, dsub, M, K, H, KB, Bm, cn2, cn);
        CRISP_COUNT_LAUNCH();
        e = cudaGetLastError();
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_asg_prep", __FILE__, __LINE__); break; }
        CUtensorMap mx, mb;
        const bool mapped =
            bf ? crisp_make_map_bf16(&mx, Xb, N, Dp, Dp, TC_BM) &&
                     crisp_make_map_bf16(&mb, (const uint16_t *)Bm, (long long)M * 2 * AS_KPAD, KB * KE, KB * KE, AS_KPAD)
               : make_map(&mx, Xr, N, Dp, Dp, TC_BM) &&
                     make_map(&mb, (const float *)Bm, (long long)M * 2 * AS_KPAD, KB * KE, KB * KE, AS_KPAD);
        if (!mapped) {
            crisp_set_error("crisp_assign_cells_tc: tensor map encoding failed");
            s = CRISP_ECUDA;
            break;
        }
        const size_t smem = asg_smem_bytes(K, HS);
        e = bf ? cudaFuncSetAttribute(k_assign_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
               : cudaFuncSetAttribute(k_assign_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__); break; }
        unsigned int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "reset error word", __FILE__, __LINE__); break; }
        const long long tiles = (N + TC_BM - 1) / TC_BM * M;
        if (tiles > 0x7FFFFFFFLL) {
            crisp_set_error("crisp_assign_cells_tc: too many rows");
            s = CRISP_EINVAL;
            break;
        }
        AsgArgs a{N, D, Dp, M, K, H, KB, Xr, dsub, cent, cn2, cn, cells, asg};
        if (bf) k_assign_tc<true><<<(unsigned)tiles, TC_NT, smem, st>>>(mx, mb, a);
        else k_assign_tc<false><<<(unsigned)tiles, TC_NT, smem, st>>>(mx, mb, a);
        CRISP_COUNT_LAUNCH();
        e = cudaGetLastError();
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_assign_tc", __FILE__, __LINE__); break; }
        unsigned int err = 0;
        e = cudaMemcpyFromSymbolAsync(&err, g_tc_error, sizeof err, 0, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = crisp_cuda_fail(e, "k_assign_tc", __FILE__, __LINE__); break; }
        if (err) {
            crisp_set_error("crisp_assign_cells_tc: a pipeline wait timed out (site %u)", err - 1);
            s = CRISP_ECUDA;
        }
    } while (0);
    cudaFreeAsync(buf, st);
    return s;
}

extern "C" crisp_status crisp_assign_cells_tc(const float *Xr, const uint16_t *Xb, int64_t N, int32_t D, int32_t Dp,
                                              int32_t M, int32_t K, int32_t H, const int32_t *sub, const float *cent,
                                              uint16_t *cells, void *stream) {
    CRISP_REQUIRE(cells && M >= 1, "crisp_assign_cells_tc: null pointer or M < 1");
    const std::vector<int32_t> eq = crisp_equal_bounds(D, M);
    return crisp_tc_assign(Xr, N, D, Dp, M, K, H, sub ? sub : eq.data(), cent, cells, nullptr, as_stream(stream), Xb);
}
