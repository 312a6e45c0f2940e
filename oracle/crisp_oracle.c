/*
 * crisp_oracle.c -- plain, slow CPU oracle of CRISP (arXiv 2603.05180).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the GPU product path never
 * does, and this file shares no code, header or table with it.
 *
 * Every function follows one passage of the paper, cited beside it.  Points
 * the paper leaves open are fixed by the readings listed in the design notes
 * (budget rounding, tie orders, the canonical FP32 summation orders below).
 *
 * Floating point.  Values that decide an integer -- a k-means argmin, the
 * multi-sequence visiting order, an ADSampling prune, a top-k membership --
 * are computed in FP32 in a fixed order, so that a GPU kernel computing in the
 * same precision can be compared bit for bit:
 *   SEQ  : acc = 0; for i in order: diff = a_i - b_i; acc = fmaf(diff, diff, acc)
 *   CR32 : per 32-dim block b, eight partial sums a_l (l = 0..7), each an fmaf
 *          chain over dims 32b+4l .. 32b+4l+3; block sum
 *          s_b = ((a0+a4)+(a2+a6)) + ((a1+a5)+(a3+a7)); prefix d_{32(b+1)} =
 *          d_{32b} + s_b from d_0 = 0.  Dims past D are zero on both sides.
 *   GEMV : y_j = fmaf chain over d = 0..D-1 of x_d * R[d][j], from 0.
 * FP64 is used where the paper's step is a statistic (covariance, means).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ index */
typedef struct {
    int64_t N;
    int32_t D, Dp, M, K, H, rotated, _pad;
    const float *R32;        /* [D][D], y = x R  (§3, §4.1); NULL if not rotated */
    const float *cent;       /* [M][2][K][H]  IMI codebooks per subspace half (§3, §4.2) */
    const int32_t *offsets;  /* [M][K*K+1]    CSR Offsets (§4.2) */
    const int32_t *ids;      /* [M][N]        CSR Vectors IDs (§4.2) */
    const float *Xr;         /* [N][Dp]       stored (rotated when triggered) rows */
    const uint32_t *codes;   /* [N][Dp/32]    sign codes b(x) (§3 Binary Quantization) */
    const uint16_t *Xb;      /* [N][Dp]       BF16 copy (coarse scoring), or NULL */
    const uint8_t *X8;       /* [N][Dp]       FP8 E4M3 copy, or NULL */
    const float *S8;         /* [N]           FP8 row scales, or NULL */
    const float *mlp;        /* learned depth model (F = 2M + 68 -> H -> H -> 2), or NULL */
    int32_t mlp_H, _pad2;
    const int32_t *sub;      /* [M+1] subspace boundaries (adaptive decomposition), or NULL = equal split */
} or_index;

typedef struct {
    int32_t k, mode;         /* mode: 0 Guaranteed (phi=0), 1 Optimized (phi=1) */
    double rho, alpha;       /* coverage fraction; minimum-collision fraction */
    int32_t patience_factor; /* P = patience_factor * k (§4.3.2 Stage 3); <= 0 disables */
    float eps0;              /* ADSampling margin (Eq. 2) */
    int64_t max_candidates;  /* 0 = no cap */
    int32_t precision;       /* Guaranteed mode coarse scoring: 0 none, 1 BF16, 2 FP8 E4M3 */
    int32_t shortlist;       /* candidates kept by the coarse score for the FP32 re-rank */
    float depth_margin;      /* learned mode: margins added to the predicted log2 depths */
    float short_margin;
    int32_t verify_order;    /* Optimized mode: 0 by (Hamming, id) (§4.3.2 Stage 2), 1 by id (ablation) */
    int32_t _pad;
} or_params;

typedef struct {
    int64_t n_candidates, n_verified, n_full, n_retrieved;
    int32_t fallback, capped, tau, _pad;
} or_stats;

/* Subspace m of M over D dims: [floor(mD/M), floor((m+1)D/M)), left half the
 * first floor(d/2) dims (§3 Subspace Collision Framework, IMI halves). */
void or_subspace(int D, int M, int m, int *lo, int *hl, int *hr) {
    int a = (int)(((int64_t)m * D) / M), b = (int)(((int64_t)(m + 1) * D) / M);
    int d = b - a;
    *lo = a;
    *hl = d / 2;
    *hr = d - d / 2;
}

/* Subspace m given explicit boundaries sub[0..M] (subspace m covers dims
 * [sub[m], sub[m+1])), or the equal split of or_subspace when sub is NULL;
 * halves as in or_subspace (the adaptive decomposition of §7 changes only
 * where the subspaces start and end). */
void or_subspace_b(const int32_t *sub, int D, int M, int m, int *lo, int *hl, int *hr) {
    if (!sub) { or_subspace(D, M, m, lo, hl, hr); return; }
    int d = sub[m + 1] - sub[m];
    *lo = sub[m];
    *hl = d / 2;
    *hr = d - d / 2;
}

/* tau = ceil(alpha*M) (Theorem 1, tau = alpha M), evaluated so that 0.3*10 is 3. */
int or_tau(double alpha, int M) { return (int)ceil(alpha * (double)M - 1e-9); }

/* budget = max(1, ceil(rho*N)) ids per subspace (Algorithm 1, "retrieved < budget"). */
int64_t or_budget(double rho, int64_t N) {
    int64_t b = (int64_t)ceil(rho * (double)N - 1e-9);
    return b < 1 ? 1 : b;
}

/* ----------------------------------------------------------- FP32 orders */
float or_seq_sqdist(const float *a, const float *b, int n) {
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) {
        float diff = a[i] - b[i];
        acc = fmaf(diff, diff, acc);
    }
    return acc;
}

/* CR32 block sums s_b, b < Dp/32 (Dp a multiple of 32, padded dims zero). */
void or_cr32_blocks(const float *x, const float *q, int Dp, float *s) {
    for (int b = 0; b < Dp / 32; ++b) {
        float a[8];
        for (int l = 0; l < 8; ++l) {
            float acc = 0.0f;
            for (int e = 0; e < 4; ++e) {
                int d = 32 * b + 4 * l + e;
                float diff = x[d] - q[d];
                acc = fmaf(diff, diff, acc);
            }
            a[l] = acc;
        }
        s[b] = ((a[0] + a[4]) + (a[2] + a[6])) + ((a[1] + a[5]) + (a[3] + a[7]));
    }
}

/* Full CR32 squared distance over Dp dims. */
float or_cr32(const float *x, const float *q, int Dp) {
    float s[Dp / 32 > 0 ? Dp / 32 : 1];
    or_cr32_blocks(x, q, Dp, s);
    float acc = 0.0f;
    for (int b = 0; b < Dp / 32; ++b) acc = acc + s[b];
    return acc;
}

/* y = x R in the GEMV order (Q1 / B2): y_j is an fmaf chain over d = 0..D-1
 * of x_d R[d][j], from 0.  The d loop is outermost so R streams by rows; every
 * y_j still sees its terms in ascending d.  x has D entries, y gets Dp. */
void or_rotate_row(const float *x, const float *R, int D, int Dp, float *y) {
    for (int j = 0; j < Dp; ++j) y[j] = 0.0f;
    for (int d = 0; d < D; ++d) {
        const float xd = x[d];
        const float *r = R + (int64_t)d * D;
        for (int j = 0; j < D; ++j) y[j] = fmaf(xd, r[j], y[j]);
    }
}

void or_rotate_rows(const float *X, int64_t N, int D, int ldx, const float *R, int Dp, float *Y) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) or_rotate_row(X + n * ldx, R, D, Dp, Y + n * Dp);
}

/* Copy rows into the padded layout without rotation (CEV <= tau_CEV path, §4.1). */
void or_pad_rows(const float *X, int64_t N, int D, int ldx, int Dp, float *Y) {
    for (int64_t n = 0; n < N; ++n) {
        memcpy(Y + n * Dp, X + n * ldx, sizeof(float) * D);
        for (int j = D; j < Dp; ++j) Y[n * Dp + j] = 0.0f;
    }
}

/* -------------------------------------------------- B1: covariance (§4.1) */
/* Sample covariance of the rows listed in `rows`, mean-centred, 1/(S-1), FP64. */
void or_covariance(const float *X, int64_t N, int D, int ldx, const int64_t *rows, int64_t S, double *cov) {
    (void)N;
    double *mu = (double *)calloc((size_t)D, sizeof(double));
    for (int64_t s = 0; s < S; ++s)
        for (int d = 0; d < D; ++d) mu[d] += (double)X[rows[s] * ldx + d];
    for (int d = 0; d < D; ++d) mu[d] /= (double)S;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < D; ++i) {
        for (int j = i; j < D; ++j) {
            double acc = 0.0;
            for (int64_t s = 0; s < S; ++s) {
                const float *x = X + rows[s] * ldx;
                acc += ((double)x[i] - mu[i]) * ((double)x[j] - mu[j]);
            }
            cov[(int64_t)i * D + j] = acc / (double)(S - 1);
            cov[(int64_t)j * D + i] = acc / (double)(S - 1);
        }
    }
    free(mu);
}

/* ----------------------------------------------- B3: k-means per half (§4.2) */
static int argmin_seq(const float *x, const float *C, int K, int H, int h) {
    int best = 0;
    float bd = or_seq_sqdist(x, C, h);
    for (int c = 1; c < K; ++c) {
        float d = or_seq_sqdist(x, C + (int64_t)c * H, h);
        if (d < bd) { bd = d; best = c; }      /* ties keep the lowest index */
    }
    return best;
}

/* Lloyd's k-means on the rows of a training matrix T (S rows, stride ldt), over
 * dims [off, off+h).  C is [K][H] (row stride H >= h), initialised from the
 * training rows `init` and updated `iters` times; an empty cluster keeps its
 * centroid.  Means are accumulated in FP64 and rounded to FP32. */
void or_kmeans(const float *T, int64_t S, int ldt, int off, int h, int K, int H,
               const int32_t *init, int iters, float *C) {
    for (int c = 0; c < K; ++c) {
        for (int d = 0; d < H; ++d) C[(int64_t)c * H + d] = d < h ? T[(int64_t)init[c] * ldt + off + d] : 0.0f;
    }
    int *asg = (int *)malloc(sizeof(int) * (size_t)(S > 0 ? S : 1));
    double *sum = (double *)malloc(sizeof(double) * (size_t)K * h);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < S; ++s) asg[s] = argmin_seq(T + s * ldt + off, C, K, H, h);
        memset(sum, 0, sizeof(double) * (size_t)K * h);
        memset(cnt, 0, sizeof(int64_t) * (size_t)K);
        for (int64_t s = 0; s < S; ++s) {
            const float *x = T + s * ldt + off;
            cnt[asg[s]]++;
            for (int d = 0; d < h; ++d) sum[(int64_t)asg[s] * h + d] += (double)x[d];
        }
        for (int c = 0; c < K; ++c)
            if (cnt[c] > 0)
                for (int d = 0; d < h; ++d) C[(int64_t)c * H + d] = (float)(sum[(int64_t)c * h + d] / (double)cnt[c]);
    }
    free(asg);
    free(sum);
    free(cnt);
}

/* Cell u_m(x) = Combine(argmin_left, argmin_right) = cL*K + cR for every row
 * and subspace (§3 u(x); §4.2 cells = K x K).  cells is [M][N]. */
void or_assign_cells(const float *Xr, int64_t N, int D, int Dp, int M, int K, int H,
                     const float *cent, const int32_t *sub, uint16_t *cells) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            int lo, hl, hr;
            or_subspace_b(sub, D, M, m, &lo, &hl, &hr);
            const float *x = Xr + n * Dp + lo;
            const float *CL = cent + ((int64_t)m * 2 + 0) * K * H;
            const float *CR = cent + ((int64_t)m * 2 + 1) * K * H;
            int cl = argmin_seq(x, CL, K, H, hl);
            int cr = argmin_seq(x + hl, CR, K, H, hr);
            cells[(int64_t)m * N + n] = (uint16_t)(cl * K + cr);
        }
    }
}

/* ------------------------------------------------------- B4: CSR (§4.2) */
/* (cell, id) tuples sorted by cell, ids ascending within a cell (the worked
 * example of §4.2); Offsets has K^2+1 entries, ids has N. */
void or_csr(const uint16_t *cells, int64_t N, int K2, int32_t *offsets, int32_t *ids) {
    memset(offsets, 0, sizeof(int32_t) * (size_t)(K2 + 1));
    for (int64_t n = 0; n < N; ++n) offsets[cells[n] + 1]++;
    for (int c = 0; c < K2; ++c) offsets[c + 1] += offsets[c];
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)K2);
    memcpy(cur, offsets, sizeof(int32_t) * (size_t)K2);
    for (int64_t n = 0; n < N; ++n) ids[cur[cells[n]]++] = (int32_t)n;
    free(cur);
}

/* ------------------------------------------- B5: sign codes (§3 BQ) */
void or_sign_codes(const float *Xr, int64_t N, int Dp, uint32_t *codes) {
    int W = Dp / 32;
    for (int64_t n = 0; n < N; ++n)
        for (int w = 0; w < W; ++w) {
            uint32_t v = 0;
            for (int b = 0; b < 32; ++b)
                if (Xr[n * Dp + 32 * w + b] > 0.0f) v |= 1u << b;
            codes[n * W + w] = v;
        }
}

/* --------------------------- Q2: partial distances + sorted half lists */
/* Dist1 / Dist2 of Algorithm 1 for subspace m, half `half` (0 left, 1 right),
 * each sorted ascending with ties by centroid index. */
void or_half_dists(const or_index *ix, const float *qr, int m, int half, float *dist, float *sorted, int32_t *perm) {
    int lo, hl, hr;
    or_subspace_b(ix->sub, ix->D, ix->M, m, &lo, &hl, &hr);
    int h = half ? hr : hl;
    const float *qh = qr + lo + (half ? hl : 0);
    const float *C = ix->cent + ((int64_t)m * 2 + half) * ix->K * ix->H;
    for (int c = 0; c < ix->K; ++c) dist[c] = or_seq_sqdist(qh, C + (int64_t)c * ix->H, h);
    for (int c = 0; c < ix->K; ++c) perm[c] = c;
    for (int a = 1; a < ix->K; ++a) {          /* insertion sort by (dist, index) */
        int32_t p = perm[a];
        int b = a - 1;
        while (b >= 0 && (dist[perm[b]] > dist[p] || (dist[perm[b]] == dist[p] && perm[b] > p))) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = p;
    }
    for (int c = 0; c < ix->K; ++c) sorted[c] = dist[perm[c]];
}

/* ------------------------- Q3: multi-sequence activation (Algorithm 1, §4.3.1) */
typedef struct { float cost; int32_t i, j; } msq_key;

static int key_less(msq_key a, msq_key b) {
    if (a.cost != b.cost) return a.cost < b.cost;
    if (a.i != b.i) return a.i < b.i;
    return a.j < b.j;
}

static void heap_push(msq_key *h, int *n, msq_key v) {
    int c = (*n)++;
    h[c] = v;
    while (c > 0) {
        int p = (c - 1) / 2;
        if (!key_less(h[c], h[p])) break;
        msq_key t = h[c]; h[c] = h[p]; h[p] = t;
        c = p;
    }
}

static msq_key heap_pop(msq_key *h, int *n) {
    msq_key top = h[0];
    h[0] = h[--(*n)];
    int c = 0;
    for (;;) {
        int l = 2 * c + 1, r = l + 1, s = c;
        if (l < *n && key_less(h[l], h[s])) s = l;
        if (r < *n && key_less(h[r], h[s])) s = r;
        if (s == c) break;
        msq_key t = h[c]; h[c] = h[s]; h[s] = t;
        c = s;
    }
    return top;
}

/* Visit cells of subspace m in ascending (cost, i, j) with a priority queue,
 * cost = Dist1s[i] + Dist2s[j] in FP32, until `retrieved >= budget`; a popped
 * cell is consumed whole.  rank counts pops (empty cells included); the weight
 * is 2 when phi = 1 and rank <= k, else 1.  Writes the popped cells (original
 * centroid indices combined as cL*K + cR) and weights in pop order; returns
 * the number popped and the ids retrieved in *retrieved. */
int or_activate_heap_costs(const or_index *ix, const float *qr, int m, int phi, int k, int64_t budget,
                           int32_t *cells, uint8_t *w, int64_t *retrieved, float *cost_first, float *cost_last);

int or_activate_heap(const or_index *ix, const float *qr, int m, int phi, int k, int64_t budget,
                     int32_t *cells, uint8_t *w, int64_t *retrieved) {
    return or_activate_heap_costs(ix, qr, m, phi, k, budget, cells, w, retrieved, NULL, NULL);
}

/* As or_activate_heap, also reporting the cost of the first and the last
 * visited cell (learned-mode features). */
int or_activate_heap_costs(const or_index *ix, const float *qr, int m, int phi, int k, int64_t budget,
                           int32_t *cells, uint8_t *w, int64_t *retrieved, float *cost_first, float *cost_last) {
    int K = ix->K;
    float d1[256], d2[256], s1[256], s2[256];
    int32_t p1[256], p2[256];
    or_half_dists(ix, qr, m, 0, d1, s1, p1);
    or_half_dists(ix, qr, m, 1, d2, s2, p2);
    int32_t rowlen[256];
    memset(rowlen, 0, sizeof rowlen);
    msq_key *heap = (msq_key *)malloc(sizeof(msq_key) * (size_t)(K * K + 1));
    int hn = 0, npop = 0, rank = 0;
    int64_t got = 0;
    const int32_t *off = ix->offsets + (int64_t)m * (K * K + 1);
    msq_key k0 = {s1[0] + s2[0], 0, 0};
    heap_push(heap, &hn, k0);
    while (got < budget && hn > 0) {
        msq_key t = heap_pop(heap, &hn);
        int cell = p1[t.i] * K + p2[t.j];
        if (rank == 0 && cost_first) *cost_first = t.cost;
        if (cost_last) *cost_last = t.cost;
        rank += 1;
        cells[npop] = cell;
        w[npop] = (uint8_t)((phi == 1 && rank <= k) ? 2 : 1);
        npop++;
        got += off[cell + 1] - off[cell];
        rowlen[t.i] = t.j + 1;
        /* next candidates: (i+1, j) once (i+1, j-1) is popped; (i, j+1) once (i-1, j+1) is */
        if (t.i + 1 < K && (t.j == 0 || rowlen[t.i + 1] >= t.j)) {
            msq_key v = {s1[t.i + 1] + s2[t.j], t.i + 1, t.j};
            heap_push(heap, &hn, v);
        }
        if (t.j + 1 < K && (t.i == 0 || rowlen[t.i - 1] > t.j + 1)) {
            msq_key v = {s1[t.i] + s2[t.j + 1], t.i, t.j + 1};
            heap_push(heap, &hn, v);
        }
    }
    free(heap);
    *retrieved = got;
    return npop;
}

static int key_cmp(const void *a, const void *b) {
    msq_key x = *(const msq_key *)a, y = *(const msq_key *)b;
    return key_less(x, y) ? -1 : (key_less(y, x) ? 1 : 0);
}

/* Second, independent form of the same order: sort all K^2 keys, walk the prefix. */
int or_activate_sorted(const or_index *ix, const float *qr, int m, int phi, int k, int64_t budget,
                       int32_t *cells, uint8_t *w, int64_t *retrieved) {
    int K = ix->K;
    float d1[256], d2[256], s1[256], s2[256];
    int32_t p1[256], p2[256];
    or_half_dists(ix, qr, m, 0, d1, s1, p1);
    or_half_dists(ix, qr, m, 1, d2, s2, p2);
    msq_key *all = (msq_key *)malloc(sizeof(msq_key) * (size_t)(K * K));
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) { all[i * K + j].cost = s1[i] + s2[j]; all[i * K + j].i = i; all[i * K + j].j = j; }
    qsort(all, (size_t)K * K, sizeof(msq_key), key_cmp);
    const int32_t *off = ix->offsets + (int64_t)m * (K * K + 1);
    int64_t got = 0;
    int n = 0;
    while (got < budget && n < K * K) {
        int cell = p1[all[n].i] * K + p2[all[n].j];
        cells[n] = cell;
        w[n] = (uint8_t)((phi == 1 && n + 1 <= k) ? 2 : 1);
        got += off[cell + 1] - off[cell];
        n++;
    }
    free(all);
    *retrieved = got;
    return n;
}

/* --------------------------------------- Q4: collision counting (Eq. 1) */
/* List walk: V[id] += w for every id of every activated cell (Algorithm 1). */
void or_scores_walk(const or_index *ix, const int32_t *ncell, const int32_t *cells, const uint8_t *w, int32_t *V) {
    int K2 = ix->K * ix->K;
    memset(V, 0, sizeof(int32_t) * (size_t)ix->N);
    for (int m = 0; m < ix->M; ++m) {
        const int32_t *off = ix->offsets + (int64_t)m * (K2 + 1);
        const int32_t *ids = ix->ids + (int64_t)m * ix->N;
        for (int c = 0; c < ncell[m]; ++c) {
            int cell = cells[(int64_t)m * K2 + c];
            for (int32_t p = off[cell]; p < off[cell + 1]; ++p) V[ids[p]] += w[(int64_t)m * K2 + c];
        }
    }
}

/* Second form, straight from Eq. 1: for each point and subspace, add the weight
 * of its own cell u_m(x) if that cell is in the activated set U_m(q).
 * point_cell is [M][N] (u_m(x)). */
void or_scores_membership(const or_index *ix, const uint16_t *point_cell, const int32_t *ncell,
                          const int32_t *cells, const uint8_t *w, int32_t *V) {
    int K2 = ix->K * ix->K;
    uint8_t *act = (uint8_t *)malloc((size_t)K2);
    memset(V, 0, sizeof(int32_t) * (size_t)ix->N);
    for (int m = 0; m < ix->M; ++m) {
        memset(act, 0, (size_t)K2);
        for (int c = 0; c < ncell[m]; ++c) act[cells[(int64_t)m * K2 + c]] = w[(int64_t)m * K2 + c];
        for (int64_t n = 0; n < ix->N; ++n) V[n] += act[point_cell[(int64_t)m * ix->N + n]];
    }
    free(act);
}

/* ---------------------------------- Q5: threshold cut + fallback (Stage 1) */
typedef struct { int32_t v, id; } vid;
static int vid_cmp(const void *a, const void *b) {       /* V descending, id ascending */
    const vid *x = (const vid *)a, *y = (const vid *)b;
    if (x->v != y->v) return x->v > y->v ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}
static int i32_cmp(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : (x > y);
}

/* C = {x : V[x] >= tau} in ascending id.  If tau >= 1 and |C| < k, C becomes the
 * min(k, #{V >= 1}) points of highest (V, -id) ("robustness fallback").  If a
 * cap is set and |C| > cap, C keeps its cap points of highest (V, -id).
 * Returns |C|; *how = 0 plain, 1 fallback, 2 capped. */
int64_t or_cut(const int32_t *V, int64_t N, int tau, int k, int64_t cap, int32_t *C, int *how) {
    int64_t n = 0;
    *how = 0;
    for (int64_t x = 0; x < N; ++x)
        if (V[x] >= tau) C[n++] = (int32_t)x;
    int lo;
    int64_t want;
    if (tau >= 1 && n < k) { lo = 1; want = k; *how = 1; }
    else if (cap > 0 && n > cap) { lo = tau; want = cap; *how = 2; }
    else return n;
    int64_t m = 0;
    for (int64_t x = 0; x < N; ++x) if (V[x] >= lo) m++;
    vid *all = (vid *)malloc(sizeof(vid) * (size_t)(m > 0 ? m : 1));
    m = 0;
    for (int64_t x = 0; x < N; ++x) if (V[x] >= lo) { all[m].v = V[x]; all[m].id = (int32_t)x; m++; }
    qsort(all, (size_t)m, sizeof(vid), vid_cmp);
    int64_t take = m < want ? m : want;
    for (int64_t i = 0; i < take; ++i) C[i] = all[i].id;
    qsort(C, (size_t)take, sizeof(int32_t), i32_cmp);
    free(all);
    return take;
}

/* ------------------------------------------------------- top-k helpers */
/* Sorted (d, id) ascending list of at most k; returns 1 if (d, id) entered. */
static int topk_offer(float *td, int64_t *ti, int *size, int k, float d, int64_t id) {
    if (*size == k) {
        float wd = td[k - 1];
        int64_t wi = ti[k - 1];
        if (!(d < wd || (d == wd && id < wi))) return 0;
        (*size)--;
    }
    int p = *size;
    while (p > 0 && (td[p - 1] > d || (td[p - 1] == d && ti[p - 1] > id))) {
        td[p] = td[p - 1];
        ti[p] = ti[p - 1];
        --p;
    }
    td[p] = d;
    ti[p] = id;
    (*size)++;
    return 1;
}

/* ------------------------------ Q6: exact re-rank (Stage 3, phi = 0) */
/* Exact CR32 distance for every candidate; top-k by (d^2, id).  Pads with
 * id -1 and +inf.  Returns the number of results. */
int or_rerank(const or_index *ix, const float *qr, const int32_t *C, int64_t nC, int k, int64_t *ids, float *d2) {
    int size = 0;
    for (int64_t c = 0; c < nC; ++c) {
        float d = or_cr32(ix->Xr + (int64_t)C[c] * ix->Dp, qr, ix->Dp);
        topk_offer(d2, ids, &size, k, d, C[c]);
    }
    for (int i = size; i < k; ++i) { ids[i] = -1; d2[i] = INFINITY; }
    return size;
}

/* ------------------- Q7: Optimized verification (Stage 2 + Stage 3, phi = 1) */
typedef struct { int32_t ham, id; } hid;
static int hid_cmp(const void *a, const void *b) {
    const hid *x = (const hid *)a, *y = (const hid *)b;
    if (x->ham != y->ham) return x->ham < y->ham ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

/* ADSampling factor (t/D)(1 + eps0/sqrt(t))^2 of Eq. 2, evaluated in FP64 and
 * rounded to FP32; the prune test is d_t > fl(r_k^2 * factor). */
float or_ads_factor(int t, int D, float eps0) {
    double a = 1.0 + (double)eps0 / sqrt((double)t);
    return (float)(((double)t / (double)D) * (a * a));
}

/* Candidates ordered by (Hamming(b(q), b(x)), id); each verified in order by
 * ADSampling checks at t = 32, 64, ... < D against the current k-th distance
 * (active once the top-k holds k entries), else an exact distance and a top-k
 * offer; the patience counter grows on every candidate that leaves the top-k
 * unchanged, resets otherwise, and the walk stops once it reaches P. */
int or_verify_opt(const or_index *ix, const float *qr, const uint32_t *qcode, const int32_t *C, int64_t nC,
                  int k, float eps0, int64_t P, int order, int64_t *ids, float *d2, int64_t *n_verified,
                  int64_t *n_full) {
    int W = ix->Dp / 32, nb = ix->Dp / 32, D = ix->D;
    hid *ord = (hid *)malloc(sizeof(hid) * (size_t)(nC > 0 ? nC : 1));
    for (int64_t c = 0; c < nC; ++c) {
        const uint32_t *bx = ix->codes + (int64_t)C[c] * W;
        int ham = 0;
        for (int w = 0; w < W; ++w) ham += __builtin_popcount(bx[w] ^ qcode[w]);
        ord[c].ham = order ? 0 : ham;   /* order 1: the ablation without Hamming re-ranking (id order) */
        ord[c].id = C[c];
    }
    qsort(ord, (size_t)nC, sizeof(hid), hid_cmp);
    float *ft = (float *)malloc(sizeof(float) * (size_t)(nb > 0 ? nb : 1));
    for (int b = 0; b < nb; ++b) ft[b] = 32 * (b + 1) < D ? or_ads_factor(32 * (b + 1), D, eps0) : 0.0f;
    float *s = (float *)malloc(sizeof(float) * (size_t)(nb > 0 ? nb : 1));
    int size = 0;
    int64_t counter = 0, done = 0, full = 0;
    for (int64_t c = 0; c < nC; ++c) {
        const float *x = ix->Xr + (int64_t)ord[c].id * ix->Dp;
        or_cr32_blocks(x, qr, ix->Dp, s);
        int pruned = 0, changed = 0;
        float acc = 0.0f;
        int b = 0;
        if (size == k) {
            float r2 = d2[k - 1];
            for (; b < nb; ++b) {
                acc = acc + s[b];
                if (32 * (b + 1) >= D) { ++b; break; }
                if (acc > r2 * ft[b]) { pruned = 1; break; }
            }
        }
        if (!pruned) {
            for (; b < nb; ++b) acc = acc + s[b];
            full++;
            changed = topk_offer(d2, ids, &size, k, acc, ord[c].id);
        }
        counter = changed ? 0 : counter + 1;
        done++;
        if (P > 0 && counter >= P) break;
    }
    for (int i = size; i < k; ++i) { ids[i] = -1; d2[i] = INFINITY; }
    *n_verified = done;
    *n_full = full;
    free(ord);
    free(ft);
    free(s);
    return size;
}

/* ------------------------------------ F2: low-precision coarse scoring */
/* BF16 with round-to-nearest-even: the upper 16 bits of the FP32 pattern,
 * rounded on the lower 16 (ties to an even upper half).  Inputs are finite. */
uint16_t or_bf16_rne(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

float or_bf16_to_f32(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* OCP FP8 E4M3 ("fn" variant: no infinities, max finite 448), round to nearest
 * even, saturating to +-448.  Exponent bias 7, 3 mantissa bits; subnormals
 * m * 2^-9.  Inputs are finite. */
uint8_t or_e4m3_rne(float x) {
    uint8_t sign = x < 0.0f || (x == 0.0f && signbit(x)) ? 0x80 : 0x00;
    double a = fabs((double)x);
    if (a >= 448.0) return sign | 0x7E;
    /* candidate values are multiples of 2^(e-3) on [2^e, 2^(e+1)), e >= -6;
     * below 2^-6 the step is 2^-9 (subnormals) */
    int ex = 0;
    if (a > 0) frexp(a, &ex);           /* a = f 2^ex, f in [0.5, 1): binade 2^(ex-1) */
    int e = a > 0 ? ex - 1 : -7;
    if (e < -6) e = -6;
    double step = ldexp(1.0, e - 3);
    double q = a / step;                 /* exact: step is a power of two */
    double fl = floor(q);
    double r = q - fl;
    double m = fl;
    if (r > 0.5 || (r == 0.5 && fmod(fl, 2.0) == 1.0)) m = fl + 1.0;
    double v = m * step;                 /* the rounded magnitude */
    if (v >= 448.0) return sign | 0x7E;
    if (v == 0.0) return sign;
    int evx = 0;
    frexp(v, &evx);
    int ev = evx - 1;
    if (ev < -6) {                       /* subnormal: v = mant * 2^-9 */
        int mant = (int)(v / ldexp(1.0, -9));
        return sign | (uint8_t)mant;
    }
    int mant = (int)(v / ldexp(1.0, ev - 3)) - 8;
    return sign | (uint8_t)(((ev + 7) << 3) | mant);
}

float or_e4m3_to_f32(uint8_t c) {
    int s = c >> 7, e = (c >> 3) & 0xF, m = c & 7;
    double v = e == 0 ? m * ldexp(1.0, -9) : (8 + m) * ldexp(1.0, e - 10);
    return (float)(s ? -v : v);
}

/* Per-row scale s = fl(max|x| / 448) (1 if the row is zero); codes e4m3(fl(x / s)). */
void or_quantize_e4m3(const float *Xr, int64_t N, int Dp, uint8_t *X8, float *scale) {
    for (int64_t n = 0; n < N; ++n) {
        const float *x = Xr + n * Dp;
        float mx = 0.0f;
        for (int d = 0; d < Dp; ++d) mx = fabsf(x[d]) > mx ? fabsf(x[d]) : mx;
        float s = mx > 0.0f ? mx / 448.0f : 1.0f;
        scale[n] = s;
        for (int d = 0; d < Dp; ++d) X8[n * Dp + d] = or_e4m3_rne(x[d] / s);
    }
}

void or_quantize_bf16(const float *Xr, int64_t N, int Dp, uint16_t *Xb) {
    for (int64_t i = 0; i < N * (int64_t)Dp; ++i) Xb[i] = or_bf16_rne(Xr[i]);
}

/* Coarse distance of one candidate in the CR32 order, the row replaced by its
 * dequantised copy: BF16 widened exactly, or E4M3 code times the row scale. */
float or_prescore(const uint16_t *xb, const uint8_t *x8, float s8, const float *q, int Dp) {
    float x[Dp];
    for (int d = 0; d < Dp; ++d) x[d] = xb ? or_bf16_to_f32(xb[d]) : or_e4m3_to_f32(x8[d]) * s8;
    return or_cr32(x, q, Dp);
}

typedef struct { float d; int32_t id; } did;
static int did_cmp(const void *a, const void *b) {
    const did *x = (const did *)a, *y = (const did *)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

/* Shortlist: the S candidates of smallest (coarse distance, id), in ascending id.
 * Returns the shortlist length min(S, nC). */
int64_t or_shortlist(const uint16_t *Xb, const uint8_t *X8, const float *S8, int Dp, const float *qr, const int32_t *C,
                     int64_t nC, int64_t S, int32_t *out) {
    if (nC <= S) {
        memcpy(out, C, sizeof(int32_t) * (size_t)nC);
        return nC;
    }
    did *all = (did *)malloc(sizeof(did) * (size_t)nC);
    for (int64_t c = 0; c < nC; ++c) {
        int64_t id = C[c];
        all[c].d = Xb ? or_prescore(Xb + id * Dp, NULL, 0.0f, qr, Dp) : or_prescore(NULL, X8 + id * Dp, S8[id], qr, Dp);
        all[c].id = C[c];
    }
    qsort(all, (size_t)nC, sizeof(did), did_cmp);
    for (int64_t i = 0; i < S; ++i) out[i] = all[i].id;
    qsort(out, (size_t)S, sizeof(int32_t), i32_cmp);
    free(all);
    return S;
}

/* --------------------------- F1: learned re-rank depth (small MLP) */
/* erf by Abramowitz & Stegun 7.1.28 (|error| <= 3e-7): for a >= 0,
 * erf(a) = 1 - (1 + a1 a + ... + a6 a^6)^-16; odd extension.  Evaluated in
 * FP32 in a fixed order (Horner with fmaf, four squarings, one division). */
float or_erf_as(float u) {
    float a = fabsf(u);
    float p = 0.0000430638f;
    p = fmaf(p, a, 0.0002765672f);
    p = fmaf(p, a, 0.0001520143f);
    p = fmaf(p, a, 0.0092705272f);
    p = fmaf(p, a, 0.0422820123f);
    p = fmaf(p, a, 0.0705230784f);
    p = fmaf(p, a, 1.0f);
    float p2 = p * p, p4 = p2 * p2, p8 = p4 * p4, p16 = p8 * p8;
    float e = 1.0f - 1.0f / p16;
    return u < 0.0f ? -e : e;
}

/* GELU(z) = z/2 (1 + erf(z / sqrt 2)), erf as above. */
float or_gelu(float z) {
    float u = z * 0.70710678118654752f;
    return (0.5f * z) * (1.0f + or_erf_as(u));
}

/* MLP F -> H -> H -> O with GELU on both hidden layers; params packed as
 * W1 [F][H], b1 [H], W2 [H][H], b2 [H], W3 [H][O], b3 [O].  Every unit is an
 * fmaf chain over its inputs in order, starting from its bias. */
void or_mlp_infer(const float *P, int F, int H, int O, const float *x, float *y) {
    const float *W1 = P, *b1 = W1 + (int64_t)F * H, *W2 = b1 + H, *b2 = W2 + (int64_t)H * H, *W3 = b2 + H,
                *b3 = W3 + (int64_t)H * O;
    float h1[1024], h2[1024];
    for (int j = 0; j < H; ++j) {
        float z = b1[j];
        for (int i = 0; i < F; ++i) z = fmaf(x[i], W1[(int64_t)i * H + j], z);
        h1[j] = or_gelu(z);
    }
    for (int j = 0; j < H; ++j) {
        float z = b2[j];
        for (int i = 0; i < H; ++i) z = fmaf(h1[i], W2[(int64_t)i * H + j], z);
        h2[j] = or_gelu(z);
    }
    for (int o = 0; o < O; ++o) {
        float z = b3[o];
        for (int j = 0; j < H; ++j) z = fmaf(h2[j], W3[(int64_t)j * O + o], z);
        y[o] = z;
    }
}

/* Feature vector of one query (F = 2M + 68), IEEE basic operations only:
 *  [0, 64)        share of the candidates at each collision score (63 = 63 and above)
 *  [64, 64+M)     cost of the first visited cell of each subspace / sum of last costs
 *  [64+M, 64+2M)  cost of the last visited cell of each subspace / sum of last costs
 *  then |C|/N, floor(log2(|C|+1))/32, k/256, tau/M. */
void or_features(const int32_t *V, const int32_t *C, int64_t nC, int64_t N, const float *first_cost,
                 const float *last_cost, int M, int k, int tau, float *f) {
    int64_t cnt[64];
    memset(cnt, 0, sizeof cnt);
    for (int64_t c = 0; c < nC; ++c) {
        int v = V[C[c]];
        cnt[v < 63 ? v : 63]++;
    }
    float den = (float)(nC > 0 ? nC : 1);
    for (int s = 0; s < 64; ++s) f[s] = (float)cnt[s] / den;
    float norm = 0.0f;
    for (int m = 0; m < M; ++m) norm = norm + last_cost[m];
    if (!(norm > 0.0f)) norm = 1.0f;
    for (int m = 0; m < M; ++m) {
        f[64 + m] = first_cost[m] / norm;
        f[64 + M + m] = last_cost[m] / norm;
    }
    int64_t v = nC + 1;
    int lg = 0;
    while (v > 1) { v >>= 1; ++lg; }
    f[64 + 2 * M] = (float)nC / (float)N;
    f[64 + 2 * M + 1] = (float)lg / 32.0f;
    f[64 + 2 * M + 2] = (float)k / 256.0f;
    f[64 + 2 * M + 3] = (float)tau / (float)M;
}

/* depth = ceil(2^(j/4)), j = ceil(4 (y + margin)) in FP32, clamped to [lo, hi];
 * 2^(1/4) and 2^(1/2) from correctly rounded square roots. */
int64_t or_depth(float y, float margin, int64_t lo, int64_t hi) {
    float t = 4.0f * (y + margin);
    if (!(t < 120.0f)) return hi;                 /* also catches NaN */
    if (t < -120.0f) return lo;
    int j = (int)ceilf(t);
    int q = j >= 0 ? j / 4 : -((-j + 3) / 4);
    int r = j - 4 * q;                            /* 0..3 */
    double s2 = sqrt(2.0), s4 = sqrt(s2);
    double fr = r == 0 ? 1.0 : r == 1 ? s4 : r == 2 ? s2 : s2 * s4;
    double v = ceil(ldexp(fr, q));
    int64_t d = v > 9.0e18 ? hi : (int64_t)v;
    if (d < lo) d = lo;
    if (d > hi) d = hi;
    return d;
}

/* The first `depth` candidates by (V desc, id asc), returned in ascending id. */
int64_t or_select_by_score(const int32_t *V, const int32_t *C, int64_t nC, int64_t depth, int32_t *out) {
    if (depth >= nC) {
        memcpy(out, C, sizeof(int32_t) * (size_t)nC);
        return nC;
    }
    vid *all = (vid *)malloc(sizeof(vid) * (size_t)(nC > 0 ? nC : 1));
    for (int64_t c = 0; c < nC; ++c) { all[c].v = V[C[c]]; all[c].id = C[c]; }
    qsort(all, (size_t)nC, sizeof(vid), vid_cmp);
    for (int64_t i = 0; i < depth; ++i) out[i] = all[i].id;
    qsort(out, (size_t)depth, sizeof(int32_t), i32_cmp);
    free(all);
    return depth;
}

/* ---------------------------------------------- whole query (Algorithm 1) */
int64_t or_shortlist(const uint16_t *Xb, const uint8_t *X8, const float *S8, int Dp, const float *qr, const int32_t *C,
                     int64_t nC, int64_t S, int32_t *out);
/* One query end to end: rotate, activate every subspace, count, cut, verify.
 * Scratch: V [N], C [N], cells/w [M][K^2]. */
static void search_one(const or_index *ix, const float *q, int ldq, const or_params *p, int64_t *ids, float *d2,
                       or_stats *st, int32_t *V, int32_t *C, int32_t *C2, int32_t *cells, uint8_t *w, float *qr,
                       uint32_t *qcode) {
    int K2 = ix->K * ix->K, M = ix->M;
    if (ix->rotated) or_rotate_row(q, ix->R32, ix->D, ix->Dp, qr);
    else { memcpy(qr, q, sizeof(float) * ix->D); for (int j = ix->D; j < ix->Dp; ++j) qr[j] = 0.0f; }
    (void)ldq;
    int32_t ncell[1024];
    float cfirst[1024], clast[1024];
    int64_t budget = or_budget(p->rho, ix->N), got = 0;
    for (int m = 0; m < M; ++m) {
        int64_t r;
        cfirst[m] = clast[m] = 0.0f;
        ncell[m] = or_activate_heap_costs(ix, qr, m, p->mode == 1, p->k, budget, cells + (int64_t)m * K2,
                                          w + (int64_t)m * K2, &r, cfirst + m, clast + m);
        got += r;
    }
    or_scores_walk(ix, ncell, cells, w, V);
    int tau = or_tau(p->alpha, M), how = 0;
    int64_t nC = or_cut(V, ix->N, tau, p->k, p->max_candidates, C, &how);
    memset(st, 0, sizeof *st);
    st->n_candidates = nC;
    st->n_retrieved = got;
    st->tau = tau;
    st->fallback = how == 1;
    st->capped = how == 2;
    if (p->mode == 1) {
        or_sign_codes(qr, 1, ix->Dp, qcode);
        int64_t P = p->patience_factor > 0 ? (int64_t)p->patience_factor * p->k : 0;
        or_verify_opt(ix, qr, qcode, C, nC, p->k, p->eps0, P, p->verify_order, ids, d2, &st->n_verified,
                      &st->n_full);
    } else if (p->mode == 2) {
        /* learned depths: features -> MLP -> keep the first depth_V by (V desc,
         * id asc), coarse BF16 scores -> shortlist of depth_S -> FP32 re-rank */
        int F = 2 * M + 68;
        float f[2 * 1024 + 68], y[2];
        or_features(V, C, nC, ix->N, cfirst, clast, M, p->k, tau, f);
        or_mlp_infer(ix->mlp, F, ix->mlp_H, 2, f, y);
        int64_t dV = or_depth(y[0], p->depth_margin, p->k, nC > p->k ? nC : p->k);
        if (dV > nC) dV = nC;
        int64_t dS = or_depth(y[1], p->short_margin, p->k, dV > p->k ? dV : p->k);
        int64_t nV = or_select_by_score(V, C, nC, dV, C2);
        int64_t ns = or_shortlist(ix->Xb, NULL, NULL, ix->Dp, qr, C2, nV, dS, C);
        or_rerank(ix, qr, C, ns, p->k, ids, d2);
        st->n_verified = nV;
        st->n_full = ns;
    } else if (p->precision > 0) {
        /* coarse scores on the low-precision copy, FP32 re-rank of the shortlist */
        int64_t ns = or_shortlist(p->precision == 1 ? ix->Xb : NULL, p->precision == 2 ? ix->X8 : NULL, ix->S8,
                                  ix->Dp, qr, C, nC, p->shortlist, C2);
        or_rerank(ix, qr, C2, ns, p->k, ids, d2);
        st->n_verified = nC;
        st->n_full = ns;
    } else {
        or_rerank(ix, qr, C, nC, p->k, ids, d2);
        st->n_verified = nC;
        st->n_full = nC;
    }
}

/* A batch of queries (rows of Q, stride ldq), OpenMP across queries only.
 * Returns the number of threads used. */
int or_search_batch(const or_index *ix, const float *Q, int64_t nq, int ldq, const or_params *p,
                    int64_t *ids, float *d2, or_stats *st, int nthreads) {
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
#ifdef _OPENMP
#pragma omp master
        used = omp_get_num_threads();
#endif
        int K2 = ix->K * ix->K;
        int32_t *V = (int32_t *)malloc(sizeof(int32_t) * (size_t)ix->N);
        int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)ix->N);
        int32_t *C2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)ix->N);
        int32_t *cells = (int32_t *)malloc(sizeof(int32_t) * (size_t)ix->M * K2);
        uint8_t *w = (uint8_t *)malloc((size_t)ix->M * K2);
        float *qr = (float *)malloc(sizeof(float) * (size_t)ix->Dp);
        uint32_t *qc = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(ix->Dp / 32 + 1));
#pragma omp for schedule(dynamic)
        for (int64_t i = 0; i < nq; ++i)
            search_one(ix, Q + i * ldq, ldq, p, ids + i * p->k, d2 + i * p->k, st + i, V, C, C2, cells, w, qr, qc);
        free(V); free(C); free(C2); free(cells); free(w); free(qr); free(qc);
    }
    return used;
}

/* ------------------------------------------- FP64 brute force (ground truth) */
/* Exact k nearest rows of X to q by FP64 squared L2, ties by id (§3 kNN). */
void or_knn_f64(const float *X, int64_t N, int D, int ldx, const float *Q, int64_t nq, int ldq, int k,
                int64_t *ids, double *d2) {
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < nq; ++i) {
        const float *q = Q + i * ldq;
        double *bd = d2 + i * k;
        int64_t *bi = ids + i * k;
        int size = 0;
        for (int64_t n = 0; n < N; ++n) {
            const float *x = X + n * ldx;
            double acc = 0.0;
            for (int d = 0; d < D; ++d) { double t = (double)x[d] - (double)q[d]; acc += t * t; }
            if (size == k && !(acc < bd[k - 1])) continue;
            if (size == k) size--;
            int p = size;
            while (p > 0 && bd[p - 1] > acc) { bd[p] = bd[p - 1]; bi[p] = bi[p - 1]; --p; }
            bd[p] = acc;
            bi[p] = n;
            size++;
        }
        for (int j = size; j < k; ++j) { bi[j] = -1; bd[j] = INFINITY; }
    }
}
