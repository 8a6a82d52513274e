/*
 * KScaNN CPU ORACLE -- test infrastructure, not part of the product.
 *
 * A plain, slow, obviously correct restatement of the query path of
 * "KScaNN: Scalable ANN Search on Kunpeng" (arXiv 2511.03298): IVF k-means,
 * PQ on residuals, ADC, the quantised LUT scan, candidate selection, exact
 * rerank, the hybrid intra-cluster search and the learned nprob/reorder MLP.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * --impl reference legs may load this library.  It shares no code, header or
 * table with the CUDA library.
 *
 * Arithmetic: FP64 everywhere, except the quantised LUT rule (Sec. 2.5 /
 * Sec. 4.5: 8-bit LUT entries), which is defined in FP32 with every
 * operation rounded separately (compiled with -ffp-contract=off) so that the
 * GPU can reproduce it bit for bit.
 *
 * Orderings: every "top" selection is lexicographic on (value, index),
 * ascending, so each has exactly one answer.
 *
 * Parity status per function is listed in the docstrings of oracle/oracle.py.
 * OpenMP only spreads independent rows or queries over threads; it changes
 * no arithmetic (every sum over rows stays sequential).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_K 16 /* 4-bit PQ: K = 16 codewords per subspace (Table 1, Sec. 4.5) */

/* ------------------------------------------------------------------ */
/* small sort helpers                                                  */
/* ------------------------------------------------------------------ */
typedef struct { double v; int64_t i; } orc_vi;

static int cmp_vi(const void* a, const void* b) {
    const orc_vi* x = (const orc_vi*)a; const orc_vi* y = (const orc_vi*)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    if (x->i < y->i) return -1;
    if (x->i > y->i) return 1;
    return 0;
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

static double sqdist_fd(const float* x, const double* c, int d) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) { double e = (double)x[t] - c[t]; s += e * e; }
    return s;
}

/* ------------------------------------------------------------------ */
/* k-means (Sec. 2.2; Alg. 1 IVF clustering and PQ codebooks)          */
/* ------------------------------------------------------------------ */
/*
 * Lloyd's algorithm in FP64 on the rows X[sample[0..ns)] (row stride ld,
 * first d columns starting at column col0).  Initial centroids are the first
 * L sample rows.  Assignment ties go to the lower centroid id; an empty
 * cluster keeps its previous centroid.  obj[it] (it = 0..iters) is the
 * objective sum of squared distances to the assigned centroid measured
 * before update it (obj[iters] after the last update).
 */
int orc_kmeans(const float* X, int64_t ld, int32_t col0, int32_t d,
               const int64_t* sample, int64_t ns, int32_t L, int32_t iters,
               double* C, double* obj) {
    if (ns < L || L <= 0 || d <= 0) return -1;
    for (int c = 0; c < L; ++c)
        for (int t = 0; t < d; ++t) C[(int64_t)c * d + t] = X[sample[c] * ld + col0 + t];
    int32_t* a = (int32_t*)malloc(sizeof(int32_t) * ns);
    double* sum = (double*)malloc(sizeof(double) * (size_t)L * d);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * L);
    for (int it = 0; it <= iters; ++it) {
        double o = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : o)
#endif
        for (int64_t s = 0; s < ns; ++s) {
            const float* x = X + sample[s] * ld + col0;
            double best = INFINITY; int32_t bi = 0;
            for (int c = 0; c < L; ++c) {
                double dd = sqdist_fd(x, C + (int64_t)c * d, d);
                if (dd < best) { best = dd; bi = c; }
            }
            a[s] = bi; o += best;
        }
        if (obj) obj[it] = o;
        if (it == iters) break;
        memset(sum, 0, sizeof(double) * (size_t)L * d);
        memset(cnt, 0, sizeof(int64_t) * L);
        for (int64_t s = 0; s < ns; ++s) {
            const float* x = X + sample[s] * ld + col0;
            cnt[a[s]]++;
            for (int t = 0; t < d; ++t) sum[(int64_t)a[s] * d + t] += x[t];
        }
        for (int c = 0; c < L; ++c)
            if (cnt[c] > 0)
                for (int t = 0; t < d; ++t) C[(int64_t)c * d + t] = sum[(int64_t)c * d + t] / (double)cnt[c];
    }
    free(a); free(sum); free(cnt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* index build (Alg. 1), with the improved residual of Sec. 4.6.1       */
/* ------------------------------------------------------------------ */
/*
 * Coarse quantiser: Lloyd on X[perm[0..min(n,256L))] for `iters` iterations.
 * Ranking centroids c_rank = the Lloyd centroids, or their unit-norm
 * versions when `spherical` (angular / inner-product data, Sec. 4.6.1).
 * Every vector goes to the list whose ranking score is lowest (ties -> lower
 * list id): L2 score ||x - c_rank||^2, spherical score -<x, c_rank>.
 * Residual centroids c_mean = the arithmetic mean of each list's members
 * (non-normalised, Sec. 4.6.1); an empty list takes its Lloyd centroid.
 * PQ (Sec. 2.3): per subspace j, Lloyd with K = 16 on the residual
 * sub-vectors of X[perm[0..min(n,65536))], same init/tie rules.
 * Encode: code_j(x) = argmin_i ||r^j - C_j[i]||^2, ties -> lower i.
 * All outputs are FP32 (the stored index); every later step reads them.
 */
int orc_build_index(const float* X, int64_t n, int32_t d, int32_t L, int32_t M,
                    int32_t spherical, const int64_t* perm, int32_t iters,
                    float* c_rank, float* c_mean, float* codebook,
                    uint8_t* codes, int32_t* assign) {
    if (d % M != 0 || n < L) return -1;
    const int dsub = d / M;
    int64_t ns = n < (int64_t)256 * L ? n : (int64_t)256 * L;
    double* C = (double*)malloc(sizeof(double) * (size_t)L * d);
    if (orc_kmeans(X, d, 0, d, perm, ns, L, iters, C, NULL) != 0) { free(C); return -1; }
    for (int c = 0; c < L; ++c) {
        double nn = 0.0;
        for (int t = 0; t < d; ++t) nn += C[(int64_t)c * d + t] * C[(int64_t)c * d + t];
        double s = (spherical && nn > 0.0) ? 1.0 / sqrt(nn) : 1.0;
        for (int t = 0; t < d; ++t) c_rank[(int64_t)c * d + t] = (float)(C[(int64_t)c * d + t] * s);
    }
    /* list assignment by the ranking score, computed from the stored fp32 c_rank */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        const float* x = X + i * d;
        double best = INFINITY; int32_t bi = 0;
        for (int c = 0; c < L; ++c) {
            const float* cr = c_rank + (int64_t)c * d;
            double s = 0.0;
            if (spherical) { for (int t = 0; t < d; ++t) s -= (double)x[t] * cr[t]; }
            else { for (int t = 0; t < d; ++t) { double e = (double)x[t] - cr[t]; s += e * e; } }
            if (s < best) { best = s; bi = c; }
        }
        assign[i] = bi;
    }
    double* sum = (double*)calloc((size_t)L * d, sizeof(double));
    int64_t* cnt = (int64_t*)calloc(L, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        cnt[assign[i]]++;
        for (int t = 0; t < d; ++t) sum[(int64_t)assign[i] * d + t] += X[i * d + t];
    }
    for (int c = 0; c < L; ++c)
        for (int t = 0; t < d; ++t)
            c_mean[(int64_t)c * d + t] = cnt[c] > 0 ? (float)(sum[(int64_t)c * d + t] / (double)cnt[c])
                                                   : (float)C[(int64_t)c * d + t];
    free(sum); free(cnt); free(C);
    /* residual r = x - c_mean, one fp32 subtraction: the stored residual */
    int64_t np = n < 65536 ? n : 65536;
    float* Rs = (float*)malloc(sizeof(float) * (size_t)np * d);
    int64_t* seq = (int64_t*)malloc(sizeof(int64_t) * np);
    for (int64_t s = 0; s < np; ++s) {
        int64_t i = perm[s]; seq[s] = s;
        for (int t = 0; t < d; ++t)
            Rs[s * d + t] = X[i * d + t] - c_mean[(int64_t)assign[i] * d + t];
    }
    double* Cj = (double*)malloc(sizeof(double) * ORC_K * dsub);
    for (int j = 0; j < M; ++j) {
        if (orc_kmeans(Rs, d, j * dsub, dsub, seq, np, ORC_K, iters, Cj, NULL) != 0) {
            free(Rs); free(seq); free(Cj); return -1;
        }
        for (int i = 0; i < ORC_K * dsub; ++i) codebook[(int64_t)j * ORC_K * dsub + i] = (float)Cj[i];
    }
    free(Rs); free(seq); free(Cj);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < M; ++j) {
            double best = INFINITY; int bi = 0;
            for (int c = 0; c < ORC_K; ++c) {
                double s = 0.0;
                for (int t = 0; t < dsub; ++t) {
                    int tt = j * dsub + t;
                    float rf = X[i * d + tt] - c_mean[(int64_t)assign[i] * d + tt]; /* stored fp32 residual */
                    double e = (double)rf - (double)codebook[((int64_t)j * ORC_K + c) * dsub + t];
                    s += e * e;
                }
                if (s < best) { best = s; bi = c; }
            }
            codes[i * M + j] = (uint8_t)bi;
        }
    }
    return 0;
}

/* Encode given residual rows (fp64 arithmetic on the given fp32 inputs). */
int orc_encode(const float* Rres, int64_t n, int32_t d, int32_t M, const float* codebook,
               uint8_t* codes, double* best2_gap) {
    const int dsub = d / M;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < M; ++j) {
            double b1 = INFINITY, b2 = INFINITY; int bi = 0;
            for (int c = 0; c < ORC_K; ++c) {
                double s = 0.0;
                for (int t = 0; t < dsub; ++t) {
                    double e = (double)Rres[i * d + j * dsub + t] - (double)codebook[((int64_t)j * ORC_K + c) * dsub + t];
                    s += e * e;
                }
                if (s < b1) { b2 = b1; b1 = s; bi = c; } else if (s < b2) { b2 = s; }
            }
            codes[i * M + j] = (uint8_t)bi;
            if (best2_gap) best2_gap[i * M + j] = b2 - b1;
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* inverted lists (Sec. 2.2): members of each list in ascending id      */
/* ------------------------------------------------------------------ */
int orc_lists(const int32_t* assign, int64_t n, int32_t L, int64_t* list_off, int32_t* list_ids) {
    if (L <= 0) return -1;
    for (int c = 0; c <= L; ++c) list_off[c] = 0;
    for (int64_t i = 0; i < n; ++i) { if (assign[i] < 0 || assign[i] >= L) return -1; list_off[assign[i] + 1]++; }
    for (int c = 0; c < L; ++c) list_off[c + 1] += list_off[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
    for (int c = 0; c < L; ++c) fill[c] = list_off[c];
    for (int64_t i = 0; i < n; ++i) list_ids[fill[assign[i]]++] = (int32_t)i;
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------ */
/* centroid ranking: TopNClusters (Alg. 2)                             */
/* ------------------------------------------------------------------ */
/* score(q,c) = ||q - c||^2 (L2) or -<q,c> (spherical / inner product),
   FP64 from the stored fp32 ranking centroids; the P lowest by (score, id). */
int orc_rank(const float* q, int32_t d, const float* c_rank, int32_t L, int32_t spherical,
             int32_t P, int32_t* probes, double* scores) {
    orc_vi* s = (orc_vi*)malloc(sizeof(orc_vi) * L);
    for (int c = 0; c < L; ++c) {
        const float* cr = c_rank + (int64_t)c * d;
        double v = 0.0;
        if (spherical) { for (int t = 0; t < d; ++t) v -= (double)q[t] * cr[t]; }
        else { for (int t = 0; t < d; ++t) { double e = (double)q[t] - cr[t]; v += e * e; } }
        s[c].v = v; s[c].i = c;
    }
    qsort(s, L, sizeof(orc_vi), cmp_vi);
    if (P > L) P = L;
    for (int r = 0; r < P; ++r) { probes[r] = (int32_t)s[r].i; if (scores) scores[r] = s[r].v; }
    free(s);
    return P;
}

/* ------------------------------------------------------------------ */
/* FP64 asymmetric distance (Eq. 1) with residual tables               */
/* ------------------------------------------------------------------ */
/* L2: sum_j ||(q - c_p)^j - C_j[code_j]||^2.
   IP: -<q, c_p> - sum_j <q^j, C_j[code_j]> (a distance: lower is better). */
double orc_adc64(const float* q, int32_t d, int32_t M, const float* c_mean_p,
                 const float* codebook, const uint8_t* code, int32_t ip) {
    const int dsub = d / M;
    double s = 0.0;
    if (ip) for (int t = 0; t < d; ++t) s -= (double)q[t] * c_mean_p[t];
    for (int j = 0; j < M; ++j) {
        const float* cw = codebook + ((int64_t)j * ORC_K + code[j]) * dsub;
        for (int t = 0; t < dsub; ++t) {
            int tt = j * dsub + t;
            if (ip) s -= (double)q[tt] * cw[t];
            else { double e = ((double)q[tt] - c_mean_p[tt]) - cw[t]; s += e * e; }
        }
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* quantised LUT (Sec. 2.5, Sec. 4.5: 8-bit LUT entries) -- FP32 rule   */
/* ------------------------------------------------------------------ */
/*
 * For one query and its P probes:
 *  T[p][j][i] (fp32): L2 : acc += e*e over t ascending, r = q_t - c_{p,t},
 *                          e = r - C_{j,i,t};  IP: acc += q_t*C_{j,i,t}, T = -acc.
 *  m[p][j] = min_i T;  R = max over p, j of (max_i T - m);  a = 255/R (a = 1 if R == 0).
 *  Q[p][j][i] = min(255, floor((T - m)*a + 0.5))
 *  L2: S = sum_j m[p][j] (j ascending);  IP: S = -<q, c_p> (t ascending) + sum_j m[j].
 *  bias[p] = floor(S*a + 0.5), clamped to [-2^30, 2^30 - 1].
 * Every operation is a separate IEEE fp32 operation (no contraction).
 */
static void lut_f32(const float* q, int32_t d, int32_t M, const float* cp, const float* codebook,
                    int32_t ip, float* T) {
    const int dsub = d / M;
    for (int j = 0; j < M; ++j)
        for (int i = 0; i < ORC_K; ++i) {
            float acc = 0.0f;
            for (int t = 0; t < dsub; ++t) {
                int tt = j * dsub + t;
                float cw = codebook[((int64_t)j * ORC_K + i) * dsub + t];
                if (ip) { float pr = q[tt] * cw; acc = acc + pr; }
                else { float r = q[tt] - cp[tt]; float e = r - cw; float sq = e * e; acc = acc + sq; }
            }
            T[j * ORC_K + i] = ip ? -acc : acc;
        }
}

int orc_lut_q8(const float* q, int32_t d, int32_t M, const float* c_mean, const float* codebook,
               int32_t ip, const int32_t* probes, int32_t P, uint8_t* Qlut, int32_t* bias, float* a_out) {
    float* T = (float*)malloc(sizeof(float) * (size_t)P * M * ORC_K);
    float* m = (float*)malloc(sizeof(float) * (size_t)P * M);
    float R = 0.0f;
    for (int p = 0; p < P; ++p) {
        lut_f32(q, d, M, c_mean + (int64_t)probes[p] * d, codebook, ip, T + (int64_t)p * M * ORC_K);
        for (int j = 0; j < M; ++j) {
            const float* Tj = T + ((int64_t)p * M + j) * ORC_K;
            float mn = Tj[0], mx = Tj[0];
            for (int i = 1; i < ORC_K; ++i) { if (Tj[i] < mn) mn = Tj[i]; if (Tj[i] > mx) mx = Tj[i]; }
            m[p * M + j] = mn;
            float rg = mx - mn;
            if (rg > R) R = rg;
        }
    }
    float a = (R == 0.0f) ? 1.0f : 255.0f / R;
    for (int p = 0; p < P; ++p) {
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < ORC_K; ++i) {
                float df = T[((int64_t)p * M + j) * ORC_K + i] - m[p * M + j];
                float sc = df * a;
                float h = sc + 0.5f;
                float f = floorf(h);
                Qlut[((int64_t)p * M + j) * ORC_K + i] = (uint8_t)(f > 255.0f ? 255.0f : f);
            }
        float S = 0.0f;
        if (ip) {
            const float* cp = c_mean + (int64_t)probes[p] * d;
            float dot = 0.0f;
            for (int t = 0; t < d; ++t) { float pr = q[t] * cp[t]; dot = dot + pr; }
            S = -dot;
        }
        for (int j = 0; j < M; ++j) S = S + m[p * M + j];
        float sa = S * a;
        float bh = sa + 0.5f;
        float bf = floorf(bh);
        if (bf < -1073741824.0f) bf = -1073741824.0f;
        if (bf > 1073741823.0f) bf = 1073741823.0f;
        bias[p] = (int32_t)bf;
    }
    if (a_out) *a_out = a;
    free(T); free(m);
    return 0;
}

/* ------------------------------------------------------------------ */
/* integer LUT16 scan + candidate pool (Alg. 3)                        */
/* ------------------------------------------------------------------ */
/* key(D, id) = ((D + 2^31) << 32) | id : lexicographic (D, id). */
static uint64_t make_key(int32_t D, int32_t id) {
    return ((uint64_t)((uint32_t)D ^ 0x80000000u) << 32) | (uint64_t)(uint32_t)id;
}

int32_t orc_int_dist(const uint8_t* Qlut_p, int32_t bias_p, const uint8_t* code, int32_t M) {
    int32_t D = bias_p;
    for (int j = 0; j < M; ++j) D += Qlut_p[j * ORC_K + code[j]];
    return D;
}

/* Every member of every probed list gets D = bias_p + sum_j Q[p][j][code_j];
   the R smallest keys are written sorted to keys_out.  Returns their count. */
int64_t orc_scan_topr(const uint8_t* codes, int32_t M, const int64_t* list_off, const int32_t* list_ids,
                      const int32_t* probes, int32_t P, const uint8_t* Qlut, const int32_t* bias,
                      int32_t R, uint64_t* keys_out) {
    int64_t tot = 0;
    for (int p = 0; p < P; ++p) tot += list_off[probes[p] + 1] - list_off[probes[p]];
    uint64_t* all = (uint64_t*)malloc(sizeof(uint64_t) * (tot > 0 ? tot : 1));
    int64_t k = 0;
    for (int p = 0; p < P; ++p) {
        int c = probes[p];
        for (int64_t s = list_off[c]; s < list_off[c + 1]; ++s) {
            int32_t id = list_ids[s];
            int32_t D = orc_int_dist(Qlut + (int64_t)p * M * ORC_K, bias[p], codes + (int64_t)id * M, M);
            all[k++] = make_key(D, id);
        }
    }
    qsort(all, tot, sizeof(uint64_t), cmp_u64);
    int64_t cnt = tot < R ? tot : R;
    memcpy(keys_out, all, sizeof(uint64_t) * cnt);
    free(all);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* hybrid intra-cluster search (Sec. 4.4; Alg. 3 graph branch)          */
/* ------------------------------------------------------------------ */
/*
 * graph: per vector id, its 32 neighbours inside its own list (padding -1).
 * entry: per list, the start node of GraphSearch.
 * Policy, per query: probes of rank < n_near are scanned fully; theta is the
 * R-th smallest key among them (all ones if fewer than R).  Every other probe
 * runs a best-first search with result capacity efs; when at least tau of
 * its results have key < theta the list is scanned fully, otherwise only the
 * results join the pool.  The final R smallest keys over the union are
 * written sorted to keys_out.  Returns the count; *n_full counts full scans.
 */
typedef struct { uint64_t* k; int32_t* v; int n; } orc_heap; /* binary heap on key */

static void hswap(orc_heap* h, int a, int b) {
    uint64_t tk = h->k[a]; h->k[a] = h->k[b]; h->k[b] = tk;
    int32_t tv = h->v[a]; h->v[a] = h->v[b]; h->v[b] = tv;
}
/* min-heap when sgn = +1, max-heap when sgn = -1 */
static int hless(uint64_t a, uint64_t b, int sgn) { return sgn > 0 ? a < b : a > b; }
static void hpush(orc_heap* h, uint64_t key, int32_t v, int sgn) {
    int i = h->n++; h->k[i] = key; h->v[i] = v;
    while (i > 0) { int p = (i - 1) / 2; if (hless(h->k[i], h->k[p], sgn)) { hswap(h, i, p); i = p; } else break; }
}
static void hpop(orc_heap* h, int sgn) {
    h->n--; h->k[0] = h->k[h->n]; h->v[0] = h->v[h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, b = i;
        if (l < h->n && hless(h->k[l], h->k[b], sgn)) b = l;
        if (r < h->n && hless(h->k[r], h->k[b], sgn)) b = r;
        if (b == i) break;
        hswap(h, i, b); i = b;
    }
}

/* GraphSearch on one list; writes up to efs result keys to W_out; returns count. */
int32_t orc_graph_search(const uint8_t* codes, int32_t M, const int32_t* graph, int32_t entry,
                         const uint8_t* Qlut_p, int32_t bias_p, int32_t efs, int64_t n_total,
                         uint64_t* W_out) {
    if (entry < 0 || efs <= 0) return 0;
    uint8_t* visited = (uint8_t*)calloc(n_total, 1);
    int cap = 1 + 32 * (efs + 1) * 4;
    orc_heap cand = { (uint64_t*)malloc(sizeof(uint64_t) * cap), (int32_t*)malloc(sizeof(int32_t) * cap), 0 };
    orc_heap W = { (uint64_t*)malloc(sizeof(uint64_t) * (efs + 2)), (int32_t*)malloc(sizeof(int32_t) * (efs + 2)), 0 };
    uint64_t ke = make_key(orc_int_dist(Qlut_p, bias_p, codes + (int64_t)entry * M, M), entry);
    visited[entry] = 1;
    hpush(&cand, ke, entry, +1);
    hpush(&W, ke, entry, -1);
    while (cand.n > 0) {
        uint64_t ku = cand.k[0]; int32_t u = cand.v[0];
        if (W.n == efs && ku > W.k[0]) break;
        hpop(&cand, +1);
        for (int e = 0; e < 32; ++e) {
            int32_t v = graph[(int64_t)u * 32 + e];
            if (v < 0 || visited[v]) continue;
            visited[v] = 1;
            uint64_t kv = make_key(orc_int_dist(Qlut_p, bias_p, codes + (int64_t)v * M, M), v);
            if (W.n < efs || kv < W.k[0]) {
                if (cand.n >= cap) { /* cannot happen: each node enters once per list */ }
                hpush(&cand, kv, v, +1);
                hpush(&W, kv, v, -1);
                if (W.n > efs) hpop(&W, -1);
            }
        }
    }
    int32_t cnt = W.n;
    for (int i = 0; i < cnt; ++i) W_out[i] = W.k[i];
    qsort(W_out, cnt, sizeof(uint64_t), cmp_u64);
    free(visited); free(cand.k); free(cand.v); free(W.k); free(W.v);
    return cnt;
}

int64_t orc_hybrid_topr(const uint8_t* codes, int32_t M, const int64_t* list_off, const int32_t* list_ids,
                        int64_t n_total, const int32_t* graph, const int32_t* entry,
                        const int32_t* probes, int32_t P, const uint8_t* Qlut, const int32_t* bias,
                        int32_t R, int32_t n_near, int32_t efs, int32_t tau,
                        uint64_t* keys_out, int32_t* n_full) {
    int64_t tot = 0;
    for (int p = 0; p < P; ++p) tot += list_off[probes[p] + 1] - list_off[probes[p]];
    uint64_t* pool = (uint64_t*)malloc(sizeof(uint64_t) * (tot + 1));
    uint64_t* W = (uint64_t*)malloc(sizeof(uint64_t) * (efs > 0 ? efs : 1));
    int64_t k = 0; int32_t full = 0;
    int nn = n_near < P ? n_near : P;
    for (int p = 0; p < nn; ++p) {
        int c = probes[p];
        for (int64_t s = list_off[c]; s < list_off[c + 1]; ++s) {
            int32_t id = list_ids[s];
            pool[k++] = make_key(orc_int_dist(Qlut + (int64_t)p * M * ORC_K, bias[p], codes + (int64_t)id * M, M), id);
        }
        full++;
    }
    uint64_t theta = ~(uint64_t)0;
    if (k >= R) {
        uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * k);
        memcpy(tmp, pool, sizeof(uint64_t) * k);
        qsort(tmp, k, sizeof(uint64_t), cmp_u64);
        theta = tmp[R - 1];
        free(tmp);
    }
    for (int p = nn; p < P; ++p) {
        int c = probes[p];
        const uint8_t* Qp = Qlut + (int64_t)p * M * ORC_K;
        int32_t w = orc_graph_search(codes, M, graph, entry[c], Qp, bias[p], efs, n_total, W);
        int32_t good = 0;
        for (int i = 0; i < w; ++i) if (W[i] < theta) good++;
        if (good >= tau) {
            for (int64_t s = list_off[c]; s < list_off[c + 1]; ++s) {
                int32_t id = list_ids[s];
                pool[k++] = make_key(orc_int_dist(Qp, bias[p], codes + (int64_t)id * M, M), id);
            }
            full++;
        } else {
            for (int i = 0; i < w; ++i) pool[k++] = W[i];
        }
    }
    qsort(pool, k, sizeof(uint64_t), cmp_u64);
    int64_t cnt = k < R ? k : R;
    memcpy(keys_out, pool, sizeof(uint64_t) * cnt);
    if (n_full) *n_full = full;
    free(pool); free(W);
    return cnt;
}

/* Exact 32-NN graph inside each list (FP64 on the stored vectors, ties -> lower
   id); lists with at most 32 other members list all of them, padded with -1.
   entry[c] = the member nearest c_mean[c] (ties -> lower id), -1 if empty. */
int orc_build_graph(const float* X, int32_t d, const int64_t* list_off, const int32_t* list_ids,
                    int32_t L, const float* c_mean, int32_t* graph, int32_t* entry) {
    for (int c = 0; c < L; ++c) {
        int64_t b = list_off[c], e = list_off[c + 1], m = e - b;
        entry[c] = -1;
        double best = INFINITY;
        for (int64_t s = b; s < e; ++s) {
            int32_t id = list_ids[s];
            double v = 0.0;
            for (int t = 0; t < d; ++t) { double df = (double)X[(int64_t)id * d + t] - c_mean[(int64_t)c * d + t]; v += df * df; }
            if (v < best || (v == best && id < entry[c])) { best = v; entry[c] = id; }
        }
        orc_vi* tmp = (orc_vi*)malloc(sizeof(orc_vi) * (m > 0 ? m : 1));
        for (int64_t s = b; s < e; ++s) {
            int32_t u = list_ids[s];
            int64_t w = 0;
            for (int64_t s2 = b; s2 < e; ++s2) {
                int32_t v = list_ids[s2];
                if (v == u) continue;
                double dd = 0.0;
                for (int t = 0; t < d; ++t) { double df = (double)X[(int64_t)u * d + t] - X[(int64_t)v * d + t]; dd += df * df; }
                tmp[w].v = dd; tmp[w].i = v; w++;
            }
            qsort(tmp, w, sizeof(orc_vi), cmp_vi);
            for (int e2 = 0; e2 < 32; ++e2) graph[(int64_t)u * 32 + e2] = e2 < w ? (int32_t)tmp[e2].i : -1;
        }
        free(tmp);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* exact distances: rerank (Alg. 2) and brute-force kNN                 */
/* ------------------------------------------------------------------ */
/* dist(q, x) in FP64: L2 = sum_t (q_t - x_t)^2 ; IP = -<q, x> (lower is better). */
static double exact_dist(const float* q, const float* x, int d, int ip) {
    double s = 0.0;
    if (ip) { for (int t = 0; t < d; ++t) s -= (double)q[t] * x[t]; }
    else { for (int t = 0; t < d; ++t) { double e = (double)q[t] - x[t]; s += e * e; } }
    return s;
}

/* Re-rank ids[0..nc) with exact distances; write the k best by (dist, id).
   Output distance: L2 squared distance ascending, IP similarity descending;
   short results are padded with id -1 and +inf (L2) / -inf (IP). */
int orc_rerank(const float* q, const float* X, int32_t d, int32_t ip, const int32_t* ids, int64_t nc,
               int32_t k, int64_t* out_ids, double* out_d) {
    orc_vi* s = (orc_vi*)malloc(sizeof(orc_vi) * (nc > 0 ? nc : 1));
    for (int64_t i = 0; i < nc; ++i) { s[i].i = ids[i]; s[i].v = exact_dist(q, X + (int64_t)ids[i] * d, d, ip); }
    qsort(s, nc, sizeof(orc_vi), cmp_vi);
    for (int r = 0; r < k; ++r) {
        if (r < nc) { out_ids[r] = s[r].i; out_d[r] = ip ? -s[r].v : s[r].v; }
        else { out_ids[r] = -1; out_d[r] = ip ? -INFINITY : INFINITY; }
    }
    free(s);
    return 0;
}

/* Brute-force exact k-NN of each query over all n rows, FP64, ties -> lower id. */
int orc_exact_knn(const float* Q, int64_t nq, const float* X, int64_t n, int32_t d, int32_t ip,
                  int32_t k, int64_t* out_ids, double* out_d, int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int64_t qi = 0; qi < nq; ++qi) {
        orc_vi* s = (orc_vi*)malloc(sizeof(orc_vi) * n);
        for (int64_t i = 0; i < n; ++i) { s[i].i = i; s[i].v = exact_dist(Q + qi * d, X + i * d, d, ip); }
        qsort(s, n, sizeof(orc_vi), cmp_vi);
        for (int r = 0; r < k; ++r) {
            out_ids[qi * k + r] = r < n ? s[r].i : -1;
            out_d[qi * k + r] = r < n ? (ip ? -s[r].v : s[r].v) : (ip ? -INFINITY : INFINITY);
        }
        free(s);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* whole search (Alg. 2 with the plain leaf scan of Alg. 3)             */
/* ------------------------------------------------------------------ */
/*
 * Per query: rank (nprobe[q] probes), quantised LUT, integer scan, R[q]
 * smallest keys (R clamped to >= k), exact rerank with the same query, top-k.
 * Optional outputs (may be NULL): probes_out [nq x pstride], cand_out
 * [nq x rstride] candidate keys (sorted), ncand_out [nq].
 * OpenMP over queries only; the per-query arithmetic is as above.
 */
int orc_search(const float* Q, int64_t nq, int32_t d, int32_t M, int32_t L, int32_t ip, int32_t spherical,
               const float* X, const float* c_rank, const float* c_mean, const float* codebook,
               const uint8_t* codes, const int64_t* list_off, const int32_t* list_ids,
               const int32_t* nprobe, const int32_t* Rr, int32_t k,
               int64_t* out_ids, double* out_d,
               int32_t* probes_out, int32_t pstride, uint64_t* cand_out, int32_t rstride, int64_t* ncand_out,
               int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float* q = Q + qi * d;
        int32_t P = nprobe[qi] < L ? nprobe[qi] : L;
        int32_t R = Rr[qi] < k ? k : Rr[qi];
        int32_t* probes = (int32_t*)malloc(sizeof(int32_t) * P);
        orc_rank(q, d, c_rank, L, spherical, P, probes, NULL);
        uint8_t* Ql = (uint8_t*)malloc((size_t)P * M * ORC_K);
        int32_t* bias = (int32_t*)malloc(sizeof(int32_t) * P);
        orc_lut_q8(q, d, M, c_mean, codebook, ip, probes, P, Ql, bias, NULL);
        uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * R);
        int64_t nc = orc_scan_topr(codes, M, list_off, list_ids, probes, P, Ql, bias, R, keys);
        int32_t* cid = (int32_t*)malloc(sizeof(int32_t) * (nc > 0 ? nc : 1));
        for (int64_t i = 0; i < nc; ++i) cid[i] = (int32_t)(keys[i] & 0xffffffffu);
        orc_rerank(q, X, d, ip, cid, nc, k, out_ids + qi * k, out_d + qi * k);
        if (probes_out) for (int r = 0; r < pstride; ++r) probes_out[qi * pstride + r] = r < P ? probes[r] : -1;
        if (cand_out) for (int r = 0; r < rstride; ++r) cand_out[qi * rstride + r] = r < nc ? keys[r] : ~(uint64_t)0;
        if (ncand_out) ncand_out[qi] = nc;
        free(probes); free(Ql); free(bias); free(keys); free(cid);
    }
    return 0;
}

/* Recall@k with ties: a returned id counts when its exact FP64 distance is no
   worse than the true k-th distance; at most k per query; mean over queries. */
double orc_recall(const float* Q, int64_t nq, const float* X, int32_t d, int32_t ip,
                  const int64_t* ids, int32_t kret, const double* true_d, int32_t ktrue, int32_t k) {
    double tot = 0.0;
    for (int64_t qi = 0; qi < nq; ++qi) {
        double kth = true_d[qi * ktrue + (k - 1)];
        int hit = 0;
        for (int r = 0; r < kret && r < k; ++r) {
            int64_t id = ids[qi * kret + r];
            if (id < 0) continue;
            int dup = 0;
            for (int r2 = 0; r2 < r; ++r2) if (ids[qi * kret + r2] == id) dup = 1;
            if (dup) continue;
            double dv = exact_dist(Q + qi * d, X + id * d, d, ip);
            if (ip ? (-dv >= kth) : (dv <= kth)) hit++;
        }
        tot += (hit > k ? k : hit) / (double)k;
    }
    return nq > 0 ? tot / nq : 0.0;
}

/* ------------------------------------------------------------------ */
/* learned nprob / reorder (Sec. 4.2.1-4.2.2, Eq. 2)                    */
/* ------------------------------------------------------------------ */
/*
 * Eq. 2 (reading of the line-broken formula):
 *   P = min(Pmax, Pmin + ceil((Pmax - Pmin) * max(0, p - p0) * (p + p1))).
 */
int32_t orc_eq2(double p, int32_t pmin, int32_t pmax, double p0, double p1) {
    double relu = p - p0 > 0.0 ? p - p0 : 0.0;
    double v = (double)(pmax - pmin) * relu * (p + p1);
    double c = ceil(v);
    double r = (double)pmin + c;
    if (r > pmax) r = pmax;
    if (r < pmin) r = pmin;
    return (int32_t)r;
}

/*
 * Multilayer perceptron F -> H1 -> H2 -> 2 with ReLU hidden units and two
 * sigmoid outputs (easy/hard probability for nprob and for reorder), FP64.
 * Weights: W1 [H1 x F], b1 [H1], W2 [H2 x H1], b2 [H2], W3 [2 x H2], b3 [2],
 * packed in that order in `w`.  Loss: mean over the batch of the sum over the
 * two heads of the binary cross-entropy with targets y [B x 2].
 * orc_mlp_forward writes probabilities [B x 2]; orc_mlp_grad returns the loss
 * and writes dL/dw (same packing).
 */
static int64_t mlp_nparams(int F, int H1, int H2) {
    return (int64_t)H1 * F + H1 + (int64_t)H2 * H1 + H2 + 2 * H2 + 2;
}

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }

int orc_mlp_forward(const double* w, int32_t F, int32_t H1, int32_t H2, const double* x, int64_t B, double* prob) {
    const double *W1 = w, *b1 = W1 + (int64_t)H1 * F, *W2 = b1 + H1, *b2 = W2 + (int64_t)H2 * H1,
                 *W3 = b2 + H2, *b3 = W3 + 2 * H2;
    double* h1 = (double*)malloc(sizeof(double) * H1);
    double* h2 = (double*)malloc(sizeof(double) * H2);
    for (int64_t s = 0; s < B; ++s) {
        for (int a = 0; a < H1; ++a) { double z = b1[a]; for (int f = 0; f < F; ++f) z += W1[(int64_t)a * F + f] * x[s * F + f]; h1[a] = z > 0 ? z : 0; }
        for (int a = 0; a < H2; ++a) { double z = b2[a]; for (int f = 0; f < H1; ++f) z += W2[(int64_t)a * H1 + f] * h1[f]; h2[a] = z > 0 ? z : 0; }
        for (int o = 0; o < 2; ++o) { double z = b3[o]; for (int f = 0; f < H2; ++f) z += W3[o * H2 + f] * h2[f]; prob[s * 2 + o] = sigm(z); }
    }
    free(h1); free(h2);
    return 0;
}

double orc_mlp_grad(const double* w, int32_t F, int32_t H1, int32_t H2, const double* x, const double* y,
                    int64_t B, double* g) {
    const double *W1 = w, *b1 = W1 + (int64_t)H1 * F, *W2 = b1 + H1, *b2 = W2 + (int64_t)H2 * H1,
                 *W3 = b2 + H2, *b3 = W3 + 2 * H2;
    int64_t np = mlp_nparams(F, H1, H2);
    memset(g, 0, sizeof(double) * np);
    double *gW1 = g, *gb1 = gW1 + (int64_t)H1 * F, *gW2 = gb1 + H1, *gb2 = gW2 + (int64_t)H2 * H1,
           *gW3 = gb2 + H2, *gb3 = gW3 + 2 * H2;
    double* z1 = (double*)malloc(sizeof(double) * H1); double* h1 = (double*)malloc(sizeof(double) * H1);
    double* z2 = (double*)malloc(sizeof(double) * H2); double* h2 = (double*)malloc(sizeof(double) * H2);
    double* d2 = (double*)malloc(sizeof(double) * H2); double* d1 = (double*)malloc(sizeof(double) * H1);
    double loss = 0.0;
    for (int64_t s = 0; s < B; ++s) {
        const double* xs = x + s * F;
        for (int a = 0; a < H1; ++a) { double z = b1[a]; for (int f = 0; f < F; ++f) z += W1[(int64_t)a * F + f] * xs[f]; z1[a] = z; h1[a] = z > 0 ? z : 0; }
        for (int a = 0; a < H2; ++a) { double z = b2[a]; for (int f = 0; f < H1; ++f) z += W2[(int64_t)a * H1 + f] * h1[f]; z2[a] = z; h2[a] = z > 0 ? z : 0; }
        for (int a = 0; a < H2; ++a) d2[a] = 0.0;
        for (int o = 0; o < 2; ++o) {
            double z = b3[o]; for (int f = 0; f < H2; ++f) z += W3[o * H2 + f] * h2[f];
            double p = sigm(z), t = y[s * 2 + o];
            /* BCE in the log-sum-exp form: max(z,0) - z t + log(1 + e^-|z|) */
            loss += (z > 0 ? z : 0) - z * t + log1p(exp(-fabs(z)));
            double dz = (p - t) / (double)B;
            gb3[o] += dz;
            for (int f = 0; f < H2; ++f) { gW3[o * H2 + f] += dz * h2[f]; d2[f] += dz * W3[o * H2 + f]; }
        }
        for (int a = 0; a < H2; ++a) d2[a] = z2[a] > 0 ? d2[a] : 0.0;
        for (int f = 0; f < H1; ++f) d1[f] = 0.0;
        for (int a = 0; a < H2; ++a) {
            gb2[a] += d2[a];
            for (int f = 0; f < H1; ++f) { gW2[(int64_t)a * H1 + f] += d2[a] * h1[f]; d1[f] += d2[a] * W2[(int64_t)a * H1 + f]; }
        }
        for (int a = 0; a < H1; ++a) {
            double da = z1[a] > 0 ? d1[a] : 0.0;
            gb1[a] += da;
            for (int f = 0; f < F; ++f) gW1[(int64_t)a * F + f] += da * xs[f];
        }
    }
    free(z1); free(h1); free(z2); free(h2); free(d2); free(d1);
    return loss / (double)B;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1) on all parameters, FP64. */
int orc_adam_step(double* w, const double* g, double* m, double* v, int64_t np, int32_t t,
                  double lr, double beta1, double beta2, double eps) {
    double bc1 = 1.0 - pow(beta1, t), bc2 = 1.0 - pow(beta2, t);
    for (int64_t i = 0; i < np; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Predictive cluster pruning (Sec. 4.2.3, Table 4; Alg. 2 f_prune)    */
/* ------------------------------------------------------------------ */
/*
 * Per-list statistics of the members' offsets r_x = x - c_p from the list's
 * mean centroid (FP64), PRUNE_NSTAT values per list:
 *   0 n_p, 1 radius rho = max |r_x|, 2 mean mu of |r_x|, 3 population std
 *   sigma of |r_x| (two passes), 4..7 the distance histogram: fractions of
 *   members with |r_x| in [0, rho/4], (rho/4, rho/2], (rho/2, 3rho/4],
 *   (3rho/4, rho], 8 outlier fraction (|r_x| > mu + 2 sigma), 9, 10 the
 *   variances lambda_1, lambda_2 along the two principal axes, 11 zero.
 * Vectors per list (3 x d): the principal axes v_1, v_2 of the offsets'
 * second moment (1/n_p) sum r_x r_x^T by `iters` power iterations each
 * (v_1 from (1,..,1)/sqrt(d); v_2 from (+1,-1,+1,..)/sqrt(d), with v_1
 * projected out of the start and of every iterate), and the outlier
 * direction, the mean offset of the outliers (zero when there are none).
 * An empty list has all zeros.
 */
#define PRUNE_NSTAT 12
#define PRUNE_NFEAT 16

static void unit_or_keep(double* v, const double* w, int32_t d) {
    double nn = 0.0;
    for (int t = 0; t < d; ++t) nn += w[t] * w[t];
    if (nn > 0.0) { double s = 1.0 / sqrt(nn); for (int t = 0; t < d; ++t) v[t] = w[t] * s; }
}

int orc_prune_stats(const float* X, int64_t n, int32_t d, const float* c_mean, int32_t L,
                    const int32_t* assign, int32_t iters, double* stats, double* vecs) {
    memset(stats, 0, sizeof(double) * (size_t)L * PRUNE_NSTAT);
    memset(vecs, 0, sizeof(double) * (size_t)L * 3 * d);
    int64_t* cnt = (int64_t*)calloc((size_t)L + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cnt[assign[i] + 1]++;
    for (int32_t p = 0; p < L; ++p) cnt[p + 1] += cnt[p];
    int64_t* mem = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* fill = (int64_t*)calloc((size_t)L, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) { int32_t p = assign[i]; mem[cnt[p] + fill[p]++] = i; }
#pragma omp parallel for schedule(dynamic)
    for (int32_t p = 0; p < L; ++p) {
        const int64_t np_ = cnt[p + 1] - cnt[p];
        if (np_ == 0) continue;
        const int64_t* ids = mem + cnt[p];
        const float* c = c_mean + (int64_t)p * d;
        double* r = (double*)malloc(sizeof(double) * (size_t)np_ * d);
        double* dist = (double*)malloc(sizeof(double) * (size_t)np_);
        for (int64_t m = 0; m < np_; ++m) {
            double s = 0.0;
            for (int t = 0; t < d; ++t) {
                double e = (double)X[ids[m] * d + t] - (double)c[t];
                r[m * d + t] = e;
                s += e * e;
            }
            dist[m] = sqrt(s);
        }
        double rho = 0.0, mu = 0.0, var = 0.0;
        for (int64_t m = 0; m < np_; ++m) { if (dist[m] > rho) rho = dist[m]; mu += dist[m]; }
        mu /= (double)np_;
        for (int64_t m = 0; m < np_; ++m) var += (dist[m] - mu) * (dist[m] - mu);
        const double sigma = sqrt(var / (double)np_);
        int64_t hist[4] = {0, 0, 0, 0}, nout = 0;
        double* st = stats + (int64_t)p * PRUNE_NSTAT;
        double* v1 = vecs + (int64_t)p * 3 * d;
        double* v2 = v1 + d;
        double* od = v2 + d;
        for (int64_t m = 0; m < np_; ++m) {
            int b = 0;
            if (dist[m] > 0.75 * rho) b = 3;
            else if (dist[m] > 0.5 * rho) b = 2;
            else if (dist[m] > 0.25 * rho) b = 1;
            hist[b]++;
            if (dist[m] > mu + 2.0 * sigma) {
                nout++;
                for (int t = 0; t < d; ++t) od[t] += r[m * d + t];
            }
        }
        if (nout > 0) for (int t = 0; t < d; ++t) od[t] /= (double)nout;
        /* power iterations */
        double* w = (double*)malloc(sizeof(double) * d);
        for (int t = 0; t < d; ++t) v1[t] = 1.0 / sqrt((double)d);
        for (int it = 0; it < iters; ++it) {
            for (int t = 0; t < d; ++t) w[t] = 0.0;
            for (int64_t m = 0; m < np_; ++m) {
                double a = 0.0;
                for (int t = 0; t < d; ++t) a += r[m * d + t] * v1[t];
                for (int t = 0; t < d; ++t) w[t] += a * r[m * d + t];
            }
            unit_or_keep(v1, w, d);
        }
        for (int t = 0; t < d; ++t) w[t] = ((t & 1) ? -1.0 : 1.0) / sqrt((double)d);
        {
            double a = 0.0;
            for (int t = 0; t < d; ++t) a += w[t] * v1[t];
            for (int t = 0; t < d; ++t) w[t] -= a * v1[t];
            unit_or_keep(v2, w, d);
        }
        for (int it = 0; it < iters; ++it) {
            for (int t = 0; t < d; ++t) w[t] = 0.0;
            for (int64_t m = 0; m < np_; ++m) {
                double a = 0.0;
                for (int t = 0; t < d; ++t) a += r[m * d + t] * v2[t];
                for (int t = 0; t < d; ++t) w[t] += a * r[m * d + t];
            }
            double a = 0.0;
            for (int t = 0; t < d; ++t) a += w[t] * v1[t];
            for (int t = 0; t < d; ++t) w[t] -= a * v1[t];
            unit_or_keep(v2, w, d);
        }
        double l1 = 0.0, l2 = 0.0;
        for (int64_t m = 0; m < np_; ++m) {
            double a1 = 0.0, a2 = 0.0;
            for (int t = 0; t < d; ++t) { a1 += r[m * d + t] * v1[t]; a2 += r[m * d + t] * v2[t]; }
            l1 += a1 * a1;
            l2 += a2 * a2;
        }
        st[0] = (double)np_;
        st[1] = rho;
        st[2] = mu;
        st[3] = sigma;
        for (int b = 0; b < 4; ++b) st[4 + b] = (double)hist[b] / (double)np_;
        st[8] = (double)nout / (double)np_;
        st[9] = l1 / (double)np_;
        st[10] = l2 / (double)np_;
        free(w); free(r); free(dist);
    }
    free(cnt); free(mem); free(fill);
    return 0;
}

/*
 * Features of (query q, probe rank r < P_q), PRUNE_NFEAT values, FP64, from
 * the list statistics above.  p = probes[r], c = its mean centroid,
 * D = |q - c|, u = (q - c) / max(D, 1e-9), D0 = |q - c_{probes[0]}| and
 * g = max(D0, 1e-9) (distances relative to the nearest probe's):
 *   0 D / max(rho, 1e-9)    1 D / g       2 (D - rho) / g   3 log(1 + n_p)
 *   4 rho / g   5 mu / g   6 sigma / g   7..10 the histogram   11 outliers
 *   12 lambda_1 <v_1, u>^2 / g^2   13 lambda_2 <v_2, u>^2 / g^2
 *   14 <outlier direction, u> / g   15 D0 / max(rho of probes[0], 1e-9).
 * Rows r >= P_q and invalid list ids are zero.
 */
int orc_prune_features(const float* Q, int64_t nq, int32_t d, const float* c_mean, int32_t L,
                       const int32_t* probes, int32_t Pmax, const int32_t* nprobe, int32_t P,
                       const double* stats, const double* vecs, double* feats) {
    memset(feats, 0, sizeof(double) * (size_t)nq * Pmax * PRUNE_NFEAT);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nq; ++q) {
        int32_t Pq = nprobe ? nprobe[q] : P;
        if (Pq < 1) Pq = 1;
        if (Pq > Pmax) Pq = Pmax;
        const float* qv = Q + q * d;
        const int32_t* pr = probes + q * Pmax;
        double D0 = 0.0, rho0 = 0.0;
        if (pr[0] >= 0 && pr[0] < L) {
            for (int t = 0; t < d; ++t) { double e = (double)qv[t] - c_mean[(int64_t)pr[0] * d + t]; D0 += e * e; }
            D0 = sqrt(D0);
            rho0 = stats[(int64_t)pr[0] * PRUNE_NSTAT + 1];
        }
        const double g = D0 > 1e-9 ? D0 : 1e-9;
        for (int32_t r = 0; r < Pq; ++r) {
            const int32_t p = pr[r];
            if (p < 0 || p >= L) continue;
            const double* st = stats + (int64_t)p * PRUNE_NSTAT;
            const double* v1 = vecs + (int64_t)p * 3 * d;
            const double* v2 = v1 + d;
            const double* od = v2 + d;
            double D = 0.0;
            for (int t = 0; t < d; ++t) { double e = (double)qv[t] - c_mean[(int64_t)p * d + t]; D += e * e; }
            D = sqrt(D);
            const double Dg = D > 1e-9 ? D : 1e-9;
            double a1 = 0.0, a2 = 0.0, ao = 0.0;
            for (int t = 0; t < d; ++t) {
                double u = ((double)qv[t] - c_mean[(int64_t)p * d + t]) / Dg;
                a1 += v1[t] * u;
                a2 += v2[t] * u;
                ao += od[t] * u;
            }
            double* f = feats + (q * Pmax + r) * PRUNE_NFEAT;
            f[0] = D / (st[1] > 1e-9 ? st[1] : 1e-9);
            f[1] = D / g;
            f[2] = (D - st[1]) / g;
            f[3] = log(1.0 + st[0]);
            f[4] = st[1] / g;
            f[5] = st[2] / g;
            f[6] = st[3] / g;
            for (int b = 0; b < 4; ++b) f[7 + b] = st[4 + b];
            f[11] = st[8];
            f[12] = st[9] * a1 * a1 / (g * g);
            f[13] = st[10] * a2 * a2 / (g * g);
            f[14] = ao / g;
            f[15] = D0 / (rho0 > 1e-9 ? rho0 : 1e-9);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Component filtration (Sec. 4.3; Alg. 1 / Alg. 2 FilterComponents)  */
/* ------------------------------------------------------------------ */
/*
 * Per dimension t of X [n x d] (FP64, two passes): mean mu_t, population
 * standard deviation sigma_t, and frac[t] = the fraction of the n values that
 * are 0 or within one standard deviation of the mean (|x - mu_t| <= sigma_t).
 * Dimensions whose fraction exceeds the threshold carry little information
 * and are dropped (oracle.py: component_keep).
 */
int orc_component_stats(const float* X, int64_t n, int32_t d, double* mu, double* sigma, double* frac) {
#pragma omp parallel for schedule(static)
    for (int32_t t = 0; t < d; ++t) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += (double)X[i * d + t];
        const double m = n > 0 ? s / (double)n : 0.0;
        double v = 0.0;
        for (int64_t i = 0; i < n; ++i) { double e = (double)X[i * d + t] - m; v += e * e; }
        const double sd = n > 0 ? sqrt(v / (double)n) : 0.0;
        int64_t c = 0;
        for (int64_t i = 0; i < n; ++i) {
            const double x = (double)X[i * d + t];
            if (x == 0.0 || fabs(x - m) <= sd) c++;
        }
        mu[t] = m;
        sigma[t] = sd;
        frac[t] = n > 0 ? (double)c / (double)n : 1.0;
    }
    return 0;
}

/*
 * Regression variant of the learned nprobe / reorder heads (the
 * regression-head variant of Sec. 4.2.2's predictor): the head's output p in
 * [0, 1] is read as the normalised log of the setting,
 *   u = clamp(p (1 + b) + a, 0, 1),  v = lo (hi / lo)^u,
 *   P = clamp(ceil(v - 1e-3), lo, hi)
 * (a value within 1e-3 above an integer counts as that integer, so the
 * rounding of the power cannot push an exact integer to the next one).
 */
int32_t orc_reg_map(double p, int32_t lo, int32_t hi, double a, double b) {
    double u = p * (1.0 + b) + a;
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    double v = (double)lo * pow((double)hi / (double)lo, u);
    double r = ceil(v - 1e-3);
    if (r < lo) r = lo;
    if (r > hi) r = hi;
    return (int32_t)r;
}
