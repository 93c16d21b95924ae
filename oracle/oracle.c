/*
 * FP64 CPU oracle for FINGER (Chen et al., "FINGER: Fast Inference for
 * Graph-based Approximate Nearest Neighbor Search", arXiv 2206.11408).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or constant with the CUDA path; only tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.
 *
 * Everything is double precision and scalar.  Keys are compared as the pair
 * (distance, id), lexicographically, everywhere (the paper is silent on ties).
 *
 * Contents
 *   orc_splitmix64      counter-based generator (Steele, Lea, Flood 2014)
 *   orc_levels          HNSW level draw floor(-ln U / ln M) per node
 *   orc_bruteforce      exact kNN by a full scan (the recall ground truth, Sec. 1)
 *   orc_hnsw_build      incremental HNSW construction (Malkov & Yashunin 2018,
 *                       insertion + heuristic neighbour selection), the graph
 *                       the paper accelerates (Sec. 4.1)
 *   orc_search          upper-layer greedy descent, then Algorithm 1 (plain) or
 *                       Algorithm 4 with Algorithm 3 as appx() (FINGER) on layer 0
 *   orc_sample_pairs    the neighbour-pair draw of Algorithm 2
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double d;
    int32_t id;
} kv_t;

static inline int kv_less(kv_t a, kv_t b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* squared L2 distance, summed in index order */
static double l2sq(const double* a, const double* b, int m) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) {
        double t = a[i] - b[i];
        s += t * t;
    }
    return s;
}

static double dot(const double* a, const double* b, int m) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

/* HNSW level of node i: floor(-ln(U_i) * mL), mL = 1/ln(M), U_i in (0,1]. */
void orc_levels(int64_t n, int M, uint64_t seed, int32_t* level) {
    double mL = 1.0 / log((double)M);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t h = orc_splitmix64(seed ^ (uint64_t)i);
        double u = (double)((h >> 11) + 1) * (1.0 / 9007199254740992.0);
        int l = (int)floor(-log(u) * mL);
        level[i] = l > 30 ? 30 : l;
    }
}

/* ------------------------------------------------------------------ sorting */

static int kv_cmp(const void* a, const void* b) {
    kv_t x = *(const kv_t*)a, y = *(const kv_t*)b;
    if (kv_less(x, y)) return -1;
    if (kv_less(y, x)) return 1;
    return 0;
}

/* insert kv into ascending array arr[0..*len) of capacity cap; drop the last
 * element when full.  Returns the insert position or -1 if not inserted. */
static int sorted_insert(kv_t* arr, int* len, int cap, kv_t x) {
    int n = *len;
    if (n == cap && !kv_less(x, arr[n - 1])) return -1;
    int p = n < cap ? n : cap - 1;
    while (p > 0 && kv_less(x, arr[p - 1])) {
        if (p < cap) arr[p] = arr[p - 1];
        --p;
    }
    arr[p] = x;
    if (n < cap) *len = n + 1;
    return p;
}

/* ------------------------------------------------------------ brute force */

void orc_bruteforce(const double* X, int64_t n, int m, const double* Q, int64_t nq, int K,
                    int64_t* ids, double* dists, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        kv_t* top = (kv_t*)malloc(sizeof(kv_t) * (size_t)(K + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t qi = 0; qi < nq; ++qi) {
            int len = 0;
            const double* q = Q + (size_t)qi * m;
            for (int64_t i = 0; i < n; ++i) {
                kv_t x = {l2sq(q, X + (size_t)i * m, m), (int32_t)i};
                sorted_insert(top, &len, K, x);
            }
            for (int k = 0; k < K; ++k) {
                ids[qi * K + k] = k < len ? top[k].id : -1;
                dists[qi * K + k] = k < len ? top[k].d : INFINITY;
            }
        }
        free(top);
    }
}

/* ------------------------------------------------------------ HNSW build */

typedef struct {
    const double* X;
    int64_t n;
    int m;
    int M;        /* cap on levels >= 1 and number of links made at insertion */
    int deg0;     /* cap on layer 0 (2M) */
    int32_t* adj0;
    int32_t* cnt0;
    const int64_t* up_off;
    int32_t* up_adj;
    int32_t* cntu;
    int32_t* stamp;
    int32_t cur_stamp;
} hnsw_t;

static int32_t* links(hnsw_t* h, int64_t v, int lc, int32_t** cnt) {
    if (lc == 0) {
        *cnt = &h->cnt0[v];
        return h->adj0 + (size_t)v * h->deg0;
    }
    int64_t row = h->up_off[v] + (lc - 1);
    *cnt = &h->cntu[row];
    return h->up_adj + (size_t)row * h->M;
}

/* SEARCH-LAYER: beam search with ef on layer lc from the entry set W (sorted,
 * len *wlen).  Result in W (ascending, at most ef). */
static void search_layer(hnsw_t* h, const double* q, kv_t* W, int* wlen, int ef, int lc,
                         kv_t* C, int ccap) {
    h->cur_stamp++;
    int clen = 0;
    for (int i = 0; i < *wlen; ++i) {
        h->stamp[W[i].id] = h->cur_stamp;
        sorted_insert(C, &clen, ccap, W[i]);
    }
    int chead = 0;
    while (chead < clen) {
        kv_t c = C[chead++];
        kv_t f = W[*wlen - 1];
        if (kv_less(f, c)) break;
        int32_t* cnt;
        int32_t* nb = links(h, c.id, lc, &cnt);
        for (int j = 0; j < *cnt; ++j) {
            int32_t e = nb[j];
            if (h->stamp[e] == h->cur_stamp) continue;
            h->stamp[e] = h->cur_stamp;
            kv_t x = {l2sq(q, h->X + (size_t)e * h->m, h->m), e};
            f = W[*wlen - 1];
            if (*wlen < ef || kv_less(x, f)) {
                /* C is consumed from the front; keep the unconsumed part sorted */
                if (clen == ccap) {
                    memmove(C, C + chead, sizeof(kv_t) * (size_t)(clen - chead));
                    clen -= chead;
                    chead = 0;
                }
                int p = clen;
                while (p > chead && kv_less(x, C[p - 1])) {
                    C[p] = C[p - 1];
                    --p;
                }
                C[p] = x;
                clen++;
                sorted_insert(W, wlen, ef, x);
            }
        }
    }
}

/* heuristic neighbour selection: walk candidates in ascending order, keep e iff
 * it is closer to the base point than to every element already kept. */
static int select_heuristic(hnsw_t* h, const kv_t* cand, int nc, int Mmax, int32_t* out) {
    int k = 0;
    for (int i = 0; i < nc && k < Mmax; ++i) {
        const double* xe = h->X + (size_t)cand[i].id * h->m;
        int good = 1;
        for (int j = 0; j < k; ++j) {
            double der = l2sq(xe, h->X + (size_t)out[j] * h->m, h->m);
            if (!(cand[i].d < der)) {
                good = 0;
                break;
            }
        }
        if (good) out[k++] = cand[i].id;
    }
    return k;
}

int orc_hnsw_build(const double* X, int64_t n, int m, int M, int efC, const int32_t* level,
                   const int64_t* up_off, int64_t up_rows, int32_t* adj0, int32_t* up_adj,
                   int32_t* entry_out, int32_t* maxlevel_out) {
    hnsw_t h;
    h.X = X;
    h.n = n;
    h.m = m;
    h.M = M;
    h.deg0 = 2 * M;
    h.adj0 = adj0;
    h.up_off = up_off;
    h.up_adj = up_adj;
    h.cnt0 = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    h.cntu = (int32_t*)calloc((size_t)(up_rows > 0 ? up_rows : 1), sizeof(int32_t));
    h.stamp = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    h.cur_stamp = 0;
    for (int64_t i = 0; i < n * h.deg0; ++i) adj0[i] = -1;
    for (int64_t i = 0; i < up_rows * M; ++i) up_adj[i] = -1;

    int wcap = efC + 1;
    int ccap = (int)n + 1;
    kv_t* W = (kv_t*)malloc(sizeof(kv_t) * (size_t)wcap);
    kv_t* C = (kv_t*)malloc(sizeof(kv_t) * (size_t)ccap);
    kv_t* tmp = (kv_t*)malloc(sizeof(kv_t) * (size_t)(h.deg0 + 2));
    int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h.deg0 + 2));
    int32_t* sel2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h.deg0 + 2));

    int32_t entry = 0;
    int L = n > 0 ? level[0] : 0;
    for (int64_t i = 1; i < n; ++i) {
        const double* q = X + (size_t)i * m;
        int l = level[i];
        int wlen = 1;
        W[0].id = entry;
        W[0].d = l2sq(q, X + (size_t)entry * m, m);
        for (int lc = L; lc > l; --lc) {
            search_layer(&h, q, W, &wlen, 1, lc, C, ccap);
        }
        for (int lc = (l < L ? l : L); lc >= 0; --lc) {
            search_layer(&h, q, W, &wlen, efC, lc, C, ccap);
            int Mmax = lc == 0 ? h.deg0 : M;
            int k = select_heuristic(&h, W, wlen, M, sel);
            int32_t* cnt;
            int32_t* li = links(&h, i, lc, &cnt);
            for (int j = 0; j < k; ++j) li[j] = sel[j];
            *cnt = k;
            for (int j = 0; j < k; ++j) {
                int32_t e = sel[j];
                int32_t* ce;
                int32_t* le = links(&h, e, lc, &ce);
                if (*ce < Mmax) {
                    le[(*ce)++] = (int32_t)i;
                    continue;
                }
                const double* xe = X + (size_t)e * m;
                int nc = 0;
                for (int t = 0; t < *ce; ++t) {
                    tmp[nc].id = le[t];
                    tmp[nc].d = l2sq(xe, X + (size_t)le[t] * m, m);
                    nc++;
                }
                tmp[nc].id = (int32_t)i;
                tmp[nc].d = l2sq(xe, q, m);
                nc++;
                qsort(tmp, (size_t)nc, sizeof(kv_t), kv_cmp);
                int kk = select_heuristic(&h, tmp, nc, Mmax, sel2);
                for (int t = 0; t < Mmax; ++t) le[t] = t < kk ? sel2[t] : -1;
                *ce = kk;
            }
        }
        if (l > L) {
            L = l;
            entry = (int32_t)i;
        }
    }
    *entry_out = entry;
    *maxlevel_out = L;
    free(W);
    free(C);
    free(tmp);
    free(sel);
    free(sel2);
    free(h.cnt0);
    free(h.cntu);
    free(h.stamp);
    return 0;
}

/* --------------------------------------------------------------- search */

enum { CNT_EXPANSIONS = 0, CNT_EXAMINED, CNT_ESTIMATES, CNT_SKIPPED, CNT_EXACT, CNT_ADMITTED,
       CNT_UPPER, CNT_N = 8 };

typedef struct {
    kv_t kv;
    int expanded;
} tent_t;

/* round to the nearest IEEE binary16 value, ties to even, directly from FP64
 * (11 significant bits; spacing 2^-24 below the smallest normal 2^-14; no
 * overflow handling: the codes are components of unit vectors) */
static double half_rne(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(fabs(x), &e);              /* |x| in [2^(e-1), 2^e) */
    int q = e - 11;                  /* spacing of binary16 values there */
    if (q < -24) q = -24;
    const double sp = ldexp(1.0, q);
    return nearbyint(x / sp) * sp;   /* the default rounding mode: ties to even */
}

double orc_half_round(double x) { return half_rne(x); }

/* round to the nearest FP8 E4M3 value (ties to even), saturating at +-448:
 * 4 exponent bits with bias 7 and 3 fraction bits, so the values in
 * [2^e, 2^(e+1)) are spaced 2^(e-3) for e >= -6, and below 2^-6 the
 * subnormals are spaced 2^-9 */
static double e4m3_rne(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(fabs(x), &e);              /* |x| in [2^(e-1), 2^e) */
    int q = e - 4;
    if (q < -9) q = -9;
    const double sp = ldexp(1.0, q);
    double v = nearbyint(x / sp) * sp;
    if (v > 448.0) v = 448.0;
    if (v < -448.0) v = -448.0;
    return v;
}

double orc_e4m3_round(double x) { return e4m3_rne(x); }

/* round to the nearest bfloat16 (ties to even) through FP32 */
static double bf16r(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* learned angle predictor r+4 -> 64 -> 64 -> 1 (weights already BF16/FP32
 * valued; W1 64 x nf, b1, W2 64 x 64, b2, w3, b3), hidden-layer inputs rounded
 * to BF16 as a tensor-core operand would be */
static double mlp_predict(const double* w, int nf, const double* f) {
    const double* W1 = w;
    const double* b1 = W1 + 64 * nf;
    const double* W2 = b1 + 64;
    const double* b2 = W2 + 64 * 64;
    const double* w3 = b2 + 64;
    double b3 = w3[64];
    double x[80], h1[64];
    for (int i = 0; i < nf; ++i) x[i] = bf16r(f[i]);
    for (int j = 0; j < 64; ++j) {
        double z = b1[j];
        for (int i = 0; i < nf; ++i) z += W1[j * nf + i] * x[i];
        h1[j] = bf16r(z > 0 ? z : 0.0);
    }
    double y = b3;
    for (int j = 0; j < 64; ++j) {
        double z = b2[j];
        for (int i = 0; i < 64; ++i) z += W2[j * 64 + i] * h1[i];
        y += w3[j] * (z > 0 ? z : 0.0);
    }
    return y;
}

/* Algorithm 3 for one neighbour d of centre c, given the per-centre parts
 * q_proj, q_res (Eq. 1), ||q_res||^2 and P q_res.  Returns the distance
 * estimate of Eq. (2) with q_res^T d_res replaced by ||q_res|| ||d_res|| t,
 * t = (t_hat - mu_hat) sigma / sigma_hat + mu + eps, t_hat = cos(P q_res, P d_res). */
static double appx_dist(const double* xc, const double* xd, int m, double cc, const double* q_proj,
                        const double* q_res, double qres_n2, const double* Pq, const double* P,
                        int r, const double* st, double* d_proj, double* d_res, double* diff,
                        double* Pd, const double* q, const double* mlp, double mlp_eps,
                        double* f_out, double* y_out, int codes, int full_c, double ub_c,
                        double mlp_delta) {
    double mu = st[0], sigma = st[1], muh = st[2], sigmah = st[3], eps = st[4];
    double ratio = sigmah > 0 ? sigma / sigmah : 0.0;
    double b = cc > 0 ? dot(xc, xd, m) / cc : 0.0;
    for (int i = 0; i < m; ++i) {
        d_proj[i] = b * xc[i];
        d_res[i] = xd[i] - d_proj[i];
        diff[i] = q_proj[i] - d_proj[i];
    }
    double dres_n2 = dot(d_res, d_res, m);
    for (int k = 0; k < r; ++k) Pd[k] = dot(P + (size_t)k * m, d_res, m);
    double nq_ = sqrt(dot(Pq, Pq, r)), nd_ = sqrt(dot(Pd, Pd, r));
    double that = (nq_ > 0 && nd_ > 0) ? dot(Pq, Pd, r) / (nq_ * nd_) : 0.0;
    if (codes == 16 && nq_ > 0 && nd_ > 0) {
        /* the stored code of the edge is its unit P d_res rounded to binary16;
         * t_hat is its dot with the unit P q_res */
        that = 0.0;
        for (int k = 0; k < r; ++k) that += (Pq[k] / nq_) * half_rne(Pd[k] / nd_);
    }
    if (codes == 8 && nq_ > 0 && nd_ > 0) {
        /* the stored code is 256 times the unit P d_res rounded to FP8 E4M3;
         * 256 times the unit P q_res enters as its E4M3 rounding h plus the
         * E4M3 rounding of the remainder */
        that = 0.0;
        for (int k = 0; k < r; ++k) {
            const double s = 256.0 * Pq[k] / nq_;
            const double h = e4m3_rne(s);
            that += e4m3_rne(256.0 * Pd[k] / nd_) * (h + e4m3_rne(s - h));
        }
        that /= 65536.0;
    }
    if (codes == 9 && nq_ > 0 && nd_ > 0) {
        /* the same FP8 codes against the unit P q_res itself */
        that = 0.0;
        for (int k = 0; k < r; ++k) that += (Pq[k] / nq_) * e4m3_rne(256.0 * Pd[k] / nd_);
        that /= 256.0;
    }
    double t = (that - muh) * ratio + mu;
    t = t + eps;
    int use_mlp = mlp != NULL;
    if (use_mlp && mlp_delta >= 0) {
        /* gated predictor (extension): only where the matched estimate lies
         * within mlp_delta * ub of the ub at the start of the expansion, and
         * only when the result list was full then */
        double est_m = dot(diff, diff, m) + qres_n2 + dres_n2 -
                       2.0 * sqrt(qres_n2) * sqrt(dres_n2) * t;
        use_mlp = full_c && fabs(est_m - ub_c) <= mlp_delta * ub_c;
    }
    if (use_mlp) {
        /* learned predictor in place of distribution matching (extension) */
        double f[80];
        double a = cc > 0 ? dot(xc, q, m) / cc : 0.0;
        for (int k = 0; k < r; ++k)
            f[k] = (nq_ > 0 && nd_ > 0) ? (Pq[k] / nq_) * (Pd[k] / nd_) : 0.0;
        double nqn = sqrt(dot(q, q, m)), ndn = sqrt(dot(xd, xd, m));
        f[r] = that;
        f[r + 1] = nqn > 0 ? sqrt(qres_n2) / nqn : 0.0;
        f[r + 2] = ndn > 0 ? sqrt(dres_n2) / ndn : 0.0;
        f[r + 3] = a / (fabs(a) + fabs(b) + 1e-6);
        double y = mlp_predict(mlp, r + 4, f);
        if (f_out)
            for (int k = 0; k < r + 4; ++k) f_out[k] = f[k];
        if (y_out) *y_out = y;
        if (isfinite(y)) t = y + mlp_eps;
    }
    (void)q_res;
    return dot(diff, diff, m) + qres_n2 + dres_n2 - 2.0 * sqrt(qres_n2) * sqrt(dres_n2) * t;
}

/* per-centre parts of Algorithm 3: q_proj, q_res, ||q_res||^2, P q_res; returns c^T c */
static double centre_parts(const double* xc, const double* q, int m, const double* P, int r,
                           double* q_proj, double* q_res, double* qres_n2, double* Pq) {
    double cc = dot(xc, xc, m);
    double a = cc > 0 ? dot(xc, q, m) / cc : 0.0;
    for (int i = 0; i < m; ++i) {
        q_proj[i] = a * xc[i];
        q_res[i] = q[i] - q_proj[i];
    }
    *qres_n2 = dot(q_res, q_res, m);
    for (int k = 0; k < r; ++k) Pq[k] = dot(P + (size_t)k * m, q_res, m);
    return cc;
}

/* Algorithm 3 on one (q, c, d) triple, exposed for tests. */
double orc_estimate(const double* q, const double* xc, const double* xd, int m, const double* P,
                    int r, const double* stats, int codes) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(6 * m + 2 * r + 2));
    double* q_proj = w;
    double* q_res = w + m;
    double* d_proj = w + 2 * m;
    double* d_res = w + 3 * m;
    double* diff = w + 4 * m;
    double* Pq = w + 5 * m;
    double* Pd = Pq + r;
    double qres_n2;
    double cc = centre_parts(xc, q, m, P, r, q_proj, q_res, &qres_n2, Pq);
    double e = appx_dist(xc, xd, m, cc, q_proj, q_res, qres_n2, Pq, P, r, stats, d_proj, d_res,
                         diff, Pd, q, NULL, 0.0, NULL, NULL, codes, 0, 0.0, -1.0);
    free(w);
    return e;
}

/* Algorithm 3 with the learned predictor in place of distribution matching
 * (extension), exposed for tests: the r + 4 features the predictor saw go to
 * f_out, its raw output to y_out; returns the estimate. */
double orc_estimate_mlp(const double* q, const double* xc, const double* xd, int m,
                        const double* P, int r, const double* stats, const double* mlp,
                        double mlp_eps, double* f_out, double* y_out) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(6 * m + 2 * r + 2));
    double* q_proj = w;
    double* q_res = w + m;
    double* d_proj = w + 2 * m;
    double* d_res = w + 3 * m;
    double* diff = w + 4 * m;
    double* Pq = w + 5 * m;
    double* Pd = Pq + r;
    double qres_n2;
    double cc = centre_parts(xc, q, m, P, r, q_proj, q_res, &qres_n2, Pq);
    double e = appx_dist(xc, xd, m, cc, q_proj, q_res, qres_n2, Pq, P, r, stats, d_proj, d_res,
                         diff, Pd, q, mlp, mlp_eps, f_out, y_out, 0, 0, 0.0, -1.0);
    free(w);
    return e;
}

/* one query: descent on levels maxlevel..1, then Algorithm 1 (finger == 0) or
 * Algorithm 4 (finger == 1) on layer 0 */
static void search_one(const double* X, int m, const int32_t* adj0, int deg0, const int64_t* up_off,
                       const int32_t* up_adj, int Mup, int entry, int maxlevel, const double* q,
                       int K, int ef, const double* P, int r, const double* st, int warmup,
                       int finger, int64_t* out_ids, double* out_d, int64_t* cnt, char* visited,
                       int32_t* touched, tent_t* T, double* work, const double* mlp,
                       double mlp_eps, int codes, double mlp_delta) {
    for (int i = 0; i < CNT_N; ++i) cnt[i] = 0;
    /* ---- upper layers: greedy descent (search-layer with ef = 1) */
    int32_t cur = entry;
    double dcur = l2sq(q, X + (size_t)cur * m, m);
    cnt[CNT_UPPER]++;
    for (int lc = maxlevel; lc >= 1; --lc) {
        for (;;) {
            kv_t best = {dcur, cur};
            const int32_t* row = up_adj + (size_t)(up_off[cur] + lc - 1) * Mup;
            for (int j = 0; j < Mup; ++j) {
                if (row[j] < 0) continue;
                kv_t x = {l2sq(q, X + (size_t)row[j] * m, m), row[j]};
                cnt[CNT_UPPER]++;
                if (kv_less(x, best)) best = x;
            }
            if (best.id == cur) break;
            cur = best.id;
            dcur = best.d;
        }
    }

    /* ---- layer 0 */
    double* q_proj = work;
    double* q_res = work + m;
    double* d_proj = work + 2 * m;
    double* d_res = work + 3 * m;
    double* diff = work + 4 * m;
    double* Pq = work + 5 * m;
    double* Pd = Pq + r;

    int ntouch = 0;
    int tlen = 1;
    T[0].kv.d = dcur;
    T[0].kv.id = cur;
    T[0].expanded = 0;
    visited[cur] = 1;
    touched[ntouch++] = cur;
    int64_t expansions = 0;

    for (;;) {
        int ci = -1;
        for (int i = 0; i < tlen; ++i)
            if (!T[i].expanded) {
                ci = i;
                break;
            }
        if (ci < 0) break;                       /* C is empty */
        if (kv_less(T[tlen - 1].kv, T[ci].kv)) break; /* dist(cur) > ub */
        T[ci].expanded = 1;
        int32_t c = T[ci].kv.id;
        expansions++;
        const double* xc = X + (size_t)c * m;
        int use_est = finger && expansions > warmup;
        /* the upper bound when this centre is expanded (gated predictor) */
        const int full_c = tlen == ef;
        const double ub_c = T[tlen - 1].kv.d;
        double cc = 0, qres_n2 = 0;
        if (use_est) cc = centre_parts(xc, q, m, P, r, q_proj, q_res, &qres_n2, Pq);
        const int32_t* row = adj0 + (size_t)c * deg0;
        for (int j = 0; j < deg0; ++j) {
            int32_t nb = row[j];
            if (nb < 0) continue;
            if (visited[nb]) continue;
            visited[nb] = 1;
            touched[ntouch++] = nb;
            cnt[CNT_EXAMINED]++;
            const double* xd = X + (size_t)nb * m;
            int full = tlen == ef;
            if (use_est && full) {
                double est = appx_dist(xc, xd, m, cc, q_proj, q_res, qres_n2, Pq, P, r, st,
                                       d_proj, d_res, diff, Pd, q, mlp, mlp_eps, NULL, NULL,
                                       codes, full_c, ub_c, mlp_delta);
                cnt[CNT_ESTIMATES]++;
                double ub = T[tlen - 1].kv.d;
                if (est > ub) {
                    cnt[CNT_SKIPPED]++;
                    continue;
                }
            }
            kv_t x = {l2sq(q, xd, m), nb};
            cnt[CNT_EXACT]++;
            if (tlen < ef || kv_less(x, T[tlen - 1].kv)) {
                int p = tlen < ef ? tlen : ef - 1;
                while (p > 0 && kv_less(x, T[p - 1].kv)) {
                    if (p < ef) T[p] = T[p - 1];
                    --p;
                }
                T[p].kv = x;
                T[p].expanded = 0;
                if (tlen < ef) tlen++;
                cnt[CNT_ADMITTED]++;
            }
        }
    }
    cnt[CNT_EXPANSIONS] = expansions;
    for (int k = 0; k < K; ++k) {
        out_ids[k] = k < tlen ? T[k].kv.id : -1;
        out_d[k] = k < tlen ? T[k].kv.d : INFINITY;
    }
    for (int i = 0; i < ntouch; ++i) visited[touched[i]] = 0;
}

int orc_search(const double* X, int64_t n, int m, const int32_t* adj0, int deg0,
               const int64_t* up_off, const int32_t* up_adj, int Mup, int entry, int maxlevel,
               const double* Q, int64_t nq, int K, int ef, const double* P, int r,
               const double* stats, int warmup, int finger, int64_t* ids, double* dists,
               int64_t* counters, int nthreads, const double* mlp, double mlp_eps, int codes,
               double mlp_delta) {
    if (ef < 1 || K < 1) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        char* visited = (char*)calloc((size_t)n, 1);
        int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        tent_t* T = (tent_t*)malloc(sizeof(tent_t) * (size_t)(ef + 1));
        double* work = (double*)malloc(sizeof(double) * (size_t)(5 * m + 2 * (r > 0 ? r : 1)));
        int64_t cnt_local[CNT_N];
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t qi = 0; qi < nq; ++qi) {
            search_one(X, m, adj0, deg0, up_off, up_adj, Mup, entry, maxlevel, Q + (size_t)qi * m,
                       K, ef, P, r, stats, warmup, finger, ids + qi * K, dists + qi * K,
                       counters ? counters + qi * CNT_N : cnt_local, visited, touched, T, work,
                       mlp, mlp_eps, codes, mlp_delta);
        }
        free(visited);
        free(touched);
        free(T);
        free(work);
    }
    return 0;
}

/* ------------------------------------------------------ Algorithm 2 sampling */

/* For every node c with at least two layer-0 neighbours, draw an ordered pair of
 * distinct neighbours (d, d') from the counter h1 = splitmix64(seed ^ (c*spn+k)),
 * h2 = splitmix64(h1): i = h1 mod deg, j = h2 mod (deg-1), j += (j >= i).
 * out has n*spn rows (c, d, d'); rows of nodes with deg < 2 hold -1. */
void orc_sample_pairs(const int32_t* adj0, int64_t n, int deg0, uint64_t seed, int spn,
                      int32_t* out) {
    for (int64_t c = 0; c < n; ++c) {
        const int32_t* row = adj0 + (size_t)c * deg0;
        int32_t valid[1024];
        int deg = 0;
        for (int j = 0; j < deg0 && j < 1024; ++j)
            if (row[j] >= 0) valid[deg++] = row[j];
        for (int k = 0; k < spn; ++k) {
            int32_t* o = out + (size_t)(c * spn + k) * 3;
            if (deg < 2) {
                o[0] = o[1] = o[2] = -1;
                continue;
            }
            uint64_t h1 = orc_splitmix64(seed ^ (uint64_t)(c * spn + k));
            uint64_t h2 = orc_splitmix64(h1);
            int i = (int)(h1 % (uint64_t)deg);
            int j = (int)(h2 % (uint64_t)(deg - 1));
            if (j >= i) j++;
            /* i, j index the valid entries of the row, in row order */
            o[0] = (int32_t)c;
            o[1] = valid[i];
            o[2] = valid[j];
        }
    }
}
