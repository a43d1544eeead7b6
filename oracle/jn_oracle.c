/*
 * jn_oracle.c -- plain CPU reference for the join path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table
 * or helper with the CUDA path.  Every function is the plain definition of
 * what it computes (or the paper's algorithm step by step), written to be
 * checked by eye against the paper, not to be fast.
 *
 * Paper: H. Wang, N. Li, Z. Wang, J. Li, "GPU-based Efficient Join
 * Algorithms on Hadoop" (arXiv 1904.11201).  Citations name its sections,
 * equations and algorithms.
 *
 * Conventions shared by every function (they follow the paper's statement
 * of the problem):
 *   - A table is a set of column buffers in the same row order (Sec. 3.2.2,
 *     row and column transformation).  key[] is the join key, key2[] the
 *     second compared column (band / two-column predicates), pay[] the
 *     payload; pay == NULL means the payload is the row index.
 *   - A match of row m of R (the paper's T) with row n of S yields the
 *     pair (pay_R[m], pay_S[n]) (Sec. 3.2.2: "extract ... all m-th records of
 *     T ... and all n-th records of S").
 *   - Keys are signed int32 (ksize 4) or int64 (ksize 8).
 *   - Predicates compare R's column with S's column: R.x op S.x.  The
 *     paper lists =, >, <, >=, <= "and so on" (Sec. 2.3) and shows != in its
 *     region figure (Sec. 4.2); ANY is the always-true predicate.
 *   - band >= 0 replaces the key2 comparison by |R.k - S.k| <= band, computed
 *     exactly in 128-bit integers.
 *   - Functions that emit pairs take (out, cap): at most cap pairs are
 *     written, and the return value is the total number of matches.
 *
 * Parity: every function here is pinned by the not-gpu tests against
 * brute force in pure Python, closed forms, or invariants; none is "parity
 * unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EQ 0
#define OR_NE 1
#define OR_LT 2
#define OR_LE 3
#define OR_GT 4
#define OR_GE 5
#define OR_ANY 6

typedef struct {
    int32_t r;
    int32_t s;
} or_pair;

typedef __int128 i128;

static int64_t key_at(const void* keys, int ksize, int64_t i) {
    if (ksize == 8) return ((const int64_t*)keys)[i];
    return (int64_t)((const int32_t*)keys)[i];
}

static int32_t pay_at(const int32_t* pay, int64_t i) {
    return pay ? pay[i] : (int32_t)i;
}

/* R.x op S.x for one pair of values (Sec. 2.3). */
static int compare(int op, int64_t x, int64_t y) {
    switch (op) {
    case OR_EQ: return x == y;
    case OR_NE: return x != y;
    case OR_LT: return x < y;
    case OR_LE: return x <= y;
    case OR_GT: return x > y;
    case OR_GE: return x >= y;
    case OR_ANY: return 1;
    default: return 0;
    }
}

/* |x - y| <= band, exactly (no overflow for any int64 pair). */
static int within_band(int64_t x, int64_t y, int64_t band) {
    i128 d = (i128)x - (i128)y;
    if (d < 0) d = -d;
    return d <= (i128)band;
}

static void put(or_pair* out, uint64_t cap, uint64_t idx, int32_t r, int32_t s) {
    if (out && idx < cap) {
        out[idx].r = r;
        out[idx].s = s;
    }
}

/* ------------------------------------------------------------------------ *
 * O1 / O3: nested-loop join (Sec. 2.3, "Nested loop join": every tuple of one
 * table is compared with every tuple of the other).  R is the outer loop,
 * S the inner loop.  The predicate is
 *     (R.key op_a S.key) AND (band >= 0 ? |R.key2 - S.key2| <= band
 *                                       : R.key2 op_k S.key2)
 * where a NULL key2 on either side makes the second conjunct true.
 * ------------------------------------------------------------------------ */
uint64_t or_nested_loop(const void* rkey, const void* rkey2, const int32_t* rpay, int64_t nr,
                        const void* skey, const void* skey2, const int32_t* spay, int64_t ns,
                        int ksize, int op_a, int op_k, int64_t band,
                        or_pair* out, uint64_t cap) {
    uint64_t cnt = 0;
    int has2 = (rkey2 != NULL && skey2 != NULL);
    for (int64_t m = 0; m < nr; m++) {
        int64_t ra = key_at(rkey, ksize, m);
        for (int64_t n = 0; n < ns; n++) {
            int64_t sa = key_at(skey, ksize, n);
            if (!compare(op_a, ra, sa)) continue;
            if (has2) {
                int64_t rk = key_at(rkey2, ksize, m);
                int64_t sk = key_at(skey2, ksize, n);
                if (band >= 0) {
                    if (!within_band(rk, sk, band)) continue;
                } else if (!compare(op_k, rk, sk)) {
                    continue;
                }
            }
            put(out, cap, cnt, pay_at(rpay, m), pay_at(spay, n));
            cnt++;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ *
 * O2: chained hash join (Sec. 2.3, "Hash join": put the smaller (inner)
 * table R into a hash table, then traverse the larger table S and look each
 * tuple up).  Buckets are explicit chains; the bucket of a key is its
 * unsigned value modulo an odd bucket count.  Equality predicate only.
 * ------------------------------------------------------------------------ */
uint64_t or_hash_join(const void* rkey, const int32_t* rpay, int64_t nr,
                      const void* skey, const int32_t* spay, int64_t ns,
                      int ksize, or_pair* out, uint64_t cap) {
    uint64_t nb = (uint64_t)(2 * nr + 1);
    int64_t* head = (int64_t*)malloc(nb * sizeof(int64_t));
    int64_t* next = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    uint64_t cnt = 0;
    if (!head || !next) {
        free(head);
        free(next);
        return UINT64_MAX;
    }
    for (uint64_t b = 0; b < nb; b++) head[b] = -1;
    /* build on R */
    for (int64_t m = 0; m < nr; m++) {
        uint64_t b = (uint64_t)key_at(rkey, ksize, m) % nb;
        next[m] = head[b];
        head[b] = m;
    }
    /* probe with S, in order */
    for (int64_t n = 0; n < ns; n++) {
        int64_t sk = key_at(skey, ksize, n);
        uint64_t b = (uint64_t)sk % nb;
        for (int64_t m = head[b]; m != -1; m = next[m]) {
            if (key_at(rkey, ksize, m) == sk) {
                put(out, cap, cnt, pay_at(rpay, m), pay_at(spay, n));
                cnt++;
            }
        }
    }
    free(head);
    free(next);
    return cnt;
}

/* ---------------------------- sorting helpers --------------------------- */

/* Sort an index array by (primary value, index) with a plain merge sort. */
static void msort_idx(int64_t* idx, int64_t* tmp, const int64_t* val, int64_t lo, int64_t hi) {
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    msort_idx(idx, tmp, val, lo, mid);
    msort_idx(idx, tmp, val, mid, hi);
    int64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi) {
        int64_t a = idx[i], b = idx[j];
        if (val[a] < val[b] || (val[a] == val[b] && a <= b))
            tmp[k++] = idx[i++];
        else
            tmp[k++] = idx[j++];
    }
    while (i < mid) tmp[k++] = idx[i++];
    while (j < hi) tmp[k++] = idx[j++];
    for (k = lo; k < hi; k++) idx[k] = tmp[k];
}

/* Returns a newly allocated array of row indices of the column, sorted by value. */
static int64_t* sorted_order(const void* keys, int ksize, int64_t n, int64_t** vals_out) {
    int64_t* val = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* idx = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* tmp = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        val[i] = key_at(keys, ksize, i);
        idx[i] = i;
    }
    msort_idx(idx, tmp, val, 0, n);
    free(tmp);
    *vals_out = val;
    return idx;
}

/* ------------------------------------------------------------------------ *
 * O5: sort-merge equi join, the third join category of Sec. 2.3: sort both
 * tables on the key, then walk the two sorted sequences together; a run of
 * equal keys in R meets the run of the same key in S as their cross product.
 * Same conventions and return value as or_hash_join.
 * ------------------------------------------------------------------------ */
uint64_t or_sort_merge_join(const void* rkey, const int32_t* rpay, int64_t nr,
                            const void* skey, const int32_t* spay, int64_t ns,
                            int ksize, or_pair* out, uint64_t cap) {
    int64_t *rv, *sv;
    int64_t* ri = sorted_order(rkey, ksize, nr, &rv);
    int64_t* si = sorted_order(skey, ksize, ns, &sv);
    uint64_t cnt = 0;
    int64_t i = 0, j = 0;
    while (i < nr && j < ns) {
        const int64_t a = rv[ri[i]], b = sv[si[j]];
        if (a < b) {
            i++;
        } else if (b < a) {
            j++;
        } else {
            int64_t i1 = i, j1 = j;  /* the two runs of key a */
            while (i1 < nr && rv[ri[i1]] == a) i1++;
            while (j1 < ns && sv[si[j1]] == a) j1++;
            for (int64_t x = i; x < i1; x++)
                for (int64_t y = j; y < j1; y++) {
                    put(out, cap, cnt, pay_at(rpay, ri[x]), pay_at(spay, si[y]));
                    cnt++;
                }
            i = i1;
            j = j1;
        }
    }
    free(ri);
    free(si);
    free(rv);
    free(sv);
    return cnt;
}

/* ------------------------------------------------------------------------ *
 * The separable checksum used to compare result sets too large to store
 * (Sec. 5.3 runs large theta joins "without storing the results").  For a
 * result multiset M of pairs (r, s):
 *     C = sum over (r, s) in M of f(r) * g(s)   (mod 2^64)
 * with f(x) = mix(0x243F6A8885A308D3 ^ (uint32)x),
 *      g(x) = mix(0x13198A2E03707344 ^ (uint32)x),
 * mix = the SplitMix64 output mixer (Steele, Lea & Flood 2014).
 * ------------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t or_mix64(uint64_t z) { return mix64(z); }

uint64_t or_f(int32_t r) { return mix64(0x243F6A8885A308D3ULL ^ (uint64_t)(uint32_t)r); }
uint64_t or_g(int32_t s) { return mix64(0x13198A2E03707344ULL ^ (uint64_t)(uint32_t)s); }

uint64_t or_checksum_pairs(const or_pair* p, uint64_t n) {
    uint64_t c = 0;
    for (uint64_t i = 0; i < n; i++) c += or_f(p[i].r) * or_g(p[i].s);
    return c;
}

/* ------------------------------------------------------------------------ *
 * Closed-form equi-join size and checksum, without any join: group both
 * tables by key value and sum, over the keys present in both,
 *     count    += c_R(k) * c_S(k)
 *     checksum += (sum of f(pay_R) over R rows with key k)
 *               * (sum of g(pay_S) over S rows with key k).
 * This is the per-group Cartesian product that Eq. (rsize) sums over
 * reducers (Sec. 3.3.3) taken at one key per group, where it is exact.
 * ------------------------------------------------------------------------ */
void or_equi_count_checksum(const void* rkey, const int32_t* rpay, int64_t nr,
                            const void* skey, const int32_t* spay, int64_t ns,
                            int ksize, uint64_t* count, uint64_t* checksum) {
    int64_t *rv, *sv;
    int64_t* ri = sorted_order(rkey, ksize, nr, &rv);
    int64_t* si = sorted_order(skey, ksize, ns, &sv);
    uint64_t cnt = 0, chk = 0;
    int64_t i = 0, j = 0;
    while (i < nr && j < ns) {
        int64_t a = rv[ri[i]], b = sv[si[j]];
        if (a < b) {
            i++;
        } else if (b < a) {
            j++;
        } else {
            uint64_t cr = 0, cs = 0, fr = 0, gs = 0;
            while (i < nr && rv[ri[i]] == a) {
                fr += or_f(pay_at(rpay, ri[i]));
                cr++;
                i++;
            }
            while (j < ns && sv[si[j]] == a) {
                gs += or_g(pay_at(spay, si[j]));
                cs++;
                j++;
            }
            cnt += cr * cs;
            chk += fr * gs;
        }
    }
    free(rv);
    free(sv);
    free(ri);
    free(si);
    *count = cnt;
    *checksum = chk;
}

/* ------------------------------------------------------------------------ *
 * O4: band join by sorting (the sort-merge idea of Sec. 2.3 applied to a band
 * predicate).  Predicate: (R.key op_a S.key) AND |R.key2 - S.key2| <= band.
 * S is sorted by key2; for every R row the S rows with key2 in
 * [R.key2 - band, R.key2 + band] are found by binary search and each is
 * tested with op_a.
 * ------------------------------------------------------------------------ */
uint64_t or_band_join_sorted(const void* rkey, const void* rkey2, const int32_t* rpay, int64_t nr,
                             const void* skey, const void* skey2, const int32_t* spay, int64_t ns,
                             int ksize, int op_a, int64_t band, or_pair* out, uint64_t cap) {
    if (band < 0) return UINT64_MAX;
    int64_t* sv;
    int64_t* si = sorted_order(skey2, ksize, ns, &sv);
    uint64_t cnt = 0;
    for (int64_t m = 0; m < nr; m++) {
        int64_t rk = key_at(rkey2, ksize, m);
        int64_t ra = key_at(rkey, ksize, m);
        i128 lo = (i128)rk - band;
        i128 hi = (i128)rk + band;
        /* first position with key2 >= lo */
        int64_t a = 0, b = ns;
        while (a < b) {
            int64_t mid = a + (b - a) / 2;
            if ((i128)sv[si[mid]] < lo)
                a = mid + 1;
            else
                b = mid;
        }
        for (int64_t p = a; p < ns && (i128)sv[si[p]] <= hi; p++) {
            int64_t n = si[p];
            if (compare(op_a, ra, key_at(skey, ksize, n))) {
                put(out, cap, cnt, pay_at(rpay, m), pay_at(spay, n));
                cnt++;
            }
        }
    }
    free(sv);
    free(si);
    return cnt;
}

/* ------------------------------------------------------------------------ *
 * Exact band-join size by a dominance sweep with a Fenwick tree, without
 * enumerating pairs: count pairs with (R.key op_a S.key) AND
 * |R.key2 - S.key2| <= band, op_a in {<, <=, >, >=, ANY}.
 * R rows are inserted into a Fenwick tree over the ranks of their key2
 * values in the order that makes "R.key op_a S.key" a prefix condition;
 * each S row then queries the key2 window.  Returns UINT64_MAX for other ops.
 * ------------------------------------------------------------------------ */
static int64_t lower_idx(const int64_t* v, int64_t n, i128 x) { /* first v[i] >= x */
    int64_t a = 0, b = n;
    while (a < b) {
        int64_t m = a + (b - a) / 2;
        if ((i128)v[m] < x) a = m + 1; else b = m;
    }
    return a;
}

uint64_t or_band_count_sweep(const void* rkey, const void* rkey2, int64_t nr,
                             const void* skey, const void* skey2, int64_t ns,
                             int ksize, int op_a, int64_t band) {
    if (band < 0) return UINT64_MAX;
    if (op_a != OR_LT && op_a != OR_LE && op_a != OR_GT && op_a != OR_GE && op_a != OR_ANY)
        return UINT64_MAX;
    /* sorted key2 values of R for coordinate ranks */
    int64_t *k2v;
    int64_t* k2i = sorted_order(rkey2, ksize, nr, &k2v);
    int64_t* ks = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nr; i++) ks[i] = k2v[k2i[i]];
    /* rank of each R row's key2 = its position in the sorted order */
    int64_t* rank = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nr; i++) rank[k2i[i]] = i;
    uint64_t* fen = (uint64_t*)calloc((size_t)nr + 1, sizeof(uint64_t));
    int64_t *rav, *sav;
    int64_t* ra = sorted_order(rkey, ksize, nr, &rav);
    int64_t* sa = sorted_order(skey, ksize, ns, &sav);
    uint64_t total = 0;
    int desc = (op_a == OR_GT || op_a == OR_GE);
    int64_t ip = 0; /* next R row (in a-order) to insert */
    for (int64_t t = 0; t < ns; t++) {
        int64_t n = desc ? sa[ns - 1 - t] : sa[t];
        int64_t s_a = sav[n];
        /* insert every R row whose a already satisfies the op against s_a */
        while (ip < nr) {
            int64_t m = desc ? ra[nr - 1 - ip] : ra[ip];
            int64_t r_a = rav[m];
            int ok;
            if (op_a == OR_ANY) ok = 1;
            else ok = compare(op_a, r_a, s_a);
            if (!ok) break;
            for (int64_t x = rank[m] + 1; x <= nr; x += x & (-x)) fen[x]++;
            ip++;
        }
        int64_t sk = key_at(skey2, ksize, n);
        int64_t lo = lower_idx(ks, nr, (i128)sk - band);       /* first >= sk-band */
        int64_t hi = lower_idx(ks, nr, (i128)sk + band + 1);   /* first >  sk+band */
        uint64_t c = 0;
        for (int64_t x = hi; x > 0; x -= x & (-x)) c += fen[x];
        for (int64_t x = lo; x > 0; x -= x & (-x)) c -= fen[x];
        total += c;
    }
    free(k2v); free(k2i); free(ks); free(rank); free(fen);
    free(rav); free(sav); free(ra); free(sa);
    return total;
}

/* ------------------------------------------------------------------------ *
 * Algorithm 1 (pre-filtering) followed by the reducer-grouped join, taken
 * literally (Sec. 3.1, Sec. 3.3.3-3.3.4):
 *   round 1: Map1 emits (join_key, tag) for every tuple; Reduce1 keeps the
 *            keys whose tag list holds both tables (unique_key_list);
 *   round 2: Setup loads unique_key_list; Map2 keeps the tuples whose key is
 *            in it and emits them under floor(join_key / alpha); Reduce2
 *            gets T' and S' of one group and joins them (here with O1);
 *   rsize   = sum over groups of |T'_i| * |S'_i|, the storage Eq. (rsize)
 *            pre-allocates (gamma*beta*|S|*|T|*sum omega_i*lambda_i).
 * Equality predicate; alpha >= 1.  Returns the number of matches.
 * ------------------------------------------------------------------------ */
static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

static int in_sorted(const int64_t* v, int64_t n, int64_t x) {
    int64_t a = 0, b = n;
    while (a < b) {
        int64_t m = a + (b - a) / 2;
        if (v[m] < x) a = m + 1; else b = m;
    }
    return a < n && v[a] == x;
}

uint64_t or_prefilter_grouped_join(const void* rkey, const int32_t* rpay, int64_t nr,
                                   const void* skey, const int32_t* spay, int64_t ns,
                                   int ksize, int64_t alpha, or_pair* out, uint64_t cap,
                                   uint64_t* rsize, uint64_t* n_survivors) {
    if (alpha < 1) return UINT64_MAX;
    /* round 1: unique_key_list = keys present in both tables */
    int64_t *rv, *sv;
    int64_t* ri = sorted_order(rkey, ksize, nr, &rv);
    int64_t* si = sorted_order(skey, ksize, ns, &sv);
    int64_t* common = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    int64_t nc = 0;
    {
        int64_t i = 0, j = 0;
        while (i < nr && j < ns) {
            int64_t a = rv[ri[i]], b = sv[si[j]];
            if (a < b) i++;
            else if (b < a) j++;
            else {
                common[nc++] = a;
                while (i < nr && rv[ri[i]] == a) i++;
                while (j < ns && sv[si[j]] == a) j++;
            }
        }
    }
    /* round 2: keep tuples whose key is common; group key = floor(key/alpha) */
    int64_t* rk = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    int64_t* sk = (int64_t*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int64_t));
    int64_t* rg = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    int64_t* sg = (int64_t*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int64_t));
    int64_t nrk = 0, nsk = 0;
    for (int64_t m = 0; m < nr; m++)
        if (in_sorted(common, nc, rv[m])) { rk[nrk] = m; rg[m] = floor_div(rv[m], alpha); nrk++; }
    for (int64_t n = 0; n < ns; n++)
        if (in_sorted(common, nc, sv[n])) { sk[nsk] = n; sg[n] = floor_div(sv[n], alpha); nsk++; }
    *n_survivors = (uint64_t)(nrk + nsk);
    /* Reduce2: visit groups in ascending order; each group is one reducer */
    int64_t* rtmp = (int64_t*)malloc((size_t)(nrk > 0 ? nrk : 1) * sizeof(int64_t));
    int64_t* stmp = (int64_t*)malloc((size_t)(nsk > 0 ? nsk : 1) * sizeof(int64_t));
    msort_idx(rk, rtmp, rg, 0, nrk);
    msort_idx(sk, stmp, sg, 0, nsk);
    uint64_t cnt = 0, rs = 0;
    int64_t i = 0, j = 0;
    while (i < nrk && j < nsk) {
        int64_t gi = rg[rk[i]], gj = sg[sk[j]];
        if (gi < gj) { i++; continue; }
        if (gj < gi) { j++; continue; }
        int64_t i1 = i, j1 = j;
        while (i1 < nrk && rg[rk[i1]] == gi) i1++;
        while (j1 < nsk && sg[sk[j1]] == gi) j1++;
        rs += (uint64_t)(i1 - i) * (uint64_t)(j1 - j);  /* NB_T * NB_S of this reducer */
        for (int64_t a = i; a < i1; a++) {           /* Join_GPU(T', S') as O1 */
            int64_t m = rk[a];
            for (int64_t b = j; b < j1; b++) {
                int64_t n = sk[b];
                if (rv[m] == sv[n]) {
                    put(out, cap, cnt, pay_at(rpay, m), pay_at(spay, n));
                    cnt++;
                }
            }
        }
        i = i1;
        j = j1;
    }
    free(rv); free(sv); free(ri); free(si); free(common);
    free(rk); free(sk); free(rg); free(sg); free(rtmp); free(stmp);
    *rsize = rs;
    return cnt;
}

/* ------------------------------------------------------------------------ *
 * Algorithm 3 (theta join on Map-Reduce) taken literally for a one-column
 * predicate R.key op S.key (Sec. 4.2).  The key range [min, max] over both
 * tables is cut into kq equal-width ranges with the same boundaries for
 * both tables, giving a kq x kq matrix of square regions.  RegionID.x is the
 * S tuple's range and RegionID.y the R (paper: T) tuple's range.  Each
 * region is:
 *   - diagonal (x == y): joined by comparing every pair (GPU_theta_join);
 *   - always true ("x matches y according to the join condition"): the
 *     cross join, with no comparison;
 *   - always false: skipped.
 * region_kind (optional, per emitted pair) records 0 = diagonal, 1 = cross.
 * stats[3] (optional) returns the number of diagonal, cross and skipped
 * regions.
 * ------------------------------------------------------------------------ */
static int region_always_true(int op, int64_t y_r, int64_t x_s) {
    switch (op) {
    case OR_LT: case OR_LE: return y_r < x_s;   /* every R value < every S value */
    case OR_GT: case OR_GE: return y_r > x_s;
    case OR_NE: return y_r != x_s;
    case OR_ANY: return 1;
    default: return 0;                             /* OR_EQ: never off-diagonal */
    }
}

uint64_t or_theta_regions(const void* rkey, const int32_t* rpay, int64_t nr,
                          const void* skey, const int32_t* spay, int64_t ns,
                          int ksize, int op, int64_t kq, or_pair* out, uint64_t cap,
                          uint8_t* region_kind, uint64_t* stats) {
    if (kq < 1) return UINT64_MAX;
    uint64_t cnt = 0;
    uint64_t nd = 0, nt = 0, nf = 0;
    if (nr == 0 || ns == 0) {
        if (stats) { stats[0] = stats[1] = stats[2] = 0; }
        return 0;
    }
    int64_t lo = key_at(rkey, ksize, 0), hi = lo;
    for (int64_t i = 0; i < nr; i++) {
        int64_t v = key_at(rkey, ksize, i);
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    for (int64_t i = 0; i < ns; i++) {
        int64_t v = key_at(skey, ksize, i);
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    i128 span = (i128)hi - (i128)lo + 1;
    /* bucket of value v: floor((v - lo) * kq / span), in [0, kq) */
    int64_t* rb = (int64_t*)malloc((size_t)nr * sizeof(int64_t));
    int64_t* sb = (int64_t*)malloc((size_t)ns * sizeof(int64_t));
    for (int64_t i = 0; i < nr; i++)
        rb[i] = (int64_t)((((i128)key_at(rkey, ksize, i) - lo) * kq) / span);
    for (int64_t i = 0; i < ns; i++)
        sb[i] = (int64_t)((((i128)key_at(skey, ksize, i) - lo) * kq) / span);
    for (int64_t x = 0; x < kq; x++) {          /* RegionID.x: S range */
        for (int64_t y = 0; y < kq; y++) {      /* RegionID.y: R range */
            int diag = (x == y);
            int cross = !diag && region_always_true(op, y, x);
            if (diag) nd++; else if (cross) nt++; else { nf++; continue; }
            for (int64_t m = 0; m < nr; m++) {
                if (rb[m] != y) continue;
                for (int64_t n = 0; n < ns; n++) {
                    if (sb[n] != x) continue;
                    if (diag && !compare(op, key_at(rkey, ksize, m), key_at(skey, ksize, n)))
                        continue;
                    if (region_kind && cnt < cap) region_kind[cnt] = (uint8_t)(diag ? 0 : 1);
                    put(out, cap, cnt, pay_at(rpay, m), pay_at(spay, n));
                    cnt++;
                }
            }
        }
    }
    free(rb);
    free(sb);
    if (stats) { stats[0] = nd; stats[1] = nt; stats[2] = nf; }
    return cnt;
}

/* ------------------------------------------------------------------------ *
 * Thread work ranges of the paper's GPU kernels.
 *   Nested loop (Sec. 3.3.1): a grid of m x n blocks of x x y threads.
 *     NB_S = |S| / (m*x) + 1                               (Eq. NBS)
 *     ID_S = (a*x + c) * NB_S for block (a, b), thread (c, d)  (Eq. IDS)
 *   Hash join (Sec. 3.3.2): n_blocks blocks of n_threads threads.
 *     ID_S = (p*n_threads + q) * NB_S                       (Eq. IDSJ)
 * Both reduce to: thread t of T threads reads rows
 *     [t*NB, min(t*NB + NB, N)),  NB = N / T + 1,
 * with the range clamped at N (the paper's "+1" over-covers; the clamp is
 * this build's reading).  Writes T (begin, end) pairs.
 * ------------------------------------------------------------------------ */
void or_thread_ranges(int64_t n, int64_t threads, int64_t* begin, int64_t* end) {
    int64_t nb = n / threads + 1;
    for (int64_t t = 0; t < threads; t++) {
        int64_t b = t * nb;
        int64_t e = b + nb;
        if (b > n) b = n;
        if (e > n) e = n;
        begin[t] = b;
        end[t] = e;
    }
}

/* ------------------------------------------------------------------------ *
 * O6: star join of three tables (the multi-table join that Sec. 6 leaves to
 * future work, built from Sec. 2.3's definition of a join applied twice):
 * the centre table R carries two join columns, fk1 (key) and fk2 (key2);
 * every row m of R, row n1 of S1 and row n2 of S2 with
 *     R.fk1[m] == S1.key[n1]  AND  R.fk2[m] == S2.key[n2]
 * yields the triple (pay_R[m], pay_S1[n1], pay_S2[n2]).  Plain nested loops:
 * R outermost, then S1, then S2.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t r;
    int32_t s1;
    int32_t s2;
} or_triple;

uint64_t or_star_nested_loop(const void* rfk1, const void* rfk2, const int32_t* rpay, int64_t nr,
                             const void* s1key, const int32_t* s1pay, int64_t n1,
                             const void* s2key, const int32_t* s2pay, int64_t n2,
                             int ksize, or_triple* out, uint64_t cap) {
    uint64_t cnt = 0;
    for (int64_t m = 0; m < nr; m++) {
        int64_t f1 = key_at(rfk1, ksize, m);
        int64_t f2 = key_at(rfk2, ksize, m);
        for (int64_t a = 0; a < n1; a++) {
            if (key_at(s1key, ksize, a) != f1) continue;
            for (int64_t b = 0; b < n2; b++) {
                if (key_at(s2key, ksize, b) != f2) continue;
                if (out && cnt < cap) {
                    out[cnt].r = pay_at(rpay, m);
                    out[cnt].s1 = pay_at(s1pay, a);
                    out[cnt].s2 = pay_at(s2pay, b);
                }
                cnt++;
            }
        }
    }
    return cnt;
}
